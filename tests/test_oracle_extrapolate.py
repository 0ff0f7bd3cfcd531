"""Pins of the eps -> 0 extrapolation (Sec. 4.4) and of the run's truncation
error (Eq. tru, reading R6)."""
import numpy as np
import pytest

from oracle.extrapolate import quadratic_fit, run_until_converged
from oracle.idmrg import ParallelIDMRG
from workloads import build_mpo, chain_bonds, dimerized_chain_bonds


def test_exact_quadratic_is_recovered():
    x = np.array([1e-6, 3e-6, 7e-6, 2e-5, 5e-5])
    y = -0.43838 + 12.5 * x - 3.0e4 * x ** 2
    c0, sd = quadratic_fit(x, y)
    assert c0 == pytest.approx(-0.43838, abs=1e-13)
    assert sd < 1e-12


def test_standard_deviation_closed_form():
    # four points at x = 0, 1, 2, 3 with residual pattern (+1, -3, +3, -1) d
    # (orthogonal to 1, x, x^2): the fit returns the quadratic, RSS = 20 d^2,
    # s^2 = 20 d^2; A^T A = [[4,6,14],[6,14,36],[14,36,98]] has determinant 80
    # and (0,0) cofactor 76, so [(A^T A)^-1]_00 = 19/20 and sd(c0) = d sqrt(19)
    x = np.array([0.0, 1.0, 2.0, 3.0])
    d = 1e-4
    y = 2.0 - 0.5 * x + 0.25 * x ** 2 + d * np.array([1.0, -3.0, 3.0, -1.0])
    c0, sd = quadratic_fit(x, y)
    assert c0 == pytest.approx(2.0, abs=1e-12)
    assert sd == pytest.approx(d * np.sqrt(19.0), rel=1e-9)


def test_exact_mps_has_no_truncation_error():
    # the fully dimerised chain is a product of singlets: kept weight 1 at any
    # m >= 2, e_g = -3/8 per site
    ref = ParallelIDMRG.from_mpo(build_mpo(dimerized_chain_bonds(4), 4), m=4)
    e_g, eps, steps, conv = run_until_converged(ref, 40, 1e-10)
    assert conv
    assert e_g == pytest.approx(-0.375, abs=1e-12)
    assert eps < 1e-14


def test_eps_decreases_with_m_and_extrapolation_nears_bethe():
    # uniform chain: eps falls with m and the eps -> 0 estimate lies below the
    # m = 16 value, within 2e-3 of 1/4 - ln 2
    pts = []
    for m in (8, 12, 16):
        ref = ParallelIDMRG.from_mpo(build_mpo(chain_bonds(4), 4), m=m)
        e_g, eps, _, _ = run_until_converged(ref, 60, 1e-7)
        pts.append((eps, e_g))
    eps = [p[0] for p in pts]
    e = [p[1] for p in pts]
    assert eps[0] > eps[1] > eps[2] > 0.0
    e0, _ = quadratic_fit(eps, e)
    bethe = 0.25 - np.log(2.0)
    assert e0 < e[-1] + 1e-12
    assert abs(e0 - bethe) < 2e-3


def test_exponential_fit_pins():
    from oracle.extrapolate import exponential_fit
    from oracle import observables as ob
    # exact exponential: xi recovered, no spread
    r = np.arange(1, 30, dtype=float)
    xi, sd = exponential_fit(r, 0.7 * np.exp(-r / 3.25) * (-1.0) ** r, r_min=5)
    assert xi == pytest.approx(3.25, rel=1e-12) and sd < 1e-12
    # closed-form spread: ln|c| = a + b x + d (1, -2, 1) at x = 0, 1, 2 gives
    # RSS = 6 d^2, s^2 = 6 d^2, [(A^T A)^-1]_11 = 1/2, sd(b) = d sqrt(3)
    a, b, d = 0.3, -0.5, 1e-3
    x = np.array([0.0, 1.0, 2.0])
    c = np.exp(a + b * x + d * np.array([1.0, -2.0, 1.0]))
    xi, sd = exponential_fit(x, c, r_min=-1)
    assert xi == pytest.approx(2.0, rel=1e-12)
    assert sd == pytest.approx(d * np.sqrt(3.0) / b ** 2, rel=1e-9)
    # AKLT: |<S^z_0 S^z_r>| = (4/3) 3^-r, so xi = 1 / ln 3 sites
    sp = np.array([[0.0, 1.0], [0.0, 0.0]])
    A = np.array([np.sqrt(2 / 3) * sp, -np.sqrt(1 / 3) * np.diag([1.0, -1.0]), -np.sqrt(2 / 3) * sp.T])
    Sz = np.diag([1.0, 0.0, -1.0])
    rr = np.arange(1, 12)
    cc = [ob.correlation([A, A], 0, Sz, Sz, 0, int(k)) for k in rr]
    xi, _ = exponential_fit(rr, cc, r_min=0)
    assert xi == pytest.approx(1 / np.log(3.0), rel=1e-9)


def test_package_fits_match_the_oracle():
    # host post-processing of the library's outputs (no GPU): the package's
    # least-squares fits against the oracle's normal-equation versions
    from oracle.extrapolate import exponential_fit
    from paper_1606_06790_gb300.scan import extrapolate, fit_correlation_length
    rng = np.random.default_rng(5)
    r = np.arange(2, 40, dtype=float)
    c = np.exp(-r / 4.7) * (1 + 0.05 * rng.standard_normal(len(r)))
    x1, s1 = fit_correlation_length(r, c, r_min=5)
    x2, s2 = exponential_fit(r, c, r_min=5)
    assert x1 == pytest.approx(x2, rel=1e-10) and s1 == pytest.approx(s2, rel=1e-8)
    eps = np.array([1e-6, 3e-6, 7e-6, 2e-5, 5e-5])
    e = -0.43838 + 12.5 * eps - 3.0e4 * eps ** 2 + 1e-9 * rng.standard_normal(5)
    c0, sd = extrapolate(eps, e)
    q0, qsd = quadratic_fit(eps, e)
    assert c0 == pytest.approx(q0, abs=1e-12) and sd == pytest.approx(qsd, rel=1e-6)


def test_exponential_fit_needs_two_points():
    from oracle.extrapolate import exponential_fit
    from paper_1606_06790_gb300.scan import fit_correlation_length
    r = np.array([1.0, 2.0, 6.0])
    c = np.array([0.5, 0.2, 0.01])
    for fit in (exponential_fit, fit_correlation_length):
        with pytest.raises(ValueError):
            fit(r, c, r_min=5)            # one point beyond r_min
        with pytest.raises(ValueError):
            fit(r, np.zeros(3), r_min=0)  # zeros are skipped


def test_library_fits_special_cases():
    """The C ABI's host fits on cases with known answers: an exact polynomial
    of each degree is recovered at eps = 0 with zero spread; a straight line
    with residuals (1, -3, 3, -1) d at x = 0..3 (orthogonal to 1 and x) is
    recovered exactly with the closed-form spread d sqrt(7); Delta+- on given
    values."""
    import paper_1606_06790_gb300 as pkg
    from paper_1606_06790_gb300.scan import extrapolate
    x = np.linspace(0.0, 1e-4, 7)
    for deg in range(0, 4):
        coef = np.array([-0.4, 3.0, -2e4, 5e7][: deg + 1])
        y = sum(c * x ** k for k, c in enumerate(coef))
        v0, sd = extrapolate(x, y, degree=deg)
        assert v0 == pytest.approx(coef[0], abs=1e-13) and sd < 1e-11
    # line fit of y = 1 + 2x + d (1, -3, 3, -1) at x = 0..3: RSS = 20 d^2,
    # s^2 = 10 d^2, [(A^T A)^-1]_00 = 7/10, so sd(c0) = d sqrt(7)
    d = 1e-3
    xx = np.arange(4.0)
    yy = 1 + 2 * xx + d * np.array([1.0, -3.0, 3.0, -1.0])
    v0, sd = extrapolate(xx, yy, degree=1)
    assert v0 == pytest.approx(1.0 + d * (0.7 * 1 + 0.4 * -3 + 0.1 * 3 - 0.2 * -1), abs=1e-12)
    assert sd == pytest.approx(d * np.sqrt(7.0), rel=1e-9)
    avg, dp, dm = pkg.delta_pm([-0.2, -0.25, -0.21])
    assert avg == pytest.approx(-0.22, abs=1e-15) and dp == pytest.approx(0.02, abs=1e-15)
    assert dm == pytest.approx(-0.03, abs=1e-15)
    with pytest.raises(ValueError):
        pkg.delta_pm([])
