"""Pins of the eps -> 0 extrapolation (Sec. 5) and of the run's truncation
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
