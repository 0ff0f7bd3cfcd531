"""Pins of the uniform-MPS observables (Eq. mps2, readings R7-R9 of
``oracle.observables``): closed forms of the AKLT chain and of a singlet
product, the transfer spectrum of a two-state MPS in closed form, brute force
on a periodic ring, and the iDMRG states of exactly solvable chains."""
import json
import os

import numpy as np
import pytest

from oracle import observables as ob
from oracle.idmrg import ParallelIDMRG
from workloads import build_mpo, chain_bonds, dimerized_chain_bonds, j1j2_chain_bonds


def aklt_unit(copies=2):
    # Affleck, Kennedy, Lieb, Tasaki (1987): A^{+1} = sqrt(2/3) s+, A^0 = -sqrt(1/3) sz,
    # A^{-1} = -sqrt(2/3) s- with Pauli matrices; transfer spectrum {1, -1/3 (x3)}
    sp = np.array([[0.0, 1.0], [0.0, 0.0]])
    A = np.array([np.sqrt(2 / 3) * sp, -np.sqrt(1 / 3) * np.diag([1.0, -1.0]), -np.sqrt(2 / 3) * sp.T])
    return [A] * copies


SZ1 = np.diag([1.0, 0.0, -1.0])
SP1 = np.sqrt(2.0) * np.diag([1.0, 1.0], 1)


GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


def test_aklt_correlations_and_length():
    # <S^z_0 S^z_r> = (4/3)(-1/3)^r and <S_0 . S_r> = 4 (-1/3)^r for r >= 1;
    # xi = 1 / ln 3 sites = 1 / (2 ln 3) two-site unit cells
    assert GOLDEN["aklt_spin_correlation"]["xi_sites"] == pytest.approx(1 / np.log(3.0), rel=1e-15)
    unit = aklt_unit()
    for i in (0, 1, 5):
        for r in range(1, 7):
            zz = ob.correlation(unit, 0, SZ1, SZ1, i, i + r)
            pm = ob.correlation(unit, 0, SP1, SP1.T, i, i + r)
            mp = ob.correlation(unit, 0, SP1.T, SP1, i, i + r)
            assert zz == pytest.approx((4 / 3) * (-1 / 3) ** r, rel=1e-12, abs=1e-15)
            assert zz + 0.5 * (pm + mp) == pytest.approx(4 * (-1 / 3) ** r, rel=1e-12, abs=1e-15)
    assert ob.correlation_length(unit) == pytest.approx(GOLDEN["aklt_spin_correlation"]["xi_sites"] / 2, rel=1e-12)


def test_two_state_transfer_spectrum_closed_form():
    # A^0 = diag(x, y), A^1 = [[0, z], [w, 0]]: on {|00>, |11>} the transfer
    # matrix is [[x^2, w^2], [z^2, y^2]], on {|01>, |10>} [[xy, zw], [zw, xy]]
    x, y, z, w = 0.9, 0.4, 0.7, 0.3
    A = np.array([np.diag([x, y]), np.array([[0.0, z], [w, 0.0]])])
    s = np.sqrt((x * x - y * y) ** 2 + 4 * z * z * w * w)
    expect = sorted([(x * x + y * y + s) / 2, (x * x + y * y - s) / 2, x * y + z * w, x * y - z * w],
                    key=lambda v: -abs(v))
    got = ob.spectrum([A])
    assert np.max(np.abs(got.imag)) < 1e-14
    assert np.allclose(got.real, expect, rtol=0, atol=1e-14)
    assert ob.correlation_length([A]) == pytest.approx(-1 / np.log(abs(expect[1]) / expect[0]), rel=1e-12)
    lv, rv, t1 = ob.fixed_points([A])
    assert t1 == pytest.approx(expect[0], rel=1e-14)
    assert np.allclose(ob.site_left(lv, A), t1 * lv, atol=1e-14)
    assert np.allclose(ob.site_right(rv, A), t1 * rv, atol=1e-14)


def test_singlet_product():
    # singlets on (0,1), (2,3), ...: <s.s> = -3/4 inside a singlet, 0 elsewhere
    A0 = np.zeros((2, 1, 2))
    A0[0, 0, 0] = A0[1, 0, 1] = 1.0
    A1 = np.zeros((2, 2, 1))
    A1[1, 0, 0] = 1 / np.sqrt(2)
    A1[0, 1, 0] = -1 / np.sqrt(2)
    unit = [A0, A1]
    sing = GOLDEN["singlet_bond_strength"]["value"]
    for (i, j), v in {(0, 1): sing, (2, 3): sing, (1, 2): 0.0, (0, 3): 0.0, (1, 4): 0.0}.items():
        assert ob.spin_dot(unit, 0, i, j) == pytest.approx(v, abs=1e-15)


def ring_state(A, N):
    """psi(s_1..s_N) = Tr(A^s1 ... A^sN) by brute force (all d^N amplitudes)."""
    d, D = A[0].shape[0], A[0].shape[1]
    M = np.eye(D)[None]                               # [states, a, b]
    for x in range(N):
        Ak = A[x % len(A)]
        M = np.einsum("pab,sbc->psac", M, Ak).reshape(-1, D, Ak.shape[2])
    psi = np.einsum("paa->p", M).reshape([d] * N)
    return psi / np.linalg.norm(psi)


def test_transfer_walk_matches_brute_force_ring():
    # a strongly gapped random MPS (|t2/t1| ~ 0.02 per cell): on a ring of 16
    # sites the finite-size corrections are below 1e-10
    rng = np.random.default_rng(7)
    A = []
    for _ in range(2):
        a = 0.3 * rng.standard_normal((2, 2, 2))
        a[0, 0, 0] += 0.8
        a[1, 0, 0] += 0.6
        A.append(a)
    psi = ring_state(A, 16)

    def corr_ring(Oa, Ob, i, j):
        phi = np.moveaxis(np.tensordot(Ob, psi, axes=([1], [j])), 0, j)
        phi = np.moveaxis(np.tensordot(Oa, phi, axes=([1], [i])), 0, i)
        return float(np.sum(psi * phi))

    for i, j in [(0, 1), (1, 2), (0, 3), (3, 6), (2, 4)]:
        for Oa, Ob in [(ob.SZ, ob.SZ), (ob.SP, ob.SM), (ob.SM, ob.SP), (ob.SP + ob.SM, ob.SZ)]:
            assert ob.correlation(A, 0, Oa, Ob, i, j) == pytest.approx(corr_ring(Oa, Ob, i, j), abs=1e-10)


def test_delta_pm():
    avg, dp, dm = ob.delta_pm([-0.25, -0.20, -0.21, -0.22])
    assert avg == pytest.approx(-0.22, abs=1e-15)
    assert dp == pytest.approx(0.02, abs=1e-15)
    assert dm == pytest.approx(-0.03, abs=1e-15)


def converged(bonds, ell, m, steps):
    ref = ParallelIDMRG.from_mpo(build_mpo(bonds, ell), m=m)
    e_g = None
    for _ in range(steps):
        r = ref.step()
        if r.e_g is not None:
            e_g = r.e_g
    return ref, e_g


@pytest.mark.parametrize("bonds", [dimerized_chain_bonds(4), j1j2_chain_bonds(4, 1.0, 0.5)])
def test_unit_of_exact_dimer_states(bonds):
    # the dimer chain and the Majumdar-Ghosh point have singlets on (0,1),
    # (2,3): the unit (reading R7) must put -3/4 exactly there and 0 between
    ref, _ = converged(bonds, 4, 4, 12)
    A, s0 = ob.uniform_unit(ref)
    for i in range(6):
        expect = -0.75 if i % 2 == 0 else 0.0
        assert ob.spin_dot(A, s0, i, i + 1) == pytest.approx(expect, abs=1e-12)
    assert ob.spin_dot(A, s0, 0, 3) == pytest.approx(0.0, abs=1e-12)


def test_unit_bond_energies_add_up_to_e_g():
    # uniform chain: the bond strengths of one unit add up to l e_g (Step 5'),
    # up to the truncation error of m = 16
    ref, e_g = converged(chain_bonds(4), 4, 16, 40)
    A, s0 = ob.uniform_unit(ref)
    vals = [ob.spin_dot(A, s0, i, i + 1) for i in range(4)]
    assert sum(vals) / 4 == pytest.approx(e_g, abs=2e-5)
    # the unit repeats: a bond one cell further on has the same strength
    assert ob.spin_dot(A, s0, 5, 6) == pytest.approx(vals[1], abs=1e-12)
    lv, rv, t1 = ob.fixed_points(A)
    assert abs(t1 - 1.0) < 1e-3
    assert ob.correlation_length(A) > 1.0
