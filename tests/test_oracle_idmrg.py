"""Pins the whole oracle iteration (Sec. 3) against exact diagonalisation,
free fermions and closed forms."""
import json
import os

import numpy as np
import pytest

from oracle import ed, rng
from oracle.idmrg import ParallelIDMRG
from workloads import (build_mpo, chain_bonds, dimerized_chain_bonds, j1j2_chain_bonds,
                       open_chain_bonds, random_chain_bonds, xx_chain_bonds)

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


def _ed_superblock(bonds, ell, p, n):
    """Superblock p at iteration n is the open cluster [2p, 2p+2n+1]."""
    N = 2 * n + 2
    return ed.ground_energy(N, open_chain_bonds(bonds, ell, 2 * p, 2 * p + N - 1))


@pytest.mark.parametrize("case", ["chain", "randchain", "j1j2"])
def test_exact_regime_equals_ed(case):
    """While 2^n <= m nothing is discarded and e_i^(n) is the exact ground
    energy of its cluster; beyond it the energy is a variational upper bound."""
    bonds, ell = {"chain": (chain_bonds(4), 4),
                  "randchain": (random_chain_bonds(8, 0.5, 1.5, 99), 8),
                  "j1j2": (j1j2_chain_bonds(4, 1.0, 0.3), 4)}[case]
    m = 32
    dm = ParallelIDMRG.from_mpo(build_mpo(bonds, ell), m=m)
    for n in range(1, 7):
        r = dm.step()
        for p in range(dm.P):
            E = _ed_superblock(bonds, ell, p, n)
            if 2 ** n <= m:
                assert abs(r.energies[p] - E) < 1e-11 * max(1, abs(E)), (n, p)
            else:
                assert r.energies[p] >= E - 1e-11
            assert abs(r.eps[p] - (2 - r.eps_best[p]) * r.eps_best[p]) < 1e-14


def test_bond_energy_matches_ed_at_n1():
    bonds, ell = random_chain_bonds(4, 0.5, 1.5, 4), 4
    dm = ParallelIDMRG.from_mpo(build_mpo(bonds, ell), m=16)
    r = dm.step()
    for p in range(dm.P):
        ob = open_chain_bonds(bonds, ell, 2 * p, 2 * p + 3)
        H = ed.dense_hamiltonian(4, ob)
        w, v = np.linalg.eigh(H)
        g = v[:, 0]
        centre = [b for b in ob if (b.i, b.j) == (1, 2)]
        Hc = ed.dense_hamiltonian(4, centre)
        assert abs(r.bond[p] - g @ Hc @ g) < 1e-12


def test_majumdar_ghosh_and_dimer_energies_are_exact():
    for bonds, key in [(j1j2_chain_bonds(4, 1.0, 0.5), "majumdar_ghosh_energy_per_site"),
                       (dimerized_chain_bonds(4), "dimer_energy_per_site")]:
        dm = ParallelIDMRG.from_mpo(build_mpo(bonds, 4), m=4)
        egs = []
        for _ in range(16):
            r = dm.step()
            if r.e_g is not None:
                egs.append(r.e_g)
            # centre bond: a singlet (-3/4) when the cut splits a dimer, else 0
            n = r.n
            expect = -0.75 if n % 2 == 0 else 0.0
            assert np.allclose(r.bond, expect, atol=1e-12)
        assert len(egs) == 4
        assert np.allclose(egs, GOLDEN[key]["value"], atol=1e-12)


def test_xx_chain_against_free_fermions():
    ell = 4
    bonds = xx_chain_bonds(ell, 0.5, 1.5, 8)
    Js = [b.jxy for b in bonds]
    dm = ParallelIDMRG.from_mpo(build_mpo(bonds, ell), m=16)
    for n in range(1, 25):
        r = dm.step()
        for p in range(dm.P):
            N = 2 * n + 2
            E = ed.xx_open_chain_energy([Js[(2 * p + k) % ell] for k in range(N - 1)])
            if 2 ** n <= 16:
                assert abs(r.energies[p] - E) < 1e-11 * N
            else:
                assert r.energies[p] >= E - 1e-10
                assert (r.energies[p] - E) / N < 2e-4


def test_bethe_ansatz_limit():
    dm = ParallelIDMRG.from_mpo(build_mpo(chain_bonds(4), 4), m=32)
    eg = None
    for _ in range(80):
        r = dm.step()
        eg = r.e_g if r.e_g is not None else eg
    assert abs(eg - GOLDEN["bethe_chain_energy_per_site"]["value"]) < 1e-3
    assert abs(eg - ed.BETHE_CHAIN_ENERGY) < 1e-3


def test_prediction_fidelity_and_speedup():
    """Eq. fid1 >= the best fidelity of a rank-m vector (Eq. fid2, with exactly
    m values), the predicted vector is nearly optimal once the run has settled,
    and it cuts the Lanczos work (Sec. 4.2)."""
    m = 16
    bonds = chain_bonds(4)
    runs = {}
    for pred in (True, False):
        dm = ParallelIDMRG.from_mpo(build_mpo(bonds, 4), m=m, predict=pred)
        its, fids = [], []
        for _ in range(30):
            r = dm.step()
            its.append(r.iters.mean())
            if pred and r.n >= 3:
                for p in range(dm.P):
                    lam = r.lam_all[p][:m]
                    best = 1.0 - np.sqrt(np.sum(lam ** 2))
                    assert r.fidelity[p] >= best - 1e-12
                fids.append(r.fidelity.max())
        runs[pred] = np.mean(its[-10:])
        if pred:
            assert max(fids[-10:]) < 1e-5
    assert runs[True] < 0.7 * runs[False]


def test_start_vector_is_deterministic_and_uniform():
    a = rng.start_vector(0, 1, 0, 10000)
    b = rng.start_vector(0, 1, 0, 10000)
    c = rng.start_vector(0, 1, 1, 10000)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.min() >= -1 and a.max() < 1 and abs(a.mean()) < 0.03


def test_splitmix64_published_vectors():
    g = GOLDEN["splitmix64_seed0"]["values_hex"]
    assert [int(x) for x in rng.splitmix64(0, 3)] == [int(h, 16) for h in g]
    assert [int(x) for x in rng.splitmix64(1234567, 5)] == GOLDEN["splitmix64_seed1234567"]["values"]


def test_wrong_prediction_reading_is_visible():
    """The prediction parity test on the GPU compares Eq. fid1 per superblock
    within 1e-9 + 1e-3 eps.  Planting a wrong reading of R4 in the oracle --
    lambda'' and u taken from superblock i instead of i + 1 -- moves the
    fidelity error far outside that bound (and costs Lanczos iterations), so a
    GPU path with that mistake would fail there even though its converged
    energies stay correct."""
    from oracle.idmrg import predict

    class WrongR4(ParallelIDMRG):
        def start_vector(self, p):
            if self.n < 3 or not self.use_prediction:
                return super().start_vector(p)
            from oracle.idmrg import sector_mask
            L, W1, W2, R = self.superblock(p)
            mask = sector_mask(L.q, self.qp, R.q, self.target)
            j = (p + 1) % self.P
            a, b, c = self.prev[p], self.prev[j], self.prev2[p]   # lambda'' of i, not i + 1
            if c.lam.shape[0] != b.U.shape[0]:
                return super().start_vector(p)
            v = predict(a.lam, a.V, b.U, b.lam, c.lam, self.zero_rel)
            return np.where(mask, v, 0.0)

    mpo = build_mpo(random_chain_bonds(8, 0.5, 1.5, 1606), 8)
    good = ParallelIDMRG.from_mpo(mpo, m=24)
    bad = WrongR4.from_mpo(mpo, m=24)
    moved = 0
    for _ in range(12):
        rg, rb = good.step(), bad.step()
        if rg.n < 5:
            continue
        assert np.max(np.abs(rg.energies - rb.energies)) / (2 * rg.n + 2) < 1e-10  # energies agree
        d = np.abs(rg.fidelity - rb.fidelity)
        moved += int(np.any(d > 1e-9 + 1e-3 * np.abs(rg.fidelity) + 1e-6))
    assert moved >= 6
