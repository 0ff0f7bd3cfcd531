"""Pins the oracle's H_eff psi (Step 3) and Lanczos solver."""
import numpy as np

from oracle import ed
from oracle.idmrg import (ParallelIDMRG, heff_apply, heff_dense, initial_blocks, lanczos,
                          sector_mask)
from workloads import (build_mpo, chain_bonds, j1j2_chain_bonds, open_chain_bonds,
                       random_chain_bonds)


def test_heff_n1_is_four_site_cluster():
    """At n = 1 with no truncation the superblock Hamiltonian is the open
    4-site cluster [2p, 2p+3] (Step 2' with the boundary blocks of Step 1)."""
    for bonds, ell in [(random_chain_bonds(8, 0.5, 1.5, 3), 8), (j1j2_chain_bonds(4, 1.0, 0.7), 4)]:
        mpo = build_mpo(bonds, ell)
        Ls, Rs = initial_blocks(mpo.W, mpo.phys_charge)
        for p in range(ell // 2):
            c1, c2 = (2 * p + 1) % ell, (2 * p + 2) % ell
            H = heff_dense(Ls[p], mpo.W[c1], mpo.W[c2], Rs[(p + 1) % (ell // 2)])
            H_ed = ed.dense_hamiltonian(4, open_chain_bonds(bonds, ell, 2 * p, 2 * p + 3))
            assert np.max(np.abs(H - H_ed)) < 1e-14


def _grown(m=6, steps=3, bonds=None, ell=8):
    bonds = bonds or random_chain_bonds(ell, 0.5, 1.5, 17)
    dm = ParallelIDMRG.from_mpo(build_mpo(bonds, ell), m=m)
    for _ in range(steps):
        dm.step()
    return dm


def test_heff_apply_equals_kronecker_matrix_and_is_symmetric():
    dm = _grown()
    rng = np.random.default_rng(0)
    for p in range(dm.P):
        L, W1, W2, R = dm.superblock(p)
        H = heff_dense(L, W1, W2, R)
        assert np.max(np.abs(H - H.T)) < 1e-12 * np.max(np.abs(H))
        for _ in range(3):
            x = rng.standard_normal((L.op.shape[1], 2, 2, R.op.shape[1]))
            y = heff_apply(L, W1, W2, R, x)
            assert np.allclose(y.ravel(), H @ x.ravel(), rtol=0, atol=1e-12 * np.abs(H).max() * 10)


def test_heff_conserves_charge():
    dm = _grown()
    rng = np.random.default_rng(1)
    for p in range(dm.P):
        L, W1, W2, R = dm.superblock(p)
        mask = sector_mask(L.q, dm.qp, R.q)
        x = np.where(mask, rng.standard_normal(mask.shape), 0.0)
        y = heff_apply(L, W1, W2, R, x)
        assert np.all(y[~mask] == 0.0)


def test_lanczos_matches_dense_eigh():
    dm = _grown(m=8, steps=3)
    for p in range(dm.P):
        L, W1, W2, R = dm.superblock(p)
        mask = sector_mask(L.q, dm.qp, R.q)
        H = heff_dense(L, W1, W2, R)[np.ix_(mask.ravel(), mask.ravel())]
        e_exact = np.linalg.eigvalsh(H)[0]
        v0 = np.where(mask, 1.0 + 0.1 * np.arange(mask.size).reshape(mask.shape) % 7, 0.0)
        e, psi, it, conv = dm.solve(p, v0)
        assert conv
        assert abs(e - e_exact) < 1e-11 * max(1.0, abs(e_exact))
        r = heff_apply(L, W1, W2, R, psi) - e * psi
        assert np.linalg.norm(r) < 1e-9
        assert abs(np.linalg.norm(psi) - 1.0) < 1e-14
        assert np.all(psi[~mask] == 0.0)


def test_lanczos_on_plain_matrix():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((60, 60))
    A = A + A.T
    e, psi, it, conv = lanczos(lambda x: A @ x, rng.standard_normal(60), tol=1e-12, maxit=200)
    assert conv and abs(e - np.linalg.eigvalsh(A)[0]) < 1e-11
