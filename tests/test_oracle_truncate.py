"""Pins Step 4 / Step 6 (SVD truncation and block-spin transformation)."""
import numpy as np

from oracle import ed
from oracle.idmrg import ParallelIDMRG, sector_mask, truncate, update_left, update_right
from workloads import build_mpo, open_chain_bonds, random_chain_bonds


def _random_psi(DL, DR, seed):
    rng = np.random.default_rng(seed)
    qL = rng.choice([-3, -1, 1, 3], size=DL)
    qR = rng.choice([-3, -1, 1, 3], size=DR)
    qp = np.array([1, -1])
    mask = sector_mask(qL, qp, qR)
    psi = np.where(mask, rng.standard_normal(mask.shape), 0.0)
    return psi / np.linalg.norm(psi), qL, qp, qR


def test_truncation_invariants():
    for seed in range(4):
        psi, qL, qp, qR = _random_psi(9, 7, seed)
        for m in (3, 6, 100):
            t = truncate(psi, qL, qp, qR, m)
            D = len(t.lam)
            assert D <= m
            assert abs(np.sum(t.lam_all ** 2) - 1.0) < 1e-13        # Step 4: sum lam^2 = 1
            assert np.all(np.diff(t.lam_all) <= 0)                     # descending (reading R1)
            U = t.U.reshape(-1, D)
            V = t.V.reshape(-1, D)
            assert np.allclose(U.T @ U, np.eye(D), atol=1e-13)
            assert np.allclose(V.T @ V, np.eye(D), atol=1e-13)
            M = psi.reshape(U.shape[0], V.shape[0])
            approx = U @ np.diag(t.lam) @ V.T
            # Eckart-Young: the discarded weight is the squared distance
            assert abs(np.linalg.norm(M - approx) ** 2 - t.eps) < 1e-13
            # Eq. tru: eps = (2 - eps') eps'
            assert abs(t.eps - (2 - t.eps_best) * t.eps_best) < 1e-14
            # kept states are charge eigenstates
            ql = (qL[:, None] + qp[None, :]).ravel()
            qr = (qp[:, None] + qR[None, :]).ravel()
            for k in range(D):
                assert np.all(U[ql != t.q[k], k] == 0.0)
                assert np.all(V[qr != -t.q[k], k] == 0.0)
            # the kept singular values are the D largest
            assert np.allclose(np.sort(t.lam)[::-1], t.lam_all[:D])


def test_tie_rule_keeps_multiplets_whole():
    """Reading R2: never cut inside a group of equal singular values."""
    lam = np.array([0.6, 0.5, 0.4, 0.4, 0.4, 0.2])
    lam = lam / np.linalg.norm(lam)
    psi = np.zeros((6, 1, 1, 6))
    qL = np.zeros(6, dtype=int)
    qR = np.zeros(6, dtype=int)
    for k in range(6):
        psi[k, 0, 0, k] = lam[k]
    qp = np.array([0])
    assert len(truncate(psi, qL, qp, qR, m=3).lam) == 2
    assert len(truncate(psi, qL, qp, qR, m=5).lam) == 5
    assert len(truncate(psi, qL, qp, qR, m=4).lam) == 2


def test_environment_identity_and_hamiltonian_channels():
    """Step 6 with orthonormal u, v: the identity channel (last for L, first
    for R) stays the unit matrix exactly; the completed-term channel (first
    for L, last for R) is the block Hamiltonian, symmetric and bounded below
    by the ground energy of the block's own sites."""
    ell = 8
    bonds = random_chain_bonds(ell, 0.5, 1.5, 23)
    dm = ParallelIDMRG.from_mpo(build_mpo(bonds, ell), m=8)
    for n in range(1, 6):
        dm.step()
        for p in range(dm.P):
            L, R = dm.L[p], dm.R[p]
            assert np.allclose(L.op[-1], np.eye(len(L.q)), atol=1e-13)
            assert np.allclose(R.op[0], np.eye(len(R.q)), atol=1e-13)
            HL, HR = L.op[0], R.op[-1]
            assert np.allclose(HL, HL.T, atol=1e-12) and np.allclose(HR, HR.T, atol=1e-12)
            # L^(n) of pair p covers sites [2p, 2p+n]; R^(n) of pair p covers [2p+n+1, 2p+2n+1]
            N = n + 1
            eL = min(ed.ground_energy(N, open_chain_bonds(bonds, ell, 2 * p, 2 * p + n), q)
                     for q in range(-N, N + 1, 2))
            eR = min(ed.ground_energy(N, open_chain_bonds(bonds, ell, 2 * p + n + 1, 2 * p + 2 * n + 1), q)
                     for q in range(-N, N + 1, 2))
            assert np.linalg.eigvalsh(HL)[0] >= eL - 1e-10
            assert np.linalg.eigvalsh(HR)[0] >= eR - 1e-10
            # charges: L_a connects x -> y only if q_x - q_y equals the channel charge
            for a in range(L.op.shape[0]):
                nz = np.abs(L.op[a]) > 0
                dq = L.q[:, None] - L.q[None, :]
                assert len(set(dq[nz].tolist())) <= 1


def test_update_left_right_are_projections():
    """With u = identity (no truncation) Eq. L is the plain product L W."""
    ell = 4
    bonds = random_chain_bonds(ell, 0.5, 1.5, 2)
    dm = ParallelIDMRG.from_mpo(build_mpo(bonds, ell), m=64)
    L, W1, W2, R = dm.superblock(0)
    D, d = L.op.shape[1], W1.shape[2]
    U = np.eye(D * d).reshape(D, d, D * d)
    Lp = update_left(L, W1, U, np.zeros(D * d, dtype=int))
    for b in range(W1.shape[1]):
        direct = sum(np.kron(L.op[a], W1[a, b]) for a in range(W1.shape[0]))
        assert np.allclose(Lp.op[b], direct, atol=1e-15)
    V = np.eye(d * R.op.shape[1]).reshape(d, R.op.shape[1], -1)
    Rp = update_right(R, W2, V, np.zeros(V.shape[2], dtype=int))
    for b in range(W2.shape[0]):
        direct = sum(np.kron(W2[b, c], R.op[c]) for c in range(W2.shape[1]))
        assert np.allclose(Rp.op[b], direct, atol=1e-15)
