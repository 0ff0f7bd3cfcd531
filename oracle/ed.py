"""Exact diagonalisation of open spin-1/2 clusters from a bond list.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Basis: N spins, state index s = sum_k b_k 2^(N-1-k) with b_k = 0 for up and 1
for down, i.e. site 0 is the most significant bit.  This is the ordering of
``np.kron(op_0, op_1, ...)`` with local index 0 = up, so dense matrices built
here can be compared entry by entry with any Kronecker-ordered construction.

Bond term (i, j, jxy, jz): jxy/2 (S+_i S-_j + S-_i S+_j) + jz Sz_i Sz_j.
"""
from __future__ import annotations

from itertools import combinations
from typing import Iterable, Sequence, Tuple

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

BondT = Tuple[int, int, float, float]


def _bit(s: int, k: int, N: int) -> int:
    return (s >> (N - 1 - k)) & 1


def dense_hamiltonian(N: int, bonds: Iterable[BondT]) -> np.ndarray:
    """Full 2^N x 2^N Hamiltonian (small N only)."""
    dim = 1 << N
    H = np.zeros((dim, dim))
    for s in range(dim):
        for (i, j, jxy, jz) in bonds:
            bi, bj = _bit(s, i, N), _bit(s, j, N)
            szi, szj = 0.5 - bi, 0.5 - bj
            H[s, s] += jz * szi * szj
            if bi != bj:
                t = s ^ (1 << (N - 1 - i)) ^ (1 << (N - 1 - j))
                H[t, s] += 0.5 * jxy
    return H


def sector_states(N: int, two_sz: int) -> np.ndarray:
    """Basis states with total 2 Sz = two_sz, ascending."""
    n_down = (N - two_sz) // 2
    out = []
    for downs in combinations(range(N), n_down):
        s = 0
        for k in downs:
            s |= 1 << (N - 1 - k)
        out.append(s)
    return np.array(sorted(out), dtype=np.int64)


def sector_hamiltonian(N: int, bonds: Sequence[BondT], two_sz: int = 0) -> sp.csr_matrix:
    states = sector_states(N, two_sz)
    index = {int(s): n for n, s in enumerate(states)}
    rows, cols, vals = [], [], []
    for n, s in enumerate(states):
        s = int(s)
        diag = 0.0
        for (i, j, jxy, jz) in bonds:
            bi, bj = _bit(s, i, N), _bit(s, j, N)
            diag += jz * (0.5 - bi) * (0.5 - bj)
            if bi != bj and jxy != 0.0:
                t = s ^ (1 << (N - 1 - i)) ^ (1 << (N - 1 - j))
                rows.append(index[t]); cols.append(n); vals.append(0.5 * jxy)
        rows.append(n); cols.append(n); vals.append(diag)
    dim = len(states)
    return sp.csr_matrix((vals, (rows, cols)), shape=(dim, dim))


def ground_energy(N: int, bonds: Sequence[BondT], two_sz: int = 0) -> float:
    """Lowest eigenvalue of an open cluster in the given 2 Sz sector."""
    H = sector_hamiltonian(N, bonds, two_sz)
    if H.shape[0] <= 2000:
        return float(np.linalg.eigvalsh(H.toarray())[0])
    v0 = np.ones(H.shape[0]) / np.sqrt(H.shape[0])
    w = spla.eigsh(H, k=1, which="SA", v0=v0, tol=1e-14, maxiter=20000)[0]
    return float(w[0])


def xx_open_chain_energy(J: Sequence[float]) -> float:
    """Ground energy of the open XX chain sum_k J_k/2 (S+_k S-_{k+1} + h.c.)
    with N = len(J) + 1 sites (N even) at 2 Sz = 0.  Jordan-Wigner maps it to
    free fermions with hopping J_k/2; half filling fills the N/2 lowest
    single-particle levels."""
    N = len(J) + 1
    h = np.zeros((N, N))
    for k, Jk in enumerate(J):
        h[k, k + 1] = h[k + 1, k] = 0.5 * Jk
    eps = np.linalg.eigvalsh(h)
    return float(np.sum(eps[: N // 2]))


BETHE_CHAIN_ENERGY = 0.25 - np.log(2.0)   # Hulthen's ground-state energy per site
