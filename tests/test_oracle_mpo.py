"""Pins the MPO builder: contracting L W ... W R over an open cluster must give
the Hamiltonian that exact diagonalisation builds straight from the bond list
(Sec. 2, Eq. mpo; Sec. 3, Eq. mpo2)."""
import numpy as np
import pytest

from oracle import ed
from oracle.idmrg import check_mpo
from workloads import (build_mpo, chain_bonds, dimerized_chain_bonds, j1j2_chain_bonds,
                       kagome_yc8_bonds, open_chain_bonds, random_chain_bonds, xx_chain_bonds,
                       yc4_j1j2_bonds)


def mpo_cluster_matrix(mpo, start, N):
    """Dense Hamiltonian of sites [start, start+N-1] from the MPO: the left
    boundary is the last row of W at the first site, the right boundary the
    first column of W at the last site (Sec. 2, text after Eq. mpo)."""
    ell = mpo.ell
    W0 = mpo.W[start % ell]
    M = [W0[-1, b] for b in range(W0.shape[1])]
    for k in range(start + 1, start + N - 1):
        W = mpo.W[k % ell]
        M = [sum(np.kron(M[a], W[a, b]) for a in range(W.shape[0])) for b in range(W.shape[1])]
    Wl = mpo.W[(start + N - 1) % ell]
    return sum(np.kron(M[a], Wl[a, 0]) for a in range(Wl.shape[0]))


CASES = [
    ("chain", chain_bonds(4), 4, 8),
    ("randchain", random_chain_bonds(8, 0.5, 1.5, 11), 8, 9),
    ("j1j2", j1j2_chain_bonds(4, 1.0, 0.5), 4, 8),
    ("xx", xx_chain_bonds(4, 0.5, 1.5, 5), 4, 8),
    ("dimer", dimerized_chain_bonds(4), 4, 8),
    ("yc4", yc4_j1j2_bonds(1.0, 0.5), 8, 9),
    ("kagome", kagome_yc8_bonds(1.0), 12, 9),
]


@pytest.mark.parametrize("name,bonds,ell,N", CASES, ids=[c[0] for c in CASES])
def test_mpo_equals_bond_hamiltonian(name, bonds, ell, N):
    mpo = build_mpo(bonds, ell)
    check_mpo(mpo.W, mpo.phys_charge, mpo.bond_charge)
    for start in range(0, ell, max(1, ell // 4)):
        H_mpo = mpo_cluster_matrix(mpo, start, N)
        H_ed = ed.dense_hamiltonian(N, open_chain_bonds(bonds, ell, start, start + N - 1))
        assert np.max(np.abs(H_mpo - H_ed)) < 1e-13, (name, start)


def test_mpo_bond_dims():
    """Naive finite-state-automaton widths: 2 + 3 x (sites with a bond across the cut)."""
    assert build_mpo(chain_bonds(4), 4).bond_dims == [5] * 4
    assert build_mpo(xx_chain_bonds(4, 1, 1, 0), 4).bond_dims == [4] * 4
    assert build_mpo(j1j2_chain_bonds(4, 1, .5), 4).bond_dims == [8] * 4
    assert max(build_mpo(kagome_yc8_bonds(), 12).bond_dims) == 20
    assert max(build_mpo(yc4_j1j2_bonds(), 8).bond_dims) == 20


def test_kagome_lattice_geometry():
    """Coordination 4, 24 bonds per 12-site ring, every site in two triangles."""
    bonds = kagome_yc8_bonds()
    assert len(bonds) == 24
    nb = {}
    for cell in range(-2, 3):
        for b in bonds:
            i, j = b.i + 12 * cell, b.j + 12 * cell
            nb.setdefault(i, set()).add(j)
            nb.setdefault(j, set()).add(i)
    for s in range(12):
        assert len(nb[s]) == 4
        tri = sum(1 for a in nb[s] for c in nb[s] if a < c and c in nb[a])
        assert tri == 2


def test_disorder_batch_recipe():
    """The 64-realisation workload: uneven unit cells and m as specified, and
    distinct couplings per realisation."""
    from workloads import disorder_batch
    work = disorder_batch(64)
    assert [len(mpo.W) for _, mpo, _ in work[:8]] == [8, 12, 16, 24] * 2
    assert [m for _, _, m in work[:12]] == [128] * 4 + [256] * 4 + [512] * 4
    assert [m for _, _, m in work[12:16]] == [128] * 4
    w0 = np.concatenate([w.ravel() for w in work[0][1].W])
    w4 = np.concatenate([w.ravel() for w in work[4][1].W])
    assert not np.array_equal(w0, w4)
