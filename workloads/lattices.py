"""Bond lists of the spin-1/2 models used as iDMRG workloads.

A model with an l-site period (Sec. 3, Eq. mpo2) is given by the bonds that
start in unit cell 0: ``Bond(i, j, jxy, jz)`` with ``0 <= i < l`` and ``j > i``;
``j`` may lie in a later cell.  The bond repeats under translation by ``l``.
The two-site term of a bond is

    jxy/2 * (S+_i S-_j + S-_i S+_j) + jz * Sz_i Sz_j,

so ``jxy == jz == J`` is the Heisenberg coupling ``J s_i . s_j`` (Sec. 4) and
``jz == 0`` the XX coupling.  Sites are 0-based here; the paper numbers them
from 1.
"""
from __future__ import annotations

from typing import List, NamedTuple, Sequence

import numpy as np


class Bond(NamedTuple):
    i: int
    j: int
    jxy: float
    jz: float


def _norm(i: int, j: int, jxy: float, jz: float, ell: int) -> Bond:
    """Order the two ends and shift the pair so that the left end is in cell 0."""
    a, b = (i, j) if i < j else (j, i)
    if a == b:
        raise ValueError("a bond needs two distinct sites")
    shift = (a // ell) * ell
    return Bond(a - shift, b - shift, float(jxy), float(jz))


def chain_bonds(ell: int, J: float = 1.0) -> List[Bond]:
    """Uniform nearest-neighbour Heisenberg chain with an l-site unit cell."""
    return [Bond(k, k + 1, J, J) for k in range(ell)]


def random_chain_bonds(ell: int, lo: float, hi: float, seed: int) -> List[Bond]:
    """Random-bond Heisenberg chain: J_k i.i.d. uniform in [lo, hi] (PCG64 seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Js = rng.uniform(lo, hi, size=ell)
    return [Bond(k, k + 1, float(J), float(J)) for k, J in enumerate(Js)]


def xx_chain_bonds(ell: int, lo: float, hi: float, seed: int) -> List[Bond]:
    """Random-bond XX chain (jz = 0); its open-chain energies are free-fermion sums."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Js = rng.uniform(lo, hi, size=ell)
    return [Bond(k, k + 1, float(J), 0.0) for k, J in enumerate(Js)]


def j1j2_chain_bonds(ell: int, J1: float, J2: float) -> List[Bond]:
    """J1-J2 Heisenberg chain (next-nearest-neighbour coupling J2)."""
    out = [Bond(k, k + 1, J1, J1) for k in range(ell)]
    out += [Bond(k, k + 2, J2, J2) for k in range(ell)]
    return out


def dimerized_chain_bonds(ell: int, J: float = 1.0) -> List[Bond]:
    """Fully dimerised chain: J on bonds (2k, 2k+1), nothing on (2k+1, 2k+2)."""
    if ell % 2:
        raise ValueError("ell must be even")
    return [Bond(k, k + 1, J, J) for k in range(0, ell, 2)]


def yc4_j1j2_bonds(J1: float = 1.0, J2: float = 0.5) -> List[Bond]:
    """J1-J2 square lattice on a 4-leg cylinder (periodic in y), snake order.

    Site (x, y) has 1D index 4x + y for even x and 4x + 3 - y for odd x; the
    unit cell holds two columns (l = 8).  J1 on vertical and horizontal bonds,
    J2 on both diagonals.
    """
    ell, W = 8, 4

    def idx(x: int, y: int) -> int:
        y %= W
        return W * x + (y if x % 2 == 0 else W - 1 - y)

    out = []
    for x in range(2):
        for y in range(W):
            out.append(_norm(idx(x, y), idx(x, y + 1), J1, J1, ell))
            out.append(_norm(idx(x, y), idx(x + 1, y), J1, J1, ell))
            out.append(_norm(idx(x, y), idx(x + 1, y + 1), J2, J2, ell))
            out.append(_norm(idx(x, y), idx(x + 1, y - 1), J2, J2, ell))
    return out


def kagome_yc8_bonds(J: float = 1.0) -> List[Bond]:
    """Nearest-neighbour kagome Heisenberg model on a YC8 cylinder, l = 12.

    Site 12 r + 3 k + a (ring r, cell k = 0..3 around the circumference, a = 0..2).
    Per cell the six bonds of its two corner-sharing triangles:
    (a0,a1), (a1,a2) in the cell, (a2, a0 of k+1), (a1, a0 of k+1), and
    (a2, a0 of ring r+1), (a2, a1 of ring r+1).  Every site then has
    coordination 4 and the longest bond spans 11 sites.  The paper shows its
    own site numbering only in a figure, so this ordering may differ from it.
    """
    ell = 12

    def s(r: int, k: int, a: int) -> int:
        return 12 * r + 3 * (k % 4) + a

    out = []
    for k in range(4):
        out.append(_norm(s(0, k, 0), s(0, k, 1), J, J, ell))
        out.append(_norm(s(0, k, 1), s(0, k, 2), J, J, ell))
        out.append(_norm(s(0, k, 2), s(0, k + 1, 0), J, J, ell))
        out.append(_norm(s(0, k, 1), s(0, k + 1, 0), J, J, ell))
        out.append(_norm(s(0, k, 2), s(1, k, 0), J, J, ell))
        out.append(_norm(s(0, k, 2), s(1, k, 1), J, J, ell))
    return out


def open_chain_bonds(unit_bonds: Sequence[Bond], ell: int, start: int, stop: int) -> List[Bond]:
    """All bonds of the periodic system with both ends in sites [start, stop],
    re-indexed so that site ``start`` becomes 0.  This is the Hamiltonian of the
    open cluster a superblock represents."""
    out = []
    for cell in range((start // ell) - 2, (stop // ell) + 2):
        for b in unit_bonds:
            i, j = b.i + cell * ell, b.j + cell * ell
            if start <= i and j <= stop:
                out.append(Bond(i - start, j - start, b.jxy, b.jz))
    return out
