"""Matrix product operator (MPO) of an l-site periodic spin-1/2 Hamiltonian.

The Hamiltonian of kl sites is the product of the l site tensors
``W_1 .. W_l`` repeated k times (Sec. 3, Eq. mpo2).  ``W_i`` is an
``a_i x a_{i+1}`` matrix of local operators ``|s><s'|`` (Sec. 2, Eq. mpo) in
the lower-triangular finite-state-automaton form:

* channel 0 of every MPO bond is "term completed", the last channel is
  "nothing placed yet" (identity);
* the boundary vectors are the last row (left) and the first column (right)
  of ``W_i`` (Sec. 2, text after Eq. mpo);
* between them, each site p with a bond still open across the cut owns one
  channel per operator it has placed (S+, S-, Sz), ordered by p.

Arrays: ``W[k]`` has shape ``[a_k, a_{k+1}, d, d]`` with
``W[k][a, b, s, s'] = <s| W_k(a,b) |s'>`` and ``a_l = a_0``; ``phys_charge[s]`` is
2 Sz of local state s (0 = up, 1 = down); ``bond_charge[k][a]`` is the 2 Sz that
channel a of bond k (the bond to the left of site k) carries, so that a
non-zero ``W[k][a,b,s,s']`` always has
``phys_charge[s] - phys_charge[s'] == bond_charge[k+1][b] - bond_charge[k][a]``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Sequence, Tuple

import numpy as np

from .lattices import Bond

SP = np.array([[0.0, 1.0], [0.0, 0.0]])   # S+ : |down> -> |up>
SM = np.array([[0.0, 0.0], [1.0, 0.0]])   # S- : |up> -> |down>
SZ = np.array([[0.5, 0.0], [0.0, -0.5]])
ID = np.eye(2)
PHYS_CHARGE = np.array([1, -1], dtype=np.int32)

# operator placed on the left end of a bond, the one that closes it, its charge
_TYPES = (
    ("+", SP, SM, 2),
    ("-", SM, SP, -2),
    ("z", SZ, SZ, 0),
)


@dataclass
class MPO:
    ell: int
    d: int
    W: List[np.ndarray]
    phys_charge: np.ndarray
    bond_charge: List[np.ndarray]
    bonds: List[Bond] = field(default_factory=list)

    @property
    def bond_dims(self) -> List[int]:
        return [w.shape[0] for w in self.W]

    def flat(self) -> Tuple[np.ndarray, np.ndarray, np.ndarray, np.ndarray]:
        """Arrays in the layout of the C ABI's ``idmrg_mpo``: bond dims (l+1
        entries, last == first), W concatenated site by site (row-major
        [a_i][a_{i+1}][d][d]), phys charges, bond charges concatenated bond by
        bond (l entries per period)."""
        dims = np.array(self.bond_dims + [self.bond_dims[0]], dtype=np.int32)
        W = np.concatenate([w.ravel() for w in self.W]).astype(np.float64)
        bc = np.concatenate(self.bond_charge).astype(np.int32)
        return dims, W, self.phys_charge.astype(np.int32), bc


def _bond_lookup(bonds: Sequence[Bond], ell: int) -> Dict[Tuple[int, int], List[Bond]]:
    """Map (left site mod l, span) -> bonds."""
    out: Dict[Tuple[int, int], List[Bond]] = {}
    for b in bonds:
        out.setdefault((b.i % ell, b.j - b.i), []).append(b)
    return out


def _channels(bonds: Sequence[Bond], ell: int, k: int, reach: int) -> List[Tuple[int, str]]:
    """Open channels on the bond to the left of site k, as (p - k, type)."""
    out = []
    for p in range(k - reach, k):
        need = set()
        for b in bonds:
            if b.i % ell != p % ell:
                continue
            j = p + (b.j - b.i)
            if j >= k:
                if b.jxy != 0.0:
                    need.update("+-")
                if b.jz != 0.0:
                    need.add("z")
        for t, *_ in _TYPES:
            if t in need:
                out.append((p - k, t))
    return out


def build_mpo(bonds: Sequence[Bond], ell: int) -> MPO:
    """Lower-triangular MPO of ``sum over bonds`` for an l-site period."""
    bonds = [b for b in bonds if (b.jxy != 0.0 or b.jz != 0.0)]
    reach = max([b.j - b.i for b in bonds] + [1])
    look = _bond_lookup(bonds, ell)
    chans = [_channels(bonds, ell, k, reach) for k in range(ell + 1)]
    assert chans[0] == chans[ell]
    W, bond_charge = [], []
    typ = {t: (op, closer, q) for t, op, closer, q in _TYPES}
    for k in range(ell):
        left = [("done",)] + chans[k] + [("id",)]
        right = [("done",)] + chans[k + 1] + [("id",)]
        li = {c: n for n, c in enumerate(left)}
        # key the right bond's channels in the left bond's offsets (p - k)
        ri = {}
        for n, c in enumerate(right):
            ri[c if len(c) == 1 else (c[0] + 1, c[1])] = n
        w = np.zeros((len(left), len(right), 2, 2))
        w[li[("done",)], ri[("done",)]] = ID
        w[li[("id",)], ri[("id",)]] = ID
        for t, (op, _, _) in typ.items():
            if (0, t) in ri:  # site k opens channel t
                w[li[("id",)], ri[(0, t)]] += op
        for c in chans[k]:
            off, t = c
            if c in ri:  # still open after site k: pass through
                w[li[c], ri[c]] += ID
            for b in look.get(((k + off) % ell, -off), []):
                _, closer, _ = typ[t]
                coef = b.jxy / 2.0 if t in "+-" else b.jz
                w[li[c], ri[("done",)]] += coef * closer
        W.append(w)
        bond_charge.append(np.array([0] + [typ[t][2] for _, t in chans[k]] + [0], dtype=np.int32))
    return MPO(ell=ell, d=2, W=W, phys_charge=PHYS_CHARGE.copy(), bond_charge=bond_charge,
               bonds=list(bonds))
