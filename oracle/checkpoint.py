"""Reader of the library's checkpoint files (idmrg_save) into an oracle state.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  It lets the FP64 oracle
take one step from a state the GPU path saved, so that a single step can be
compared at sizes the oracle could never reach from n = 1 in a test: the
file is read as data (placement of numbers into the oracle's dense arrays),
nothing of the library is imported or executed, and everything the oracle
then computes is its own arithmetic.

File layout (little-endian, every scalar written on its own, no padding; a
"vector" is an int64 count followed by that many items):

* 8 bytes magic ``IDMRGCK1``; int32 l, d, P, m, prec, target; int32 vector
  of the MPO bond dimensions (l + 1 entries);
* int32 n (the iteration the next step performs), int32 n of the last e_g
  estimate, float64 that estimate; int32 and float64 vectors of the e^(n)_1
  history (iteration, energy) and of the eps^(n)_1 history;
* per pair q = 0 .. P-1:
  - the left block L^(n-1) of pair q, then the right block R^(n-1) of pair
    q, each as: basis (int32 vector of sector charges, int32 vector of
    sector sizes; the states of a sector are contiguous, sectors in the
    stored order), int32 vector of the MPO channel charges chq[a], float64
    vector of blocks: for channel a (outer loop) and in-sector si (inner
    loop), when the basis has a sector of charge q[si] + chq[a] (the
    out-sector so), a dense row-major dim[so] x dim[si] block of
    <x| O_a |y>, x in so, y in si;
  - the truncations of superblock q at n-1 and at n-2, each as: int32
    valid; four bases (left block, right block, kept left states U, kept
    right states V; U's sectors in ascending charge Q, V's sector g the
    charge target - Q of U's sector g, state k of either pairing with state k
    of the other); int64 number of kept sectors, then per sector int32 Q, k,
    r, c, job, int64 u_off, v_off, int32 lam_off, and two vectors of int32
    triples (the count is of triples): row groups (left sector i, site
    state s, first row) and column groups (site state t, right sector j,
    first row); float64 vectors of the
    kept singular values (basis order) and of all singular values
    (descending); float64 eps, eps_best; int64 sizes of U and V; float64
    vectors U and V: sector g's U block is r x k row-major at u_off (row
    first_row + x of a row group = left state off(i) + x with site state s),
    its V block c x k row-major at v_off (row first_row + y of a column group
    = site state t with right state off(j) + y).
"""
from __future__ import annotations

import struct
from typing import List, Tuple

import numpy as np

from .idmrg import Block, ParallelIDMRG, Truncation

MAGIC = b"IDMRGCK1"


class _Reader:
    def __init__(self, data: bytes):
        self.b = data
        self.o = 0

    def take(self, fmt: str):
        size = struct.calcsize("<" + fmt)
        if self.o + size > len(self.b):
            raise ValueError("checkpoint truncated")
        v = struct.unpack_from("<" + fmt, self.b, self.o)
        self.o += size
        return v if len(v) > 1 else v[0]

    def vec(self, dtype: str, width: int = 1) -> np.ndarray:
        """A vector of `count` items of `width` numbers each (flattened)."""
        n = self.take("q") * width
        dt = np.dtype(dtype).newbyteorder("<")
        size = n * dt.itemsize
        if n < 0 or self.o + size > len(self.b):
            raise ValueError("checkpoint truncated")
        a = np.frombuffer(self.b, dtype=dt, count=n, offset=self.o).astype(dtype)
        self.o += size
        return a

    def basis(self) -> Tuple[np.ndarray, np.ndarray]:
        q = self.vec("i4").astype(np.int64)
        dim = self.vec("i4").astype(np.int64)
        if len(q) != len(dim):
            raise ValueError("damaged basis")
        return q, dim


def _offsets(dim: np.ndarray) -> np.ndarray:
    return np.concatenate([[0], np.cumsum(dim)[:-1]]).astype(np.int64) if len(dim) else np.zeros(0, np.int64)


def _states(q: np.ndarray, dim: np.ndarray) -> np.ndarray:
    return np.repeat(q, dim)


def _block(r: _Reader) -> Block:
    q, dim = r.basis()
    chq = r.vec("i4").astype(np.int64)
    data = r.vec("f8")
    off = _offsets(dim)
    D = int(dim.sum())
    op = np.zeros((len(chq), D, D))
    pos = 0
    where = {int(c): i for i, c in enumerate(q)}
    for a, ch in enumerate(chq):
        for si in range(len(q)):
            so = where.get(int(q[si] + ch))
            if so is None:
                continue
            n = int(dim[so] * dim[si])
            op[a, off[so]:off[so] + dim[so], off[si]:off[si] + dim[si]] = data[pos:pos + n].reshape(dim[so], dim[si])
            pos += n
    if pos != len(data):
        raise ValueError("block data does not match its layout")
    return Block(op, _states(q, dim))


def _truncation(r: _Reader, d: int):
    valid = r.take("i")
    qL, dL = r.basis()
    qR, dR = r.basis()
    qU, dU = r.basis()
    qV, dV = r.basis()
    nsec = r.take("q")
    secs = []
    for _ in range(nsec):
        Q, k, rr, cc, job = r.take("iiiii")
        u_off, v_off = r.take("qq")
        lam_off = r.take("i")
        rg = r.vec("i4", 3).reshape(-1, 3)
        cg = r.vec("i4", 3).reshape(-1, 3)
        secs.append((Q, k, rr, cc, u_off, v_off, lam_off, rg, cg))
    lam = r.vec("f8")
    lam_all = r.vec("f8")
    eps, eps_best = r.take("dd")
    usize, vsize = r.take("qq")
    U = r.vec("f8")
    V = r.vec("f8")
    if not valid:
        return None
    if len(U) != usize or len(V) != vsize:
        raise ValueError("damaged truncation record")
    offL, offR, offU = _offsets(dL), _offsets(dR), _offsets(dU)
    kept = int(dU.sum())
    Ud = np.zeros((int(dL.sum()), d, kept))
    Vd = np.zeros((d, int(dR.sum()), kept))
    for g, (Q, k, rr, cc, u_off, v_off, lam_off, rg, cg) in enumerate(secs):
        if qU[g] != Q or dU[g] != k:
            raise ValueError("kept sectors out of order")
        col = slice(offU[g], offU[g] + k)
        blkU = U[u_off:u_off + rr * k].reshape(rr, k)
        blkV = V[v_off:v_off + cc * k].reshape(cc, k)
        for i, s, first in rg:
            Ud[offL[i]:offL[i] + dL[i], s, col] = blkU[first:first + dL[i]]
        for t, j, first in cg:
            Vd[t, offR[j]:offR[j] + dR[j], col] = blkV[first:first + dR[j]]
    qk = _states(qU, dU)
    return Truncation(U=Ud, V=Vd, lam=lam, q=qk, lam_all=lam_all, eps=eps, eps_best=eps_best)


def read_checkpoint(path: str) -> dict:
    """Parse a checkpoint into plain arrays (see the module docstring)."""
    with open(path, "rb") as f:
        data = f.read()
    if data[:8] != MAGIC:
        raise ValueError(f"{path} is not a checkpoint")
    r = _Reader(data)
    r.o = 8
    ell, d, P, m, prec, target = r.take("iiiiii")
    adim = r.vec("i4")
    n, eg_n = r.take("ii")
    eg_last = r.take("d")
    e1n, e1v = r.vec("i4"), r.vec("f8")
    ern, erv = r.vec("i4"), r.vec("f8")
    Ls: List[Block] = []
    Rs: List[Block] = []
    prev, prev2 = [], []
    for _ in range(P):
        Ls.append(_block(r))
        Rs.append(_block(r))
        prev.append(_truncation(r, d))
        prev2.append(_truncation(r, d))
    if r.o != len(data):
        raise ValueError("trailing bytes in checkpoint")
    return dict(ell=ell, d=d, P=P, m=m, prec=prec, target=target, adim=adim, n=n, eg_n=eg_n, eg_last=eg_last,
                e1=dict(zip(e1n.tolist(), e1v.tolist())), eps1=dict(zip(ern.tolist(), erv.tolist())),
                L=Ls, R=Rs, prev=prev, prev2=prev2)


def load_state(path: str, mpo, m: int, **kw) -> ParallelIDMRG:
    """An oracle ParallelIDMRG positioned where the saved run stood: same n,
    environments, the last two truncations and the e_g / eps history."""
    ck = read_checkpoint(path)
    dims = [w.shape[0] for w in mpo.W] + [mpo.W[0].shape[0]]
    if ck["ell"] != len(mpo.W) or list(ck["adim"]) != dims or ck["m"] != m:
        raise ValueError("checkpoint of another MPO or m")
    ref = ParallelIDMRG.from_mpo(mpo, m=m, target=ck["target"], **kw)
    ref.n = ck["n"]
    ref.L, ref.R = ck["L"], ck["R"]
    ref.prev, ref.prev2 = ck["prev"], ck["prev2"]
    ref.e1 = {-1: 0.0, **{int(k): float(v) for k, v in ck["e1"].items()}}
    ref.eps1 = {int(k): float(v) for k, v in ck["eps1"].items()}
    return ref
