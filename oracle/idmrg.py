"""Parallel iDMRG, plain FP64 numpy (Sec. 2 Steps 1-7 with Sec. 3 Steps 2', 3', 5').

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  Nothing here is tuned:
every contraction is written out with dense arrays, every step follows the
paper's order.  Sites and superblocks are 0-based: superblock p (the paper's
i = p + 1) at iteration n covers the sites [2p, 2p + 2n + 1], its centre sites
are c1 = f(2p + n) and c2 = f(2p + n + 1) with f(k) = k mod l (Sec. 3, Step 2'),
its left block is L^(n-1) of pair p and its right block is R^(n-1) of pair
p + 1 (mod l/2).

Conventions
-----------
* A block is ``Block(op, q)``: ``op[a, x, y] = <x| O_a |y>`` for MPO channel a
  and block basis states x, y; ``q[x]`` is 2 Sz of state x.  Left blocks carry
  the channels of the bond to their right, right blocks those of the bond to
  their left.
* ``W[a, b, s, t] = <s| W(a,b) |t>`` (see ``workloads.mpo``).
* A superblock wavefunction is ``psi[x, s, t, y]`` (left block, site c1,
  site c2, right block), non-zero only where the charges add up to the target.
* All data are real, so the complex conjugations of Eqs. L, R and
  wfprediction are the identity.

Readings of points the paper leaves open (each marked where used):
R1 singular values are kept in descending order (the printed ascending
   inequality of Step 4 contradicts "keep beta = 1..m" of Eqs. fid2, tru);
R2 the cut never splits a group of equal singular values: keep the largest
   D <= m with lam_{D+1} < lam_D (1 - tie_rel); singular values at or below
   zero_rel * lam_max are treated as zero and dropped (Step 4, Step 6).
   tie_rel = 1e-7: states degenerate by symmetry (SU(2) multiplets spread over
   the 2Sz sectors) come out of any eigensolver stopped at a residual tol |E|
   split by up to about tol |E| / gap, i.e. ~1e-9 relative near the cut for
   tol = 1e-12; a smaller tie_rel would let solver rounding decide the cut;
R3 in the prediction, lam^(n-2) <= zero_rel * max(lam^(n-2)) counts as zero;
R4 in Eq. wfprediction lam^(n-2) and u^(n-1) belong to superblock i+1 and
   v^(n-1), lam^(n-1) (left factor) to superblock i; i+1 wraps to 1;
R5 Lanczos stops when the residual b_k |y_k| of the lowest Ritz pair is at or
   below tol * max(1, |theta|), or on breakdown, or after maxit matvecs;
R6 energy per site (Step 5'): estimated when (n + 1) mod l == 0 from
   superblock 1 (p = 0); the truncation error of Eq. tru is the maximum of
   eps^(n)_1 over the last l iterations.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np
from scipy.linalg import eigh_tridiagonal

from . import rng


@dataclass
class Block:
    op: np.ndarray  # [w, D, D]
    q: np.ndarray   # [D]


# ---------------------------------------------------------------- MPO checks
def check_mpo(W: List[np.ndarray], phys_charge: np.ndarray, bond_charge: List[np.ndarray]) -> None:
    """The boundary conventions the method relies on (Sec. 2, Eq. mpo): channel 0
    of each bond is the completed term, the last channel the identity; W(0,0)
    = W(last,last) = 1, row 0 and the last column hold nothing else; every
    non-zero entry conserves 2 Sz."""
    ell = len(W)
    for k, w in enumerate(W):
        a, b = w.shape[:2]
        assert a == len(bond_charge[k]) and b == len(bond_charge[(k + 1) % ell])
        I = np.eye(w.shape[2])
        assert np.array_equal(w[0, 0], I) and np.array_equal(w[-1, -1], I)
        assert not np.any(w[0, 1:]) and not np.any(w[:-1, -1])
        dq = phys_charge[:, None] - phys_charge[None, :]
        for x in range(a):
            for y in range(b):
                nz = w[x, y] != 0
                need = bond_charge[(k + 1) % ell][y] - bond_charge[k][x]
                assert np.all(dq[nz] == need), (k, x, y)


def initial_blocks(W, phys_charge):
    """Step 1: L^(0) of pair p is the last row of W at site 2p, R^(0) the first
    column of W at site 2p+1 (0-based sites)."""
    ell = len(W)
    Ls = [Block(np.ascontiguousarray(W[2 * p][-1]), phys_charge.copy()) for p in range(ell // 2)]
    Rs = [Block(np.ascontiguousarray(W[2 * p + 1][:, 0]), phys_charge.copy()) for p in range(ell // 2)]
    return Ls, Rs


# ------------------------------------------------------------- Step 3: H_eff
def heff_apply(L: Block, W1: np.ndarray, W2: np.ndarray, R: Block, psi: np.ndarray) -> np.ndarray:
    """(L W1 W2 R) psi, the superblock Hamiltonian of Step 3 applied to psi:
    out[x,s,t,y] = sum L[a,x,x'] W1[a,b,s,s'] W2[b,c,t,t'] R[c,y,y'] psi[x',s',t',y'].
    The expanded blocks of Step 2' (script L = L W1, script R = W2 R) are
    never formed; the contraction order is L, W1, W2, R."""
    T1 = np.tensordot(L.op, psi, axes=([2], [0]))            # [a, x, s', t', y']
    T2 = np.tensordot(W1, T1, axes=([0, 3], [0, 2]))          # [b, s, x, t', y']
    T3 = np.tensordot(W2, T2, axes=([0, 3], [0, 3]))          # [c, t, s, x, y']
    out = np.tensordot(R.op, T3, axes=([0, 2], [0, 4]))       # [y, t, s, x]
    return np.ascontiguousarray(out.transpose(3, 2, 1, 0))


def heff_dense(L: Block, W1: np.ndarray, W2: np.ndarray, R: Block) -> np.ndarray:
    """Explicit superblock matrix sum_{a,b,c} L_a (x) W1_ab (x) W2_bc (x) R_c
    (Kronecker products; rows/columns in psi's C order).  Tiny sizes only."""
    wa, wb = W1.shape[:2]
    wc = W2.shape[1]
    D = L.op.shape[1] * W1.shape[2] * W2.shape[2] * R.op.shape[1]
    H = np.zeros((D, D))
    for a in range(wa):
        for b in range(wb):
            if not W1[a, b].any():
                continue
            for c in range(wc):
                if not W2[b, c].any():
                    continue
                H += np.kron(np.kron(np.kron(L.op[a], W1[a, b]), W2[b, c]), R.op[c])
    return H


def sector_mask(qL, qp, qR, target=0) -> np.ndarray:
    tot = qL[:, None, None, None] + qp[None, :, None, None] + qp[None, None, :, None] + qR[None, None, None, :]
    return tot == target


# ------------------------------------------------------------ Step 3: solver
def lanczos(matvec, v0: np.ndarray, tol: float = 1e-12, maxit: int = 300):
    """Lowest eigenpair by Lanczos with full re-orthogonalisation (classical
    Gram-Schmidt applied twice).  Stopping rule R5.  Returns
    (theta, psi (unit norm), number of matvecs, converged)."""
    v = v0 / np.linalg.norm(v0)
    V = [v]
    alpha: List[float] = []
    beta: List[float] = []
    theta, y, converged = 0.0, np.ones(1), False
    for k in range(maxit):
        w = matvec(V[k])
        a = float(np.dot(V[k], w))
        w = w - a * V[k]
        if k > 0:
            w = w - beta[k - 1] * V[k - 1]
        B = np.array(V)
        for _ in range(2):
            w = w - B.T @ (B @ w)
        b = float(np.linalg.norm(w))
        alpha.append(a)
        ev, evec = eigh_tridiagonal(np.array(alpha), np.array(beta), select="i", select_range=(0, 0))
        theta, y = float(ev[0]), evec[:, 0]
        scale = max(1.0, abs(theta))
        if b * abs(y[-1]) <= tol * scale or b <= 1e-14 * scale:
            converged = True
            break
        beta.append(b)
        V.append(w / b)
    psi = np.array(V[: len(alpha)]).T @ y
    psi = psi / np.linalg.norm(psi)
    return theta, psi, len(alpha), converged


# ------------------------------------------------------------- Step 4: SVD
@dataclass
class Truncation:
    U: np.ndarray        # [D_L, d, k]
    V: np.ndarray        # [d, D_R, k]
    lam: np.ndarray      # [k]   kept singular values, in basis order
    q: np.ndarray        # [k]   2 Sz of the kept left states (right states carry -q)
    lam_all: np.ndarray  # every singular value, descending
    eps: float           # Eq. tru
    eps_best: float      # Eq. fid2 (best fidelity error)


def truncate(psi, qL, qp, qR, m: int, tie_rel: float = 1e-7, zero_rel: float = 1e-12,
             target: int = 0) -> Truncation:
    """Step 4 and the truncation of Step 6.  psi is split as (x s) x (t y); for
    every charge Q of the left half the block with rows of charge Q and columns
    of charge target - Q is decomposed by numpy's SVD.  Kept states: readings
    R1, R2.  The kept states are ordered by Q, then by descending singular
    value.  Singular values are not renormalised after the cut (Step 4 fixes
    sum lam^2 = 1 over all of them)."""
    DL, d, _, DR = psi.shape
    M = psi.reshape(DL * d, d * DR)
    ql = (qL[:, None] + qp[None, :]).ravel()
    qr = (qp[:, None] + qR[None, :]).ravel()
    cand = []
    blocks = {}
    for Q in np.unique(ql):
        rows = np.nonzero(ql == Q)[0]
        cols = np.nonzero(qr == target - Q)[0]
        if len(rows) == 0 or len(cols) == 0:
            continue
        u, s, vt = np.linalg.svd(M[np.ix_(rows, cols)], full_matrices=False)
        blocks[int(Q)] = (rows, cols, u, vt)
        cand += [(float(lam), int(Q), k) for k, lam in enumerate(s)]
    cand.sort(key=lambda c: (-c[0], abs(c[1]), c[1], c[2]))
    lam_all = np.array([c[0] for c in cand])
    nz = int(np.sum(lam_all > zero_rel * lam_all[0]))
    top = min(m, nz)
    D = top
    while D > 0 and D < nz and not (lam_all[D] < lam_all[D - 1] * (1.0 - tie_rel)):
        D -= 1
    if D == 0:
        D = top
    kept = sorted(cand[:D], key=lambda c: (c[1], c[2]))
    U = np.zeros((DL * d, D))
    V = np.zeros((d * DR, D))
    for col, (lam, Q, k) in enumerate(kept):
        rows, cols, u, vt = blocks[Q]
        U[rows, col] = u[:, k]
        V[cols, col] = vt[k]
    lam = np.array([c[0] for c in kept])
    w2 = float(np.sum(lam ** 2))
    return Truncation(U=U.reshape(DL, d, D), V=V.reshape(d, DR, D), lam=lam,
                      q=np.array([c[1] for c in kept], dtype=np.int64), lam_all=lam_all,
                      eps=1.0 - w2, eps_best=1.0 - np.sqrt(w2))


# ----------------------------------------------------- Step 6: block spin
def update_left(L: Block, W1: np.ndarray, U: np.ndarray, qU: np.ndarray) -> Block:
    """Eq. L: L'[b,j,k] = sum u[x,s,j] L[a,x,x'] W1[a,b,s,s'] u[x',s',k]."""
    X = np.tensordot(L.op, U, axes=([2], [0]))            # [a, x, s', k]
    Y = np.tensordot(W1, X, axes=([0, 3], [0, 2]))         # [b, s, x, k]
    op = np.tensordot(U, Y, axes=([0, 1], [2, 1]))         # [j, b, k]
    return Block(np.ascontiguousarray(op.transpose(1, 0, 2)), qU.copy())


def update_right(R: Block, W2: np.ndarray, V: np.ndarray, qV: np.ndarray) -> Block:
    """Eq. R: R'[b,j,k] = sum v[s,y,j] W2[b,c,s,s'] R[c,y,y'] v[s',y',k]."""
    X = np.tensordot(R.op, V, axes=([2], [1]))             # [c, y, s', k]
    Y = np.tensordot(W2, X, axes=([1, 3], [0, 2]))          # [b, s, y, k]
    op = np.tensordot(V, Y, axes=([0, 1], [1, 2]))          # [j, b, k]
    return Block(np.ascontiguousarray(op.transpose(1, 0, 2)), qV.copy())


# ------------------------------------------------------ Step 3': prediction
def predict(lam_i, V_i, U_j, lam_j, lam_jj, zero_rel: float = 1e-12) -> np.ndarray:
    """Eq. wfprediction with reading R4:
    u~[b,t,g] = u_{i+1}[b,t,g] lam_{i+1}[g] / lam''_{i+1}[b]   (0 where lam'' is zero, R3),
    psi~[a,s,t,g] = sum_b lam_i[a] v_i[s,b,a] u~[b,t,g]."""
    inv = np.where(lam_jj > zero_rel * np.max(lam_jj), 1.0 / np.where(lam_jj > 0, lam_jj, 1.0), 0.0)
    ut = U_j * inv[:, None, None] * lam_j[None, None, :]           # [b, t, g]
    vl = V_i * lam_i[None, None, :]                                  # [s, b, a]
    out = np.tensordot(vl, ut, axes=([1], [0]))                      # [s, a, t, g]
    return np.ascontiguousarray(out.transpose(1, 0, 2, 3))


def fidelity_error(psi_tilde: np.ndarray, psi: np.ndarray) -> float:
    """Eq. fid1 for a unit-norm psi."""
    return 1.0 - abs(float(np.vdot(psi_tilde, psi))) / float(np.linalg.norm(psi_tilde))


def bond_energy(psi: np.ndarray, W1: np.ndarray, W2: np.ndarray) -> float:
    """<psi| h(c1,c2) |psi> with h(c1,c2) = sum_b W1(last,b) (x) W2(b,0) over the
    channels b that open on c1 and close on c2 (b != 0, last): the bond terms
    between the two centre sites."""
    d = W1.shape[2]
    h = np.zeros((d * d, d * d))
    for b in range(1, W1.shape[1] - 1):
        h += np.kron(W1[-1, b], W2[b, 0])
    h4 = h.reshape(d, d, d, d)
    return float(np.einsum("xsty,stuv,xuvy->", psi, h4, psi))


# ------------------------------------------------------------------ driver
@dataclass
class StepReport:
    n: int
    energies: np.ndarray
    iters: np.ndarray
    eps: np.ndarray
    eps_best: np.ndarray
    fidelity: np.ndarray
    bond: np.ndarray
    kept: np.ndarray
    lam_all: List[np.ndarray]
    e_g: Optional[float]


class ParallelIDMRG:
    """The parallel iDMRG of Sec. 3 for an l-site periodic MPO.

    ``step()`` performs one parallel iteration n (Steps 2', 3', 4, 5', 6, 7)
    on all l/2 superblocks, in the order p = 0 .. l/2 - 1 (the superblocks are
    independent within an iteration, Sec. 2, last paragraph)."""

    def __init__(self, W, phys_charge, bond_charge, m: int, lanczos_tol: float = 1e-12,
                 lanczos_maxit: int = 300, predict: bool = True, seed: int = 0,
                 zero_rel: float = 1e-12, tie_rel: float = 1e-7, target: int = 0):
        self.W = [np.asarray(w, dtype=np.float64) for w in W]
        self.qp = np.asarray(phys_charge, dtype=np.int64)
        check_mpo(self.W, self.qp, [np.asarray(c) for c in bond_charge])
        self.ell = len(self.W)
        assert self.ell % 2 == 0
        self.P = self.ell // 2
        self.m, self.tol, self.maxit = m, lanczos_tol, lanczos_maxit
        self.use_prediction, self.seed = predict, seed
        self.zero_rel, self.tie_rel, self.target = zero_rel, tie_rel, target
        self.L, self.R = initial_blocks(self.W, self.qp)
        self.n = 1
        self.e1: Dict[int, float] = {-1: 0.0}
        self.eps1: Dict[int, float] = {}
        self.prev: List[Optional[Truncation]] = [None] * self.P     # at n-1
        self.prev2: List[Optional[Truncation]] = [None] * self.P    # at n-2
        self.last_psi: List[Optional[np.ndarray]] = [None] * self.P

    @classmethod
    def from_mpo(cls, mpo, m: int, **kw):
        return cls(mpo.W, mpo.phys_charge, mpo.bond_charge, m, **kw)

    def centre_sites(self, p: int):
        return (2 * p + self.n) % self.ell, (2 * p + self.n + 1) % self.ell

    def superblock(self, p: int):
        c1, c2 = self.centre_sites(p)
        return self.L[p], self.W[c1], self.W[c2], self.R[(p + 1) % self.P]

    def start_vector(self, p: int) -> np.ndarray:
        L, W1, W2, R = self.superblock(p)
        mask = sector_mask(L.q, self.qp, R.q, self.target)
        if self.n >= 3 and self.use_prediction:
            j = (p + 1) % self.P
            a, b, c = self.prev[p], self.prev[j], self.prev2[j]
            v = predict(a.lam, a.V, b.U, b.lam, c.lam, self.zero_rel)
        else:
            v = rng.start_vector(self.seed, self.n, p, mask.size).reshape(mask.shape)
        return np.where(mask, v, 0.0)

    def solve(self, p: int, v0: np.ndarray):
        L, W1, W2, R = self.superblock(p)
        shape = v0.shape
        mv = lambda x: heff_apply(L, W1, W2, R, x.reshape(shape)).ravel()  # noqa: E731
        e, psi, it, conv = lanczos(mv, v0.ravel(), self.tol, self.maxit)
        return e, psi.reshape(shape), it, conv

    def superblock_step(self, p: int) -> dict:
        """Steps 3', 3, 4 and 6 of superblock p at the current n, without
        changing the state (the superblocks of one iteration are independent):
        start vector, solve, truncation, the new blocks and the reported
        quantities."""
        L, W1, W2, R = self.superblock(p)
        v0 = self.start_vector(p)
        e, psi, it, _ = self.solve(p, v0)
        t = truncate(psi, L.q, self.qp, R.q, self.m, self.tie_rel, self.zero_rel, self.target)
        fid = fidelity_error(v0, psi) if (self.n >= 3 and self.use_prediction) else np.nan
        return dict(energy=e, iters=it, psi=psi, trunc=t, fidelity=fid, bond=bond_energy(psi, W1, W2),
                    newL=update_left(L, W1, t.U, t.q), newR=update_right(R, W2, t.V, self.target - t.q),
                    start_norm=float(np.linalg.norm(v0)))

    def step(self) -> StepReport:
        return self.step_range(0, self.P)

    def step_range(self, p0: int, p1: int) -> StepReport:
        """One parallel iteration on the superblocks p0 .. p1-1 only (the
        others are another worker's, Sec. 3): their blocks and truncations are
        renewed, those of the other pairs keep their old values (a worker
        receives the one it needs from its neighbour); entries of the report
        outside the range are left at zero / NaN.  e_g needs superblock 0."""
        n, P = self.n, self.P
        newL, newR, trunc = list(self.L), list(self.R), list(self.prev)
        rep = dict(energies=np.zeros(P), iters=np.zeros(P, dtype=int), eps=np.zeros(P),
                   eps_best=np.zeros(P), fidelity=np.full(P, np.nan), bond=np.zeros(P),
                   kept=np.zeros(P, dtype=int), lam_all=[None] * P)
        for p in range(p0, p1):
            r = self.superblock_step(p)
            t = r["trunc"]
            newL[p], newR[p] = r["newL"], r["newR"]
            trunc[p] = t
            self.last_psi[p] = r["psi"]
            rep["energies"][p] = r["energy"]
            rep["iters"][p] = r["iters"]
            rep["eps"][p] = t.eps
            rep["eps_best"][p] = t.eps_best
            rep["fidelity"][p] = r["fidelity"]
            rep["bond"][p] = r["bond"]
            rep["kept"][p] = len(t.lam)
            rep["lam_all"][p] = t.lam_all
        # Step 7 with the rotation of Step 2': R^(n) of pair p+1 is the right
        # block of superblock p at n+1; lambda^(n-1) becomes lambda^(n-2).
        self.L, self.R = newL, newR
        self.prev2, self.prev = self.prev, trunc
        e_g = None
        if p0 == 0 < p1:
            self.e1[n] = float(rep["energies"][0])
            self.eps1[n] = float(rep["eps"][0])
            e_g = self.energy_per_site(n)
        self.n = n + 1
        return StepReport(n=n, e_g=e_g, **rep)

    def energy_per_site(self, n: int) -> Optional[float]:
        """Step 5': e_g^(n) = (e_1^(n) - e_1^(n-l)) / 2l when (n+1) mod l == 0."""
        if (n + 1) % self.ell != 0:
            return None
        return (self.e1[n] - self.e1[n - self.ell]) / (2.0 * self.ell)

    def truncation_error(self) -> float:
        """Eq. tru with reading R6: max of eps^(n)_1 over the last l iterations."""
        ns = sorted(self.eps1)[-self.ell:]
        return max(self.eps1[k] for k in ns)
