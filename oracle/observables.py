"""Observables of the uniform MPS of the parallel iDMRG (Sec. 3, Eq. mps2) and
the quantities of the paper's benchmark section built on them: bond strengths
<s_i . s_i'>, their spread Delta+- (Eqs. diff1, diff2), spin-spin correlations
along the chain and the correlation length.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  Everything is dense
numpy float64; the transfer matrix is formed explicitly and diagonalised by
``numpy.linalg.eig``, so the sizes are small (bond dimension <= ~24).

Conventions
-----------
* A site tensor is ``A[s, a, b]`` (physical state s, left bond a, right
  bond b); a unit is the list of its l site tensors, A[k] carrying the
  lattice site (s0 + k) mod l.
* An operator is ``O[s, t] = <s| O |t>``.
* A left environment is ``rho[a, a']`` (bra index first): one site maps it to
  ``sum_{s,t} O[s,t] A[s]^T rho A[t]``; a right environment ``r[b, b']`` maps
  to ``sum_{s,t} O[s,t] A[s] r A[t]^T``.
* Lattice sites are numbered along the infinite chain; site x carries the
  MPO site x mod l.

Readings (each marked where used):
R7 the unit of Eq. mps2 after iteration n is V^(n)_1^T u~^(n)_2 ... V^(n)_{l/2}^T
   u~^(n)_1 with u~^(n)_{i+1} = (lam^(n-1)_{i+1})^-1 u^(n)_{i+1} lam^(n)_{i+1},
   the same scaled tensors Eq. wfprediction uses at iteration n + 1 (R3: a
   lam^(n-1) at or below zero_rel * max counts as zero, its rows vanish); V^T
   carries site f(2i + n) and u~ site f(2i + n + 1) (1-based i, Sec. 3 Step 2').
   The unit is not exactly right-normalised away from convergence, so every
   expectation value uses the dominant left and right eigenvectors of its
   transfer matrix instead of assuming a canonical form.
R8 <s_i . s_i'> = <Sz Sz> + (<S+ S-> + <S- S+>) / 2, evaluated on the uniform MPS
   (Sec. 4.5, bond strength); Delta+- of Eqs. diff1, diff2 are taken over the
   values a caller groups as equivalent.
R9 the correlation length is xi = -1 / ln(|t2| / t1) unit cells, t1 > |t2| the
   two largest moduli of the unit's transfer-matrix eigenvalues (the paper fits
   the decay of the correlation function; its asymptotic rate is this one).
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np

SZ = np.array([[0.5, 0.0], [0.0, -0.5]])
SP = np.array([[0.0, 1.0], [0.0, 0.0]])
SM = np.array([[0.0, 0.0], [1.0, 0.0]])


# ------------------------------------------------------------- the unit
def uniform_unit(state) -> Tuple[List[np.ndarray], int]:
    """Eq. mps2 (reading R7) from a ``ParallelIDMRG`` after at least two
    completed iterations.  Returns (site tensors, s0): A[k] carries lattice
    site s0 + k (mod l)."""
    P, ell = state.P, state.ell
    n = state.n - 1                       # last completed iteration
    if n < 2 or any(t is None for t in state.prev) or any(t is None for t in state.prev2):
        raise ValueError("the unit needs two completed iterations")
    A: List[np.ndarray] = []
    for p in range(P):
        q = (p + 1) % P
        a, b, bb = state.prev[p], state.prev[q], state.prev2[q]
        # V^T: A[s][alpha, beta] = v_p[s, beta, alpha]
        A.append(np.ascontiguousarray(a.V.transpose(0, 2, 1)))
        lam2 = bb.lam
        inv = np.where(lam2 > state.zero_rel * np.max(lam2), 1.0 / np.where(lam2 > 0, lam2, 1.0), 0.0)
        ut = b.U * inv[:, None, None] * b.lam[None, None, :]        # [beta, t, gamma]
        A.append(np.ascontiguousarray(ut.transpose(1, 0, 2)))
    return A, (n + 1) % ell


# ------------------------------------------------------ one-site maps
def site_left(rho: np.ndarray, A: np.ndarray, O: np.ndarray = None) -> np.ndarray:
    d = A.shape[0]
    O = np.eye(d) if O is None else O
    out = np.zeros((A.shape[2], A.shape[2]))
    for s in range(d):
        for t in range(d):
            if O[s, t] != 0.0:
                out += O[s, t] * (A[s].T @ rho @ A[t])
    return out


def site_right(r: np.ndarray, A: np.ndarray, O: np.ndarray = None) -> np.ndarray:
    d = A.shape[0]
    O = np.eye(d) if O is None else O
    out = np.zeros((A.shape[1], A.shape[1]))
    for s in range(d):
        for t in range(d):
            if O[s, t] != 0.0:
                out += O[s, t] * (A[s] @ r @ A[t].T)
    return out


# ---------------------------------------------------- transfer matrix
def transfer_matrix(A: Sequence[np.ndarray]) -> np.ndarray:
    """The unit's transfer matrix acting on row-major vec(rho) of a left
    environment: one site is sum_s kron(A[s]^T, A[s]^T) (vec(X^T rho Y) =
    kron(X^T, Y^T) vec(rho) for row-major vec); the unit multiplies them in
    site order."""
    T = np.eye(A[0].shape[1] ** 2)
    for Ak in A:
        Tk = sum(np.kron(Ak[s].T, Ak[s].T) for s in range(Ak.shape[0]))
        T = Tk @ T
    return T


def spectrum(A: Sequence[np.ndarray]) -> np.ndarray:
    """Eigenvalues of the unit's transfer matrix, largest modulus first."""
    ev = np.linalg.eigvals(transfer_matrix(A))
    return ev[np.argsort(-np.abs(ev), kind="stable")]


def fixed_points(A: Sequence[np.ndarray]) -> Tuple[np.ndarray, np.ndarray, float]:
    """Dominant left and right eigenvectors of the unit (at the bond before
    A[0]) and the dominant eigenvalue t1, from the dense eigendecomposition of
    the transfer matrix and of its transpose; normalised to (l|r) = 1 with a
    positive trace of l."""
    T = transfer_matrix(A)
    D = A[0].shape[1]
    w, v = np.linalg.eig(T)
    k = int(np.argmax(np.abs(w)))
    t1 = float(np.real(w[k]))
    lv = np.real(v[:, k]).reshape(D, D)
    w2, v2 = np.linalg.eig(T.T)
    k2 = int(np.argmax(np.abs(w2)))
    rv = np.real(v2[:, k2]).reshape(D, D)
    if np.trace(lv) < 0:
        lv = -lv
    rv = rv / float(np.sum(lv * rv))
    return lv, rv, t1


def correlation_length(A: Sequence[np.ndarray]) -> float:
    """Reading R9, in unit cells."""
    ev = np.abs(spectrum(A))
    if len(ev) < 2 or ev[1] == 0.0:
        return 0.0
    return float(-1.0 / np.log(ev[1] / ev[0]))


# ----------------------------------------------------- two-point functions
def correlation(A: Sequence[np.ndarray], s0: int, Oa: np.ndarray, Ob: np.ndarray, i: int, j: int) -> float:
    """<Oa_i Ob_j> (i < j, lattice sites) on the infinite uniform MPS: the
    left fixed point carried to the bond left of site i, the sites i..j
    applied with Oa at i and Ob at j, closed with the right fixed point
    carried back to the bond right of site j; divided by the same walk with
    identities, so no normalisation of the fixed points enters."""
    if not i < j:
        raise ValueError("need i < j")
    ell = len(A)
    lv, rv, _ = fixed_points(A)
    ki = (i - s0) % ell
    kj = (j - s0) % ell
    L = lv
    for k in range(ki):
        L = site_left(L, A[k])
    R = rv
    for k in range(ell - 1, kj, -1):
        R = site_right(R, A[k])
    num, den = L, L
    for x in range(i, j + 1):
        Ak = A[(x - s0) % ell]
        O = Oa if x == i else (Ob if x == j else None)
        num = site_left(num, Ak, O)
        den = site_left(den, Ak)
    return float(np.sum(num * R) / np.sum(den * R))


def spin_dot(A: Sequence[np.ndarray], s0: int, i: int, j: int) -> float:
    """<s_i . s_j> for spin 1/2 (reading R8)."""
    return (correlation(A, s0, SZ, SZ, i, j)
            + 0.5 * (correlation(A, s0, SP, SM, i, j) + correlation(A, s0, SM, SP, i, j)))


def delta_pm(values: Sequence[float]) -> Tuple[float, float, float]:
    """Eqs. diff1, diff2: (average, max - average, min - average) of bond
    strengths that translational symmetry makes equal."""
    v = np.asarray(values, dtype=np.float64)
    avg = float(np.sum(v) / len(v))
    return avg, float(np.max(v)) - avg, float(np.min(v)) - avg
