"""Sec. 4.4 of the paper (oracle side, test infrastructure): a run at fixed m
until e_g converges, the truncation error eps of the run (Eq. tru, reading
R6: the largest eps^(n)_1 over the last l iterations), the quadratic
extrapolation of e_g to eps -> 0, and the exponential fit of a correlation
function for the correlation length, both written from the normal equations.

Imported only by tests, smoke() and bench.py's reference arm."""
from __future__ import annotations

from typing import Optional, Tuple

import numpy as np

from .idmrg import ParallelIDMRG


def run_until_converged(ref: ParallelIDMRG, max_steps: int, de_tol: float) -> Tuple[float, float, int, bool]:
    """Steps until two successive e_g estimates differ by less than de_tol."""
    last: Optional[float] = None
    e_g = float("nan")
    for k in range(1, max_steps + 1):
        r = ref.step()
        if r.e_g is not None:
            e_g = r.e_g
            if last is not None and abs(e_g - last) < de_tol:
                return e_g, ref.truncation_error(), k, True
            last = e_g
    return e_g, ref.truncation_error(), max_steps, False


def quadratic_fit(eps, e) -> Tuple[float, float]:
    """e = c0 + c1 eps + c2 eps^2 by least squares: the normal equations
    (sum_k x_k^(i+j)) c = sum_k x_k^i y_k solved directly; the standard
    deviation of c0 is sqrt(s^2 [(A^T A)^-1]_00) with s^2 = RSS / (N - 3)."""
    x = np.asarray(eps, dtype=np.float64)
    y = np.asarray(e, dtype=np.float64)
    G = np.array([[np.sum(x ** (i + j)) for j in range(3)] for i in range(3)])
    b = np.array([np.sum(x ** i * y) for i in range(3)])
    c = np.linalg.solve(G, b)
    if len(x) <= 3:
        return float(c[0]), 0.0
    res = y - (c[0] + c[1] * x + c[2] * x * x)
    s2 = float(np.sum(res * res)) / (len(x) - 3)
    return float(c[0]), float(np.sqrt(max(s2 * np.linalg.inv(G)[0, 0], 0.0)))


def exponential_fit(r, c, r_min: float = 5.0) -> Tuple[float, float]:
    """ln|c| = a + b r over the points with r > r_min, by the 2 x 2 normal
    equations; xi = -1 / b and its standard deviation sd(b) / b^2 with
    sd(b)^2 = s^2 [(A^T A)^-1]_11, s^2 = RSS / (N - 2)."""
    x = np.asarray(r, dtype=np.float64)
    y = np.abs(np.asarray(c, dtype=np.float64))
    keep = (x > r_min) & (y > 0.0)
    x, y = x[keep], np.log(y[keep])
    if len(x) < 2:
        raise ValueError("the fit needs two points with r > r_min and c != 0")
    G = np.array([[len(x), np.sum(x)], [np.sum(x), np.sum(x * x)]])
    rhs = np.array([np.sum(y), np.sum(x * y)])
    a, b = np.linalg.solve(G, rhs)
    xi = -1.0 / b
    if len(x) <= 2:
        return float(xi), 0.0
    res = y - (a + b * x)
    s2 = float(np.sum(res * res)) / (len(x) - 2)
    sd_b = float(np.sqrt(max(s2 * np.linalg.inv(G)[1, 1], 0.0)))
    return float(xi), sd_b / (b * b)
