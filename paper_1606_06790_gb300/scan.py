"""The m scan of Sec. 5: e_g against the truncation error eps for several m,
extrapolated to eps -> 0 with a quadratic polynomial (the paper's Eq. tru
and the quadratic fit of its Fig. ene_vs_tru); the same fit serves the bond
strengths and Delta+- of Eqs. diff1, diff2.  Also the exponential fit of a
spin-spin correlation function that gives the paper's correlation length.

Every point runs through the C ABI (`idmrg_run`: unit-cell steps until two
successive e_g estimates agree to `de_tol`); only the final least-squares fit
of a handful of (eps, e_g) points is host arithmetic.
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

import numpy as np


def m_scan(W, phys_charge, bond_charge, ms: Sequence[int], prec: str = "fp64", max_steps: int = 400,
           de_tol: float = 1e-8, **opts) -> List[Dict[str, float]]:
    """One converged run per m: [{m, e_g, eps, steps, converged}]."""
    from . import Context
    out = []
    for m in ms:
        ctx = Context(W, phys_charge, bond_charge, m=int(m), prec=prec, **opts)
        try:
            e_g, eps, steps, conv = ctx.run(max_steps, de_tol)
        finally:
            ctx.close()
        out.append(dict(m=int(m), e_g=e_g, eps=eps, steps=steps, converged=conv))
    return out


def extrapolate(eps: Sequence[float], e: Sequence[float], degree: int = 2) -> Tuple[float, float]:
    """Least-squares polynomial in eps through the points; returns the value
    at eps = 0 and its standard deviation (from the residual variance and the
    normal matrix; 0 when the points determine the polynomial exactly)."""
    x = np.asarray(eps, dtype=np.float64)
    y = np.asarray(e, dtype=np.float64)
    A = np.vander(x, degree + 1, increasing=True)
    coef, _, _, _ = np.linalg.lstsq(A, y, rcond=None)
    dof = len(x) - (degree + 1)
    if dof <= 0:
        return float(coef[0]), 0.0
    r = y - A @ coef
    s2 = float(r @ r) / dof
    cov = s2 * np.linalg.inv(A.T @ A)
    return float(coef[0]), float(np.sqrt(max(cov[0, 0], 0.0)))


def fit_correlation_length(r: Sequence[float], c: Sequence[float], r_min: float = 5.0) -> Tuple[float, float]:
    """Least-squares fit of ln|c(r)| = a - r / xi over the points with r > r_min
    (Sec. 5: |<s_i . s_2>| decays as exp(-|r_i - r_2| / xi)); returns xi and its
    standard deviation from the residual variance of the fit (0 with two
    points).  Points with c = 0 are skipped."""
    x = np.asarray(r, dtype=np.float64)
    y = np.abs(np.asarray(c, dtype=np.float64))
    keep = (x > r_min) & (y > 0.0)
    x, y = x[keep], np.log(y[keep])
    if len(x) < 2:
        raise ValueError("need two points beyond r_min")
    A = np.vander(x, 2, increasing=True)
    coef, _, _, _ = np.linalg.lstsq(A, y, rcond=None)
    slope = float(coef[1])
    xi = -1.0 / slope
    dof = len(x) - 2
    if dof <= 0:
        return xi, 0.0
    res = y - A @ coef
    s2 = float(res @ res) / dof
    sd_slope = float(np.sqrt(max(s2 * np.linalg.inv(A.T @ A)[1, 1], 0.0)))
    return xi, sd_slope / (slope * slope)
