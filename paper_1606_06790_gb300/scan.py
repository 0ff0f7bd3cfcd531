"""The m scan of Sec. 4.4: e_g against the truncation error eps for several m,
extrapolated to eps -> 0 with a quadratic polynomial (the paper's Eq. tru
and the quadratic fit of its Fig. ene_vs_tru); the same fit serves the bond
strengths and Delta+- of Eqs. diff1, diff2.  Also the exponential fit of a
spin-spin correlation function that gives the paper's correlation length.

Every point runs through the C ABI (`idmrg_run`: unit-cell steps until two
successive e_g estimates agree to `de_tol`), and so do the fits
(`idmrg_extrapolate`, `idmrg_fit_correlation_length`: host code of the
library); this module only marshals the arguments.
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
    """Least-squares polynomial in eps through the points (idmrg_extrapolate);
    returns the value at eps = 0 and its standard deviation (0 when the points
    determine the polynomial exactly)."""
    import ctypes as C
    from . import _dptr, load_library
    x = np.ascontiguousarray(np.asarray(eps, dtype=np.float64).ravel())
    y = np.ascontiguousarray(np.asarray(e, dtype=np.float64).ravel())
    if len(x) != len(y):
        raise ValueError("eps and e differ in length")
    v0, sd = C.c_double(), C.c_double()
    s = load_library().idmrg_extrapolate(_dptr(x, C.c_double), _dptr(y, C.c_double), len(x), int(degree),
                                         C.byref(v0), C.byref(sd))
    if s != 0:
        raise ValueError("extrapolate: too few points or a singular fit")
    return v0.value, sd.value


def fit_correlation_length(r: Sequence[float], c: Sequence[float], r_min: float = 5.0) -> Tuple[float, float]:
    """Least-squares fit of ln|c(r)| = a - r / xi over the points with r > r_min
    (Sec. 4.6: |<s_i . s_2>| decays as exp(-|r_i - r_2| / xi)), by
    idmrg_fit_correlation_length; returns xi and its standard deviation (0
    with two points).  Points with c = 0 are skipped."""
    import ctypes as C
    from . import _dptr, load_library
    x = np.ascontiguousarray(np.asarray(r, dtype=np.float64).ravel())
    y = np.ascontiguousarray(np.asarray(c, dtype=np.float64).ravel())
    if len(x) != len(y):
        raise ValueError("r and c differ in length")
    xi, sd = C.c_double(), C.c_double()
    s = load_library().idmrg_fit_correlation_length(_dptr(x, C.c_double), _dptr(y, C.c_double), len(x),
                                                    float(r_min), C.byref(xi), C.byref(sd))
    if s != 0:
        raise ValueError("need two points beyond r_min")
    return xi.value, sd.value
