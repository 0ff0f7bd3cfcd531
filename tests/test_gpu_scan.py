"""The m scan and eps -> 0 extrapolation of Sec. 4.4 through the library
(idmrg_run per m, idmrg_truncation_error) against the oracle's."""
import numpy as np
import pytest

from oracle.extrapolate import quadratic_fit, run_until_converged
from oracle.idmrg import ParallelIDMRG
from paper_1606_06790_gb300.scan import extrapolate, m_scan
from workloads import build_mpo, chain_bonds, random_chain_bonds

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("tf32x3", 1e-8)])
def test_m_scan_against_oracle(prec, tol):
    mpo = build_mpo(chain_bonds(4), 4)
    ms = (8, 12, 16)
    opts = {} if prec == "fp64" else {"lanczos_tol": 1e-13}
    pts = m_scan(mpo.W, mpo.phys_charge, mpo.bond_charge, ms, prec=prec, max_steps=60, de_tol=1e-7, **opts)
    ref = []
    for m in ms:
        r = ParallelIDMRG.from_mpo(mpo, m=m, **opts)
        ref.append(run_until_converged(r, 60, 1e-7))
    for p, (e_g, eps, steps, conv) in zip(pts, ref):
        assert abs(p["e_g"] - e_g) < tol
        assert abs(p["eps"] - eps) < tol
        assert p["converged"] == conv
        if prec == "fp64":
            assert p["steps"] == steps
    e0, sd = extrapolate([p["eps"] for p in pts], [p["e_g"] for p in pts])
    r0, _ = quadratic_fit([r[1] for r in ref], [r[0] for r in ref])
    assert abs(e0 - r0) < 100 * tol


def test_truncation_error_is_max_over_a_period():
    mpo = build_mpo(random_chain_bonds(8, 0.5, 1.5, 3), 8)
    import paper_1606_06790_gb300 as pkg
    ctx = pkg.Context(mpo.W, mpo.phys_charge, mpo.bond_charge, m=12)
    hist = [float(ctx.unit_cell_step()["eps"][0]) for _ in range(12)]
    assert ctx.truncation_error() == pytest.approx(max(hist[-8:]), abs=0.0)
    ctx.close()
