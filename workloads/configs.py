"""Named workloads (model, unit cell, kept states m) with their seeds.

Each entry gives the bond list and the iDMRG options of one workload.  The
random-bond draws use numpy's PCG64 with the stated seed; the Lanczos start
vectors for n = 1, 2 come from a counter-based generator inside each
implementation (see ``start_vector_seed``).
"""
from __future__ import annotations

from typing import Dict

from . import lattices as lat
from .mpo import build_mpo

CONFIGS: Dict[str, dict] = {
    # uniform S=1/2 chain, converges towards 1/4 - ln 2 per site
    "chain_l4_m32": dict(bonds=lambda: lat.chain_bonds(4), ell=4, m=32, steps=200,
                         lanczos_tol=1e-12),
    # random-bond chain, J_k ~ U[0.5, 1.5] (PCG64 seed 1606), 8 solves per step
    "randchain_l16_m256": dict(bonds=lambda: lat.random_chain_bonds(16, 0.5, 1.5, 1606),
                               ell=16, m=256, steps=40, lanczos_tol=1e-12),
    # J1-J2 square lattice on a 4-leg cylinder, snake order, two columns per cell
    "yc4_j1j2_l8_m1024": dict(bonds=lambda: lat.yc4_j1j2_bonds(1.0, 0.5), ell=8, m=1024,
                              steps=20, lanczos_tol=1e-12),
    # kagome Heisenberg model on a YC8 cylinder, 12-site cell
    "kagome_yc8_l12_m2048": dict(bonds=lambda: lat.kagome_yc8_bonds(1.0), ell=12, m=2048,
                                 steps=10, lanczos_tol=1e-12),
}


def make_config(name: str, **override):
    """Return (mpo, options dict) for a named workload."""
    cfg = dict(CONFIGS[name])
    cfg.update(override)
    mpo = build_mpo(cfg["bonds"](), cfg["ell"])
    opts = {k: v for k, v in cfg.items() if k not in ("bonds",)}
    return mpo, opts


def start_vector_seed() -> int:
    """Seed of the Lanczos start vectors for n = 1, 2 (0 for every workload)."""
    return 0


def disorder_batch(count: int = 64, lo: float = 0.2, hi: float = 1.8):
    """Disorder realisations r = 0..count-1 of the random-bond Heisenberg chain
    with uneven unit cells: l = (8, 12, 16, 24)[r % 4], m = (128, 256,
    512)[(r // 4) % 3], J_k ~ U[lo, hi] i.i.d. from PCG64 seed 1000 + r.
    Returns a list of (name, mpo, m)."""
    out = []
    for r in range(count):
        ell = (8, 12, 16, 24)[r % 4]
        m = (128, 256, 512)[(r // 4) % 3]
        bonds = lat.random_chain_bonds(ell, lo, hi, 1000 + r)
        out.append((f"disorder_r{r}_l{ell}_m{m}", build_mpo(bonds, ell), m))
    return out
