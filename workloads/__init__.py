"""Seeded, synthetic inputs shared by the FP64 oracle, the tests and the benchmark.

This package only *describes* workloads: lattice bond lists, the matrix product
operator (MPO) that encodes them, coupling draws from a seed.  It contains none
of the iDMRG arithmetic (no environment, matvec, eigen-solve, SVD or prediction
step), so both sides of every parity check can take their inputs from here
without sharing any of the method's code.
"""
from .lattices import (  # noqa: F401
    Bond,
    chain_bonds,
    random_chain_bonds,
    j1j2_chain_bonds,
    dimerized_chain_bonds,
    xx_chain_bonds,
    yc4_j1j2_bonds,
    kagome_yc8_bonds,
    open_chain_bonds,
)
from .mpo import MPO, build_mpo  # noqa: F401
from .configs import CONFIGS, disorder_batch, make_config  # noqa: F401
