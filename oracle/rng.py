"""Counter-based SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) for Lanczos start vectors.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Output k (k = 0, 1, ...) of a SplitMix64 stream started at state s is
mix(s + (k + 1) * GAMMA) with GAMMA = 0x9E3779B97F4A7C15 and the mixing
function below, all modulo 2^64.  The iDMRG start vector of superblock p at
iteration n (Step 3: random for n = 1, 2) is built from it as follows:

* stream state  s_np = output number (1024 n + p) of the stream seeded by ``seed``;
* element k of the dense wavefunction psi[alpha, s, s', alpha'] (C order) gets
  2 * u_k - 1 with u_k = (output k of the stream s_np >> 11) * 2^-53,
  and elements outside the target charge sector are set to zero.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(state: int, count: int, first: int = 0) -> np.ndarray:
    """Outputs first .. first+count-1 of the stream with initial state ``state``."""
    k = np.arange(first + 1, first + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(state) + k * GAMMA
    return _mix(z)


def stream_state(seed: int, n: int, p: int) -> int:
    return int(splitmix64(seed, 1, first=1024 * n + p)[0])


def start_vector(seed: int, n: int, p: int, size: int) -> np.ndarray:
    """Uniform numbers in [-1, 1) for the dense elements 0 .. size-1."""
    z = splitmix64(stream_state(seed, n, p), size)
    u = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return 2.0 * u - 1.0
