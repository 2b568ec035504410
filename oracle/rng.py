"""SplitMix64 counter-based generator (Steele, Lea & Flood, OOPSLA 2014).

Test infrastructure (see oracle/__init__.py). The eigenvalue estimate of the multigrid
smoother (Sec. 7: 30 CG iterations) needs a start vector; both the oracle and the CUDA
library draw it from this published generator so that they start from identical vectors.
Entry i of the vector for a given seed: z = seed + (i + 1) * 0x9E3779B97F4A7C15 (mod 2^64),
then the SplitMix64 finaliser, then the top 53 bits mapped to [-1, 1).
"""
from __future__ import annotations

import numpy as np


def splitmix64_uniform(seed: int, n: int) -> np.ndarray:
    i = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + i * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return 2.0 * u - 1.0
