"""Seeded synthetic inputs (no sampling arithmetic here).

The paper's workloads are synthetic ranges (Sec. 6: universe 2^50, varying
sample sizes); no dataset is involved.  This module only draws request
parameters; the samples themselves come from the library.
"""
from __future__ import annotations

import numpy as np


def batch_requests(R: int = 100_000, seed: int = 20161017, log10_n_max: float = 6.0, log2_N_max: int = 48,
                   n0: int = 4096):
    """R independent requests: n log-uniform in [1, 10^log10_n_max), N log-uniform in [n, 2^log2_N_max],
    request seed i + 1, outputs packed back to back.  Returns numpy arrays
    (n, N, seed, out_off, n0) and the total number of output values."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.random(R)
    u2 = rng.random(R)
    n = np.maximum(1, np.floor(10.0 ** (log10_n_max * u))).astype(np.uint64)
    ln_n = np.log(n.astype(np.float64))
    N = np.floor(np.exp(ln_n + u2 * (log2_N_max * np.log(2.0) - ln_n)))
    N = np.minimum(np.maximum(N, n.astype(np.float64)), float(2**log2_N_max)).astype(np.uint64)
    N = np.maximum(N, n)
    seeds = np.arange(1, R + 1, dtype=np.uint64)
    out_off = np.zeros(R, dtype=np.uint64)
    out_off[1:] = np.cumsum(n)[:-1]
    n0s = np.full(R, n0, dtype=np.uint32)
    return n, N, seeds, out_off, n0s, int(n.sum())
