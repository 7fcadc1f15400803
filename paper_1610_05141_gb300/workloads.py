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


def serve_trees(T: int = 8, seed: int = 5, n: int = 10**8, log2_N_max: int = 56):
    """Resident trees for the serving mix: T samples of n values each, N
    log-uniform in [n, 2^log2_N_max].  Returns a list of (n, N, seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for t in range(T):
        lnN = np.log(n) + rng.random() * (log2_N_max * np.log(2.0) - np.log(n))
        out.append((n, int(min(max(np.floor(np.exp(lnN)), n), 2**log2_N_max)), 9000 + t))
    return out


def serve_jobs(count: int, trees, seed: int = 5, query_frac: float = 0.2, log10_n_min: float = 2.0,
               log10_n_max: float = 8.0, log2_N_max: int = 56, hits_min: float = 1e3, hits_max: float = 1e5):
    """A serving mix: sampling jobs with n log-uniform in [10^2, 10^8) and N
    log-uniform in [n, 2^56] (sample seed 5,000,000 + i), and range queries
    (a fraction query_frac) on the trees with expected hits log-uniform in
    [10^3, 10^5].  Returns a dict of numpy arrays: op (0 sample, 1 query), n,
    N, seed, tree, a, b, cap."""
    rng = np.random.Generator(np.random.PCG64(seed))
    op = (rng.random(count) < query_frac).astype(np.uint32)
    u, u2, u3, u4 = rng.random(count), rng.random(count), rng.random(count), rng.random(count)
    ln_n = np.log(10.0) * (log10_n_min + u * (log10_n_max - log10_n_min))
    n = np.floor(np.exp(ln_n)).astype(np.uint64)
    N = np.floor(np.exp(ln_n + u2 * (log2_N_max * np.log(2.0) - ln_n)))
    N = np.maximum(np.minimum(N, float(2**log2_N_max)), n.astype(np.float64)).astype(np.uint64)
    N = np.maximum(N, n)
    tree = rng.integers(0, len(trees), count).astype(np.uint32)
    hits = np.exp(np.log(hits_min) + u3 * (np.log(hits_max) - np.log(hits_min)))
    tn = np.array([t[0] for t in trees], dtype=np.float64)[tree]
    tN = np.array([t[1] for t in trees], dtype=np.float64)[tree]
    width = np.maximum(1.0, np.floor(hits * tN / tn))
    a = 1 + np.floor(u4 * np.maximum(tN - width, 1.0))
    b = a + width
    cap = np.ceil(hits + 10.0 * np.sqrt(hits) + 100.0).astype(np.uint64)
    seeds = np.arange(5_000_000, 5_000_000 + count, dtype=np.uint64)
    return {"op": op, "n": n, "N": N, "seed": seeds, "tree": tree, "a": a.astype(np.uint64),
            "b": b.astype(np.uint64), "cap": cap}


def union_segments(p: int = 4096, seed: int = 4, log2_min: float = 20.0, log2_max: float = 40.0):
    """Segment sizes of a union: p sizes log-uniform in [2^log2_min, 2^log2_max]
    (uneven shares, as the uneven distribution of the universe over owners)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    e = log2_min + (log2_max - log2_min) * rng.random(p)
    return np.floor(np.exp2(e)).astype(np.uint64)
