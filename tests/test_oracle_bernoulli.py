"""Pins for Bernoulli sampling by independent subranges with geometric skips
(Sec. 4.7; Sec. 2, Algorithm B): the count is Binomial(N, p), gaps are
Geometric(p), every position (chunk starts included) is taken with
probability p, windows are slices of the whole, and the degenerate p."""
import math

import numpy as np
import pytest
from scipy import stats


def test_chunk_size_rule(oracle):
    """Smallest c with 2^c p >= n0 (capped at 62)."""
    assert oracle.bern_chunk_log2(1e-4, 4096) == 26
    assert oracle.bern_chunk_log2(1e-2, 4096) == 19
    assert oracle.bern_chunk_log2(0.5, 4096) == 13
    assert oracle.bern_chunk_log2(1.0, 4096) == 12
    assert oracle.bern_chunk_log2(1.0, 1) == 0
    assert oracle.bern_chunk_log2(1e-30, 4096) == 62
    assert oracle.bern_chunk_log2(0.0, 4096) == 62


@pytest.mark.parametrize("p", [0.003, 0.2])
def test_count_is_binomial(oracle, p):
    N, n0, runs = 2**16, 64, 400
    counts = np.array([len(oracle.bernoulli(p, N, seed, n0)) for seed in range(1, runs + 1)], dtype=float)
    mean, var = N * p, N * p * (1 - p)
    assert abs((counts.mean() - mean) / math.sqrt(var / runs)) < 5
    assert abs(counts.var(ddof=1) / var - 1) < 5 * math.sqrt(2 / (runs - 1))


@pytest.mark.parametrize("p", [0.1, 0.5, 0.9])
def test_gaps_are_geometric(oracle, p):
    """Within a chunk, gap - 1 between successive positions is Geometric(p)."""
    N, n0 = 2**22, 2**20
    pos = oracle.bernoulli(p, N, 3, n0).astype(np.int64)
    C = 1 << oracle.bern_chunk_log2(p, n0)
    same_chunk = (pos[1:] - 1) // C == (pos[:-1] - 1) // C
    gaps = (np.diff(pos) - 1)[same_chunk]
    kmax = int(np.log(1e-4) / np.log(1 - p)) + 1 if p < 0.9 else 3
    obs = np.array([np.sum(gaps == k) for k in range(kmax)] + [np.sum(gaps >= kmax)], dtype=float)
    probs = np.array([(1 - p) ** k * p for k in range(kmax)] + [(1 - p) ** kmax])
    assert stats.chisquare(obs, probs * obs.sum()).pvalue > 1e-4


def test_every_position_has_probability_p(oracle):
    """Including the first and last position of each chunk."""
    p, N, n0, runs = 0.25, 64, 4, 6000
    assert oracle.bern_chunk_log2(p, n0) == 4   # chunks of 16
    hits = np.zeros(N)
    for seed in range(1, runs + 1):
        hits[oracle.bernoulli(p, N, seed, n0).astype(np.int64) - 1] += 1
    # each position's hit count is Binomial(runs, p), independently
    chi2 = np.sum((hits - runs * p) ** 2 / (runs * p * (1 - p)))
    assert stats.chi2.sf(chi2, N) > 1e-4


def test_windows_are_slices(oracle):
    p, N, n0, seed = 0.01, 10**7 + 123, 1024, 7
    C = 1 << oracle.bern_chunk_log2(p, n0)
    full = oracle.bernoulli(p, N, seed, n0)
    for a, b in [(0, C), (C, 5 * C), (3 * C, N), (0, N), ((N // C) * C, N), (2 * C, 2 * C)]:
        got = oracle.bernoulli(p, N, seed, n0, a, b)
        want = full[(full >= a + 1) & (full < b + 1)]
        assert np.array_equal(got, want), (a, b)


def test_degenerate_p_and_errors(oracle):
    assert len(oracle.bernoulli(0.0, 1000, 1, 16)) == 0
    assert np.array_equal(oracle.bernoulli(1.0, 1000, 1, 16), np.arange(1, 1001, dtype=np.uint64))
    assert oracle.bernoulli_rc(-0.1, 100, 1, 16, 0, 100, 10)[0] == oracle.EINVAL
    assert oracle.bernoulli_rc(1.5, 100, 1, 16, 0, 100, 10)[0] == oracle.EINVAL
    assert oracle.bernoulli_rc(0.5, 100, 1, 16, 3, 100, 100)[0] == oracle.EINVAL   # unaligned window
    rc, cnt = oracle.bernoulli_rc(0.5, 1000, 1, 16, 0, 1000, 10)
    assert rc == oracle.ECAPACITY and cnt == len(oracle.bernoulli(0.5, 1000, 1, 16))


def test_huge_universe_tiny_p(oracle):
    """N = 2^62, p = 1e-15: one or a few chunks of 2^62 (cap), about 4612
    positions, strictly increasing within [1, N]."""
    p, N = 1e-15, 2**62
    s = oracle.bernoulli(p, N, 5, 4096).astype(object)
    assert abs(len(s) - N * p) < 6 * math.sqrt(N * p)
    assert all(b > a for a, b in zip(s, s[1:])) and s[0] >= 1 and s[-1] <= N


# ---- Bernoulli sampling by its size (Sec. 4.7, relation to Bernoulli sampling) ----

@pytest.mark.parametrize("p,N", [(0.3, 20), (0.05, 40), (0.8, 15)])
def test_size_is_binomial_exactly(oracle, p, N):
    """The size of the sample is BIN(N, p): chi-square against the exact pmf
    over 6000 seeds (p > 1/2 through the complement)."""
    runs = 6000
    sizes = np.array([oracle.bernoulli_size(p, N, s) for s in range(1, runs + 1)])
    pmf = stats.binom.pmf(np.arange(N + 1), N, p)
    keep = pmf * runs >= 5
    obs = np.bincount(sizes, minlength=N + 1)
    o = np.append(obs[keep], obs[~keep].sum())
    e = np.append(pmf[keep] * runs, pmf[~keep].sum() * runs)
    if e[-1] < 1e-9:
        o, e = o[:-1], e[:-1]
    chi2 = ((o - e) ** 2 / e).sum()
    assert stats.chi2.sf(chi2, len(o) - 1) > 1e-4, (p, N, chi2)


def test_size_moments_at_large_n(oracle):
    """Mean and variance of BIN(2^40, 1e-3) over 400 seeds (ratio-of-uniforms
    branch), and the degenerate p."""
    N, p, runs = 2**40, 1e-3, 400
    x = np.array([oracle.bernoulli_size(p, N, s) for s in range(1, runs + 1)], dtype=float)
    mu, var = N * p, N * p * (1 - p)
    assert abs(x.mean() - mu) < 5 * math.sqrt(var / runs)
    assert 0.7 < x.var(ddof=1) / var < 1.4
    assert oracle.bernoulli_size(0.0, 1000, 3) == 0 and oracle.bernoulli_size(1.0, 1000, 3) == 1000


def test_by_size_positions(oracle):
    """Each position is taken with probability p (chi-square over 2000
    seeds), positions increase strictly inside 1..N, the window is a slice
    of the whole, and the full window holds the whole size."""
    p, N, runs = 0.3, 40, 2000
    hits = np.zeros(N)
    for s in range(1, runs + 1):
        pos, tot = oracle.bernoulli_by_size(p, N, s, 4)
        assert len(pos) == tot and np.all(np.diff(pos.astype(np.int64)) > 0) and (len(pos) == 0 or pos[0] >= 1)
        hits[pos.astype(np.int64) - 1] += 1
    e = runs * p
    chi2 = (((hits - e) ** 2) / (e * (1 - p))).sum()
    assert stats.chi2.sf(chi2, N) > 1e-4
    full, tot = oracle.bernoulli_by_size(0.01, 10**7 + 3, 9, 1024)
    assert len(full) == tot and abs(tot - 1e5) < 6 * math.sqrt(1e5)
    for a, b in [(0, 12345), (777, 10**6 + 1), (5 * 10**6, 10**7 + 3), (10, 10)]:
        got, tot2 = oracle.bernoulli_by_size(0.01, 10**7 + 3, 9, 1024, a, b)
        assert tot2 == tot
        assert np.array_equal(got, full[(full >= a + 1) & (full < b + 1)]), (a, b)
