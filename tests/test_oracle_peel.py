"""Pins for online sorted sampling by peeling (Sec. 4.1): the sample is a
uniform n-subset (brute force over every subset of tiny universes, with
many peels), the first batch's count has the exact hypergeometric law,
batches hold about n0 samples each and lie in consecutive ranges, and the
degenerate cases (n = 0, n = N, n0 >= n: one batch)."""
import itertools
import math

import numpy as np
import pytest
from scipy import stats


@pytest.mark.parametrize("N,n,n0", [(9, 3, 1), (8, 4, 2), (10, 2, 1)])
def test_peel_sample_is_uniform_subset(oracle, N, n, n0):
    subsets = {s: i for i, s in enumerate(itertools.combinations(range(1, N + 1), n))}
    runs = 150 * len(subsets)
    obs = np.zeros(len(subsets))
    nb = []
    for seed in range(1, runs + 1):
        v, c = oracle.peel_sample(n, N, seed, n0)
        obs[subsets[tuple(int(x) for x in v)]] += 1
        nb.append(len(c))
    assert stats.chisquare(obs).pvalue > 1e-4
    assert max(nb) >= 3   # several peels, not one leaf


@pytest.mark.parametrize("N,n,n0", [(50, 10, 3), (20, 6, 1), (1000, 7, 3)])
def test_first_batch_count_is_hypergeometric(oracle, N, n, n0):
    """m = ceil(N n0 / n) positions peeled first: 15 (exact), 4 (rounded up
    from 3.3) and 429 (from 428.6), so a floor in place of the ceiling
    changes the law."""
    runs = 20000
    m = -(-N * n0 // n)
    obs = np.zeros(n + 1)
    for seed in range(1, runs + 1):
        _, c = oracle.peel_sample(n, N, seed, n0)
        obs[int(c[0])] += 1
    pmf = np.array([math.comb(m, k) * math.comb(N - m, n - k) / math.comb(N, n) for k in range(n + 1)])
    keep = pmf * runs >= 5
    o = np.append(obs[keep], obs[~keep].sum())
    e = np.append(pmf[keep] * runs, pmf[~keep].sum() * runs)
    if e[-1] == 0:
        assert o[-1] == 0
        o, e = o[:-1], e[:-1]
    assert stats.chisquare(o, e).pvalue > 1e-4


def test_batches_lie_in_consecutive_ranges(oracle):
    """Batch t's values lie in (lo_t, lo_t + m_t], the peeled range, and the
    whole sample increases strictly inside 1..N."""
    n, N, n0 = 20000, 10**12, 500
    v, c = oracle.peel_sample(n, N, 17, n0)
    assert len(v) == n and int(c.sum()) == n
    assert np.all(np.diff(v.astype(np.int64)) > 0) and v[0] >= 1 and v[-1] <= N
    nr, Nr, lo, off = n, N, 0, 0
    for t, ct in enumerate(c.tolist()):
        m = min(-(-Nr * n0 // nr), Nr)
        seg = v[off:off + ct]
        if ct:
            assert int(seg[0]) > lo and int(seg[-1]) <= lo + m, t
        if m == Nr:
            assert ct == nr and t == len(c) - 1
        lo, Nr, nr, off = lo + m, Nr - m, nr - ct, off + ct
    assert nr == 0


def test_batch_sizes_near_n0(oracle):
    """E[c_t | state] = n_t m_t / N_t, which is n0 up to the rounding of m_t."""
    n, N, n0 = 200000, 2**40, 1000
    _, c = oracle.peel_sample(n, N, 5, n0)
    body = c[:-1].astype(float)
    assert abs(len(c) - n / n0) < 10
    assert abs(body.mean() - n0) < 5 * math.sqrt(n0 / len(body))
    assert 0.5 < body.var() / n0 < 1.5


def test_degenerate_cases(oracle):
    v, c = oracle.peel_sample(0, 100, 1, 4)
    assert len(v) == 0 and len(c) == 0
    v, c = oracle.peel_sample(37, 37, 2, 8)
    assert np.array_equal(v, np.arange(1, 38)) and int(c.sum()) == 37
    # n0 >= n: one batch, the leaf of node 1 over the whole range
    v, c = oracle.peel_sample(300, 10**9, 3, 4096)
    assert np.array_equal(c, [300])
    assert np.array_equal(v, oracle.leaf_h(3, 1, 0, 10**9, 300))
    with pytest.raises(Exception):
        oracle.peel_sample(5, 4, 1, 2)
    with pytest.raises(Exception):
        oracle.peel_sample(5, 2**62 + 1, 1, 2)
