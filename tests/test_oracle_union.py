"""Pins for sampling from a union of uneven segments (Sec. 4.3): the counts
per segment follow the multivariate hypergeometric law (exact pmf), the
union's sample is a uniform n-subset of all the segments' elements (brute
force over every subset of a tiny universe), and the degenerate cases
(empty segments, n = 0, n = N, one segment, padding to a power of two)."""
import itertools
import math

import numpy as np
import pytest
from scipy import stats

W = 0x9E3779B97F4A7C15


def _mvhg_pmf(L, c):
    return math.prod(math.comb(l, x) for l, x in zip(L, c)) / math.comb(sum(L), sum(c))


def _count_vectors(L, n):
    for c in itertools.product(*(range(l + 1) for l in L)):
        if sum(c) == n:
            yield c


@pytest.mark.parametrize("L,n", [([2, 3, 1, 4], 4), ([5, 0, 2, 1, 3], 5), ([1, 6, 2], 3)])
def test_counts_are_multivariate_hypergeometric(oracle, L, n):
    """Uneven sizes make a swapped child, a dropped padding node or a wrong
    node sum change the law; p = 5 and 3 pad the tree to 8 and 4 leaves."""
    runs = 12000
    vecs = list(_count_vectors(L, n))
    index = {c: i for i, c in enumerate(vecs)}
    obs = np.zeros(len(vecs))
    for seed in range(1, runs + 1):
        c = tuple(int(x) for x in oracle.union_counts(np.array(L), n, seed))
        obs[index[c]] += 1
    probs = np.array([_mvhg_pmf(L, c) for c in vecs])
    assert abs(probs.sum() - 1) < 1e-12
    keep = probs * runs >= 5
    exp = probs * runs
    o = np.append(obs[keep], obs[~keep].sum())
    e = np.append(exp[keep], exp[~keep].sum())
    if e[-1] == 0:
        o, e = o[:-1], e[:-1]
    assert stats.chisquare(o, e).pvalue > 1e-4


def test_union_sample_is_uniform_subset(oracle):
    """Every 3-subset of the 10 elements of segments of sizes 4, 1, 0, 5 is
    equally likely (120 subsets)."""
    L, n, runs = [4, 1, 0, 5], 3, 24000
    starts = np.concatenate([[0], np.cumsum(L)[:-1]])
    subsets = {s: i for i, s in enumerate(itertools.combinations(range(sum(L)), n))}
    obs = np.zeros(len(subsets))
    for seed in range(1, runs + 1):
        pos, counts = oracle.union_sample(np.array(L), n, seed, 2)
        seg = np.repeat(np.arange(len(L)), counts.astype(np.int64))
        glob = tuple(int(starts[s] + p - 1) for s, p in zip(seg, pos))
        obs[subsets[glob]] += 1
    assert stats.chisquare(obs).pvalue > 1e-4


def test_positions_within_segments(oracle):
    L = np.array([10**6, 3, 0, 2**40, 17, 5 * 10**5, 1], dtype=np.uint64)
    n = 5000
    pos, counts = oracle.union_sample(L, n, 11, 64)
    assert int(counts.sum()) == n and np.all(counts <= L)
    assert counts[2] == 0
    off = 0
    for l, c in zip(L.tolist(), counts.tolist()):
        seg = pos[off:off + c].astype(np.int64) if l < 2**62 else pos[off:off + c]
        if c:
            assert int(seg[0]) >= 1 and int(seg[-1]) <= l and np.all(np.diff(seg.astype(object)) > 0)
        off += c
    # the 2^40 segment holds nearly all the mass
    assert counts[3] > n - 10


def test_segment_sample_is_the_segment_key_sample(oracle):
    """Segment i samples with key seed + (i+1) * 0x9E3779B97F4A7C15 mod 2^64
    and the same n0 (an interface fact of the union sample)."""
    L = np.array([1000, 77, 5000, 1], dtype=np.uint64)
    seed = 2**64 - 3
    pos, counts = oracle.union_sample(L, 400, seed, 16)
    off = 0
    for i, (l, c) in enumerate(zip(L.tolist(), counts.tolist())):
        assert oracle.union_key(seed, i) == (seed + (i + 1) * W) % 2**64
        assert np.array_equal(pos[off:off + c], oracle.sample(c, l, (seed + (i + 1) * W) % 2**64, 16))
        off += c


def test_degenerate_cases(oracle):
    L = np.array([3, 0, 5, 2], dtype=np.uint64)
    assert np.array_equal(oracle.union_counts(L, 0, 1), [0, 0, 0, 0])
    assert np.array_equal(oracle.union_counts(L, 10, 1), L)
    pos, counts = oracle.union_sample(L, 10, 1, 4)
    assert np.array_equal(pos, [1, 2, 3, 1, 2, 3, 4, 5, 1, 2])
    assert np.array_equal(oracle.union_counts(np.array([7], dtype=np.uint64), 4, 9), [4])
    # one segment: the union sample is that segment's sample
    pos, _ = oracle.union_sample(np.array([10**9], dtype=np.uint64), 300, 5, 64)
    assert np.array_equal(pos, oracle.sample(300, 10**9, (5 + W) % 2**64, 64))
    with pytest.raises(Exception):
        oracle.union_counts(L, 11, 1)
    with pytest.raises(Exception):
        oracle.union_counts(np.array([2**61, 2**61, 1], dtype=np.uint64), 1, 1)


def test_left_share_mean(oracle):
    """Large counts: the first of two halves of sizes 3e9 and 1e10 gets
    n 3/13 on average, with the hypergeometric variance."""
    L = np.array([10**9, 2 * 10**9, 10**10], dtype=np.uint64)
    n, runs = 10**6, 400
    first_two = np.array([int(oracle.union_counts(L, n, s)[:2].sum()) for s in range(1, runs + 1)], dtype=float)
    N = int(L.sum())
    q = 3 / 13
    var = n * q * (1 - q) * (N - n) / (N - 1)
    assert abs((first_two.mean() - n * q) / math.sqrt(var / runs)) < 5
    assert abs(first_two.var(ddof=1) / var - 1) < 5 * math.sqrt(2 / (runs - 1))
