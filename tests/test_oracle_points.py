"""Pins for sampling with replacement from a d-dimensional box by bisection
(Sec. 4.6, random points in a rectangle): one dimension (and boxes whose
other extents are 1) reduces to the one-dimensional sampler with
replacement; the multiset of points has the exact multinomial law (brute
force over every multiset, odd extents and unit extents); coordinates are
uniform at scale; the first split halves the largest extent (lowest index
on ties) and a single leaf lists its points in row-major order; argument
checks."""
import itertools
import math
from collections import Counter

import numpy as np
import pytest
from scipy import stats


@pytest.mark.parametrize("n,N,seed,n0", [(1000, 10**6, 4, 64), (5000, 2**40, 7, 100), (37, 37, 1, 8),
                                        (300, 5, 2, 16)])
def test_one_dimension_is_sampling_with_replacement(oracle, n, N, seed, n0):
    want = oracle.sample(n, N, seed, n0, oracle.KIND_WR).astype(np.int64) - 1
    assert np.array_equal(oracle.points(n, [N], seed, n0)[:, 0].astype(np.int64), want)
    # unit extents elsewhere: the same values in the one dimension that is not 1
    for E, k in (([N, 1, 1], 0), ([1, N], 1), ([1, 1, 1, N], 3)):
        P = oracle.points(n, E, seed, n0).astype(np.int64)
        assert np.array_equal(P[:, k], want)
        assert not np.delete(P, k, axis=1).any()


def _multiset_law(V, n):
    """All multisets of n lattice indices in [0, V) with their probability."""
    out = {}
    for ms in itertools.combinations_with_replacement(range(V), n):
        cnt = Counter(ms)
        out[ms] = math.factorial(n) / math.prod(math.factorial(c) for c in cnt.values()) / V**n
    return out


@pytest.mark.parametrize("E,n,n0", [([3, 2], 3, 1), ([2, 2, 3], 2, 1), ([2, 1, 3], 4, 1)])
def test_multiset_law(oracle, E, n, n0):
    V = math.prod(E)
    law = _multiset_law(V, n)
    keys = list(law)
    index = {k: i for i, k in enumerate(keys)}
    runs = 120 * len(keys)
    obs = np.zeros(len(keys))
    strides = [math.prod(E[k + 1:]) for k in range(len(E))]
    for seed in range(1, runs + 1):
        P = oracle.points(n, E, seed, n0).astype(np.int64)
        lin = tuple(sorted(int(np.dot(p, strides)) for p in P))
        obs[index[lin]] += 1
    exp = np.array([law[k] for k in keys]) * runs
    assert abs(exp.sum() - runs) < 1e-6
    assert stats.chisquare(obs, exp).pvalue > 1e-4


def test_coordinates_uniform_at_scale(oracle):
    E, n = [7, 5], 70000
    P = oracle.points(n, E, 11, 16).astype(np.int64)
    assert P.shape == (n, 2) and (P >= 0).all() and (P[:, 0] < 7).all() and (P[:, 1] < 5).all()
    cells = np.bincount(P[:, 0] * 5 + P[:, 1], minlength=35)
    assert stats.chisquare(cells).pvalue > 1e-4
    # a wide box: every coordinate inside its extent, marginals uniform by decile
    E = [2**30, 3, 2**20]
    P = oracle.points(200000, E, 12, 4096).astype(np.float64)
    for k, e in enumerate(E):
        assert (P[:, k] < e).all()
        dec = np.bincount(np.minimum((P[:, k] * 10 / e).astype(int), 9), minlength=10) if e > 3 else \
            np.bincount(P[:, k].astype(int), minlength=e)
        assert stats.chisquare(dec).pvalue > 1e-4


@pytest.mark.parametrize("E,k", [([8, 2], 0), ([2, 8], 1), ([4, 4], 0), ([3, 5, 5], 1)])
def test_first_split_halves_the_largest_extent(oracle, E, k):
    """With two leaves, the left leaf's points (listed first) lie in the
    lower half along the split dimension, the right leaf's in the upper."""
    n = 2000
    P = oracle.points(n, E, 5, n // 2).astype(np.int64)   # depth 1
    low = P[:, k] < E[k] // 2
    c = int(low.sum())
    assert 0 < c < n and low[:c].all() and not low[c:].any()


def test_single_leaf_is_row_major(oracle):
    P = oracle.points(3000, [6, 5, 4], 9, 4096).astype(np.int64)   # depth 0
    lin = P[:, 0] * 20 + P[:, 1] * 4 + P[:, 2]
    assert np.all(np.diff(lin) >= 0)


def test_degenerate_and_invalid(oracle):
    assert oracle.points(0, [3, 4], 1, 8).shape == (0, 2)
    assert not oracle.points(50, [1, 1], 1, 8).any()
    for E in ([3, 0], [2**31, 2**31, 2], [1, 1, 1, 1, 1]):
        with pytest.raises(Exception):
            oracle.points(5, E, 1, 8)
    with pytest.raises(Exception):
        oracle.points(5, [4], 1, 0)
    # the largest volume
    P = oracle.points(100, [2**31, 2**31], 3, 8).astype(np.uint64)
    assert (P < 2**31).all()
