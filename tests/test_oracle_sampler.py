"""Pins for the whole sampler in the oracle.

- uniformity over all n-subsets of 1..N (the problem statement, Sec. 1-2) by
  brute-force enumeration on tiny inputs, for both base cases (Algorithm H
  and Algorithm B) and several tree depths;
- the multiset law of sampling with replacement (Sec. 4.6);
- inclusion probability n/N of every element;
- structural invariants of the split tree (Sec. 3.1: counts add up, ranges
  halve at floor(S/2), offsets are prefix sums) and of every output (sorted,
  distinct, in range, n values);
- the leaf semantics (first k distinct valid candidates; complement when
  more than half the leaf is taken), recomputed from the candidates;
- range queries are slices of the full sample (Sec. 4.1).
"""
import itertools
import math
from collections import Counter

import numpy as np
import pytest
from scipy import stats

H, WR, B = 0, 1, 2


def _subset_chisq(oracle, n, N, n0, kind, runs, seed0=1):
    subsets = list(itertools.combinations(range(1, N + 1), n))
    index = {s: i for i, s in enumerate(subsets)}
    counts = np.zeros(len(subsets))
    for seed in range(seed0, seed0 + runs):
        s = oracle.sample(n, N, seed, n0, kind)
        counts[index[tuple(int(x) for x in s)]] += 1
    if len(subsets) == 1:
        return 1.0
    return stats.chisquare(counts).pvalue


@pytest.mark.parametrize("n,N,n0", [(5, 10, 1), (3, 10, 2), (4, 12, 1), (6, 7, 1), (2, 9, 4), (7, 8, 2),
                                    (1, 5, 1), (5, 5, 1), (3, 6, 1)])
def test_uniform_over_subsets_leaf_h(oracle, n, N, n0):
    runs = max(6000, 40 * math.comb(N, n))
    assert _subset_chisq(oracle, n, N, n0, H, runs) > 1e-4


@pytest.mark.parametrize("n,N,n0", [(5, 10, 1), (3, 10, 2), (6, 7, 1), (2, 9, 4), (4, 11, 2)])
def test_uniform_over_subsets_leaf_b(oracle, n, N, n0):
    runs = max(6000, 40 * math.comb(N, n))
    assert _subset_chisq(oracle, n, N, n0, B, runs, seed0=100000) > 1e-4


@pytest.mark.parametrize("n,N,n0", [(3, 5, 1), (4, 4, 2), (2, 7, 1), (5, 3, 2)])
def test_with_replacement_multiset_law(oracle, n, N, n0):
    """P(multiset) = n! / prod(m_i!) / N^n."""
    cells = list(itertools.combinations_with_replacement(range(1, N + 1), n))
    index = {c: i for i, c in enumerate(cells)}
    exp = np.array([math.factorial(n) / math.prod(math.factorial(m) for m in Counter(c).values()) / N**n
                    for c in cells])
    runs = 20000
    counts = np.zeros(len(cells))
    for seed in range(1, runs + 1):
        s = oracle.sample(n, N, seed, n0, WR)
        assert np.all(np.diff(s.astype(np.int64)) >= 0)
        counts[index[tuple(int(x) for x in s)]] += 1
    assert stats.chisquare(counts, exp * runs).pvalue > 1e-4


@pytest.mark.parametrize("kind", [H, B])
def test_inclusion_probability(oracle, kind):
    """Every element is in the sample with probability n/N."""
    n, N, n0, runs = 60, 600, 8, 3000
    hits = np.zeros(N)
    for seed in range(1, runs + 1):
        hits[oracle.sample(n, N, seed, n0, kind).astype(np.int64) - 1] += 1
    exp = np.full(N, runs * n / N)
    assert stats.chisquare(hits, exp).pvalue > 1e-4


def test_depth_rule(oracle):
    """D is the least depth with n <= n0 2^D, then lowered until 2^D <= N."""
    assert oracle.depth(10**6, 10**9, 4096) == 8
    assert oracle.depth(10**9, 2**50, 4096) == 18
    assert oracle.depth(10**9, 2**40, 4096) == 18
    assert oracle.depth(4096, 10**9, 4096) == 0
    assert oracle.depth(4097, 10**9, 4096) == 1
    assert oracle.depth(0, 10, 4) == 0
    assert oracle.depth(10, 4, 1) == 2
    assert oracle.depth(2**62, 2**62, 1) == 62
    for n, N, n0 in [(10**6, 10**9, 4096), (999, 1000, 3), (12345, 10**7, 100)]:
        D = oracle.depth(n, N, n0)
        assert n <= n0 * 2**D and (D == 0 or n > n0 * 2 ** (D - 1) or 2 ** (D + 1) > N)


@pytest.mark.parametrize("n,N,n0,kind", [(10**6, 10**9, 4096, H), (10**5, 2**50, 512, H), (999, 1000, 3, H),
                                         (10**6, 2**40, 4096, WR), (5000, 77, 16, WR), (1, 2**62, 1, H)])
def test_tree_invariants(oracle, n, N, n0, kind):
    recs, D = oracle.tree(n, N, 11, n0, kind)
    lo, s, c, off = (recs[:, i].astype(object) for i in range(4))
    assert len(recs) == 2**D
    assert sum(c) == n
    assert lo[0] == 0 and all(lo[i] + s[i] == lo[i + 1] for i in range(len(recs) - 1))
    assert lo[-1] + s[-1] == N
    assert set(s) <= {N >> D, -(-N >> D)}
    assert off[0] == 0 and all(off[i] + c[i] == off[i + 1] for i in range(len(recs) - 1))
    if kind == H:
        assert all(c[i] <= s[i] for i in range(len(recs)))


@pytest.mark.parametrize("n,N,n0,kind,seed", [(10**6, 10**9, 4096, H, 1), (20000, 30000, 512, H, 2),
                                              (3000, 3001, 64, H, 3), (50000, 2**62, 1024, H, 4),
                                              (10**5, 2**40, 4096, WR, 5), (40000, 1000, 256, WR, 6),
                                              (20000, 10**7, 1024, B, 7), (5000, 6000, 128, B, 8)])
def test_output_invariants(oracle, n, N, n0, kind, seed):
    s = oracle.sample(n, N, seed, n0, kind).astype(object)
    assert len(s) == n
    assert min(s) >= 1 and max(s) <= N
    d = np.diff(np.array(s, dtype=object))
    if kind == WR:
        assert all(x >= 0 for x in d)
    else:
        assert all(x > 0 for x in d)


def _first_distinct(oracle, seed, tag, node, s, k):
    sel, seen, j = [], set(), 0
    while len(sel) < k:
        ok, v = oracle.candidate(seed, tag, node, s, j)
        j += 1
        if ok and v not in seen:
            seen.add(v)
            sel.append(v)
    return sel


@pytest.mark.parametrize("s,np_", [(2**32, 3800), (3906250, 3906), (1000, 400), (1000, 600), (1000, 1000),
                                   (7, 3), (3 * 2**30 + 1, 500), (2**45 + 3, 700), (10, 0), (64, 33)])
def test_leaf_h_semantics(oracle, s, np_):
    """Leaf H = sorted first k distinct valid candidates of stream (LEAF_H,
    id); if 2n' > s, k = s - n' and the output is the rest of [0, s)."""
    seed, node, lo = 5, 77, 123
    got = [int(x) for x in oracle.leaf_h(seed, node, lo, s, np_)]
    comp = 2 * np_ > s
    k = s - np_ if comp else np_
    sel = _first_distinct(oracle, seed, 2, node, s, k)
    want = sorted(set(range(s)) - set(sel)) if comp else sorted(sel)
    assert got == [lo + v + 1 for v in want]


def test_leaf_wr_semantics(oracle):
    seed, node, lo, s, np_ = 8, 3, 1000, 1003, 900
    vals, j = [], 0
    while len(vals) < np_:
        ok, v = oracle.candidate(seed, 6, node, s, j)
        j += 1
        if ok:
            vals.append(v)
    assert [int(x) for x in oracle.leaf_wr(seed, node, lo, s, np_)] == [lo + v + 1 for v in sorted(vals)]


@pytest.mark.parametrize("s,np_", [(8, 3), (20, 1), (12, 10)])
def test_leaf_b_uniform(oracle, s, np_):
    """Algorithm B as a base case draws a uniform n'-subset of the leaf."""
    subsets = {c: i for i, c in enumerate(itertools.combinations(range(1, s + 1), np_))}
    counts = np.zeros(len(subsets))
    runs = max(8000, 40 * len(subsets))
    for node in range(1, runs + 1):
        counts[subsets[tuple(int(x) for x in oracle.leaf_b(4, node, 0, s, np_))]] += 1
    assert stats.chisquare(counts).pvalue > 1e-4


def test_leaf_b_removal_semantics(oracle):
    """Leaf B keeps the Bernoulli positions whose indices are not among the
    first c - n' distinct FIXUP candidates over [0, c)."""
    seed, node, s, np_ = 6, 41, 100000, 700
    rho = min(1.0, (np_ + 3 * math.sqrt(np_) + 10) / s)
    L = oracle.log1p(-rho)
    for attempt in range(64):
        pos, p, j = [], -1, 0
        while True:
            q = oracle.log(oracle.u_open(oracle.value(seed, 3 + 256 * attempt, node, j))) / L
            j += 1
            if q >= 2.0**62:
                break
            p = p + math.floor(q) + 1
            if p >= s:
                break
            pos.append(p)
        if len(pos) >= np_:
            break
    drop = set(_first_distinct(oracle, seed, 4, node, len(pos), len(pos) - np_))
    want = [x + 1 for i, x in enumerate(pos) if i not in drop]
    assert [int(x) for x in oracle.leaf_b(seed, node, 0, s, np_)] == want


@pytest.mark.parametrize("kind", [H, WR, B])
def test_range_query_is_slice(oracle, kind):
    n, N, n0, seed = 30000, 10**7, 512, 9
    full = oracle.sample(n, N, seed, n0, kind)
    for a, b in [(1, N + 1), (5, 6), (123456, 7654321), (N // 2, N // 2 + 10**5), (N, N + 1), (7, 7)]:
        want = full[(full >= a) & (full < b)]
        got = oracle.range_query(n, N, seed, n0, kind, a, b)
        assert np.array_equal(got, want), (a, b)


def test_argument_checks(oracle):
    assert oracle.sample_rc(11, 10, 1, 4, H) == oracle.EINVAL
    assert oracle.sample_rc(11, 10, 1, 4, B) == oracle.EINVAL
    assert oracle.sample_rc(11, 10, 1, 4, WR) == oracle.OK
    assert oracle.sample_rc(1, 10, 1, 0, H) == oracle.EINVAL
    assert oracle.sample_rc(1, 0, 1, 4, H) == oracle.EINVAL
    assert oracle.sample_rc(1, 2**62 + 1, 1, 4, H) == oracle.EINVAL
    assert oracle.sample_rc(0, 0, 1, 4, H) == oracle.OK
    assert oracle.sample_rc(0, 10, 1, 4, H) == oracle.OK


def test_determinism_and_seed_sensitivity(oracle):
    a = oracle.sample(10**5, 10**8, 42, 1024)
    b = oracle.sample(10**5, 10**8, 42, 1024)
    c = oracle.sample(10**5, 10**8, 43, 1024)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


@pytest.mark.parametrize("N,D", [(1001, 3), (2**40 + 12345, 5), (97, 6), (10**9, 8)])
def test_split_point_is_floor_half(oracle, N, D):
    """Algorithm R splits 1..N at l = floor(N/2): the left part has floor(S/2)
    elements at every level, so the leaf ranges are those of repeated
    floor-halving (written out here by walking each leaf's path)."""
    n0 = 1
    n = min(N, 2**D)
    assert oracle.depth(n, N, n0) == D
    recs, _ = oracle.tree(n, N, 3, n0)
    for i in range(2**D):
        lo, S = 0, N
        for level in range(D - 1, -1, -1):
            left = S // 2
            if (i >> level) & 1:
                lo, S = lo + left, S - left
            else:
                S = left
        assert (int(recs[i, 0]), int(recs[i, 1])) == (lo, S), i
