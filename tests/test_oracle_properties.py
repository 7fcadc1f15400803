"""Invariants of the oracle over randomly drawn small arguments (hypothesis):
every sampler's output has the shape its definition fixes — sorted,
distinct where it must be, inside its range, of the right length — and the
pieces agree with each other (a union's counts with its sample, a peel's
batches with the whole, a box's points with its extents)."""
import numpy as np
import pytest

try:
    from hypothesis import given, settings, strategies as st
except ImportError:   # a machine without hypothesis (the GPU machine) collects one placeholder instead
    given = None

if given is None:
    def test_properties_need_hypothesis():
        pytest.skip("hypothesis is not installed")

else:
    SETTINGS = dict(max_examples=60, deadline=None)


    @settings(**SETTINGS)
    @given(N=st.integers(1, 10**12), frac=st.floats(0, 1), seed=st.integers(0, 2**64 - 1),
           n0=st.sampled_from([1, 3, 64, 4096]), kind=st.sampled_from([0, 1, 2]))
    def test_sample_shape(oracle, N, frac, seed, n0, kind):
        n = min(int(frac * min(N, 3000)), N)
        v = oracle.sample(n, N, seed, n0, kind).astype(object)
        assert len(v) == n
        if n:
            assert v[0] >= 1 and v[-1] <= N
            d = np.diff(np.array(v, dtype=object)) if n > 1 else []
            assert all(x > 0 for x in d) if kind != 1 else all(x >= 0 for x in d)


    @settings(**SETTINGS)
    @given(sizes=st.lists(st.integers(0, 10**9), min_size=1, max_size=40), frac=st.floats(0, 1),
           seed=st.integers(0, 2**64 - 1))
    def test_union_counts_and_sample_agree(oracle, sizes, frac, seed):
        L = np.array(sizes, dtype=np.uint64)
        n = int(frac * min(int(L.sum()), 2000))
        pos, counts = oracle.union_sample(L, n, seed, 16)
        assert np.array_equal(counts, oracle.union_counts(L, n, seed))
        assert int(counts.sum()) == n and np.all(counts <= L)
        off = 0
        for l, c in zip(L.tolist(), counts.tolist()):
            seg = pos[off:off + c].astype(np.int64)
            assert np.all(seg >= 1) and np.all(seg <= l) and np.all(np.diff(seg) > 0)
            off += c


    @settings(**SETTINGS)
    @given(N=st.integers(1, 10**15), frac=st.floats(0, 1), seed=st.integers(0, 2**64 - 1),
           n0=st.integers(1, 600))
    def test_peel_batches_make_the_sample(oracle, N, frac, seed, n0):
        n = min(int(frac * min(N, 5000)), N)
        v, c = oracle.peel_sample(n, N, seed, n0)
        assert len(v) == n and int(c.sum()) == n
        if n:
            w = v.astype(object)
            assert w[0] >= 1 and w[-1] <= N and all(x > 0 for x in np.diff(np.array(w, dtype=object)))
            assert c[-1] > 0 or len(c) == 1


    @settings(**SETTINGS)
    @given(E=st.lists(st.integers(1, 2**15), min_size=1, max_size=4), n=st.integers(0, 3000),
           seed=st.integers(0, 2**64 - 1), n0=st.sampled_from([1, 7, 256, 4096]))
    def test_points_inside_the_box(oracle, E, n, seed, n0):
        P = oracle.points(n, E, seed, n0).astype(np.int64)
        assert P.shape == (n, len(E))
        assert np.all(P >= 0) and np.all(P < np.array(E, dtype=np.int64))
