"""GPU parity of sampling from a union of uneven segments (Sec. 4.3): the
counts per segment from the device's tree of hypergeometric splits and the
union's sample equal the oracle's, bit for bit, including empty segments,
a single segment, segment counts that are not powers of two, n = 0 and
n = N, and, at the size the benchmark times, sampled segments."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1610_05141_gb300 as rs
    from paper_1610_05141_gb300 import build
    build.build()
    rs.load()
    return rs


@pytest.fixture(scope="module")
def ctx(rs):
    c = rs.rs_create(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def oracle():
    import oracle as o
    o.build()
    return o


def _sizes(p, seed, lo, hi, zeros=0):
    rng = np.random.default_rng(seed)
    L = np.floor(np.exp2(lo + (hi - lo) * rng.random(p))).astype(np.uint64)
    if zeros:
        L[rng.integers(0, p, zeros)] = 0
    return L


COUNT_CASES = [
    (np.array([5, 100, 0, 37, 1000, 3], dtype=np.uint64), 300, 7),
    (np.array([7], dtype=np.uint64), 4, 9),
    (np.array([2**61, 2**61], dtype=np.uint64), 10**9, 3),
    (_sizes(1000, 1, 0, 30, zeros=50), 10**6, 11),
    (_sizes(4097, 2, 10, 48), 10**8, 12),
    (_sizes(3, 3, 40, 58), 5 * 10**8, 2**64 - 1),
]


@pytest.mark.parametrize("case", range(len(COUNT_CASES)))
def test_union_counts_match_oracle(rs, ctx, oracle, case):
    L, n, seed = COUNT_CASES[case]
    got = rs.rs_union_counts(ctx, L, n, seed)
    want = oracle.union_counts(L, n, seed)
    assert np.array_equal(got, want), (case, int(np.argmax(got != want)))


SAMPLE_CASES = [
    (np.array([5, 100, 0, 37, 1000, 3], dtype=np.uint64), 300, 7, 16),
    (np.array([3, 0, 5, 2], dtype=np.uint64), 10, 1, 4),            # n = N
    (np.array([10**9], dtype=np.uint64), 5000, 5, 64),               # one segment
    (_sizes(37, 4, 8, 40, zeros=3), 200000, 13, 1024),
    (_sizes(1000, 5, 0, 34, zeros=20), 10**6, 14, 4096),
]


@pytest.mark.parametrize("case", range(len(SAMPLE_CASES)))
def test_union_sample_matches_oracle(rs, ctx, oracle, case):
    L, n, seed, n0 = SAMPLE_CASES[case]
    out = torch.full((max(n, 1),), -1, dtype=torch.int64, device="cuda")
    counts = rs.rs_union_sample(ctx, L, n, seed, n0, out)
    want, wcounts = oracle.union_sample(L, n, seed, n0)
    assert np.array_equal(counts, wcounts)
    got = out[:n].cpu().numpy().view(np.uint64)
    if not np.array_equal(got, want):
        bad = int(np.argmax(got != want))
        raise AssertionError(f"case {case}: first mismatch at {bad}: gpu {got[bad]} oracle {want[bad]}")


def test_union_zero_and_invalid(rs, ctx):
    L = np.array([3, 0, 5], dtype=np.uint64)
    assert np.array_equal(rs.rs_union_counts(ctx, L, 0, 1), [0, 0, 0])
    out = torch.full((4,), -1, dtype=torch.int64, device="cuda")
    assert np.array_equal(rs.rs_union_sample(ctx, L, 0, 1, 16, out), [0, 0, 0])
    assert int(out[0]) == -1
    for bad in [(L, 9, 1), (np.array([2**62, 1], dtype=np.uint64), 1, 1)]:
        with pytest.raises(rs.RSError) as e:
            rs.rs_union_counts(ctx, *bad)
        assert e.value.code == rs.RS_EINVAL
    with pytest.raises(rs.RSError):
        rs.rs_union_sample(ctx, L, 2, 1, 0, out)
    assert rs.rs_union_key(5, 0) == (5 + 0x9E3779B97F4A7C15) % 2**64


def test_union_full_size(rs, ctx, oracle):
    """The union the benchmark times (4096 segments of sizes log-uniform in
    2^20..2^40, n = 1e8): counts equal the oracle's, every segment's values
    increase strictly inside 1..L_i (checked on the device), and sampled
    segments equal the oracle's samples of their size and key."""
    from paper_1610_05141_gb300.workloads import union_segments
    L, n, seed, n0 = union_segments(), 10**8, 5, 4096
    out = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    counts = rs.rs_union_sample(ctx, L, n, seed, n0, out)
    assert np.array_equal(counts, oracle.union_counts(L, n, seed))
    off = np.zeros(len(L), dtype=np.int64)
    off[1:] = np.cumsum(counts.astype(np.int64))[:-1]
    starts = torch.zeros(n, dtype=torch.bool, device="cuda")
    nz = counts > 0
    starts[torch.as_tensor(off[nz], device="cuda")] = True
    assert bool(((out[1:] > out[:-1]) | starts[1:]).all()) and bool((out >= 1).all())
    last = torch.as_tensor(off[nz] + counts[nz].astype(np.int64) - 1, device="cuda")
    assert bool((out[last] <= torch.as_tensor(L[nz].astype(np.int64), device="cuda")).all())
    rng = np.random.default_rng(seed)
    idx = np.flatnonzero(nz)
    for i in sorted(set(rng.choice(idx, 12).tolist()) | {int(idx[0]), int(idx[-1]), int(np.argmax(counts))}):
        c = int(counts[i])
        want = oracle.sample(c, int(L[i]), oracle.union_key(seed, i), n0)
        got = out[off[i]:off[i] + c].cpu().numpy().view(np.uint64)
        assert np.array_equal(got, want), (i, c, int(L[i]))
    del out, starts
    torch.cuda.empty_cache()
