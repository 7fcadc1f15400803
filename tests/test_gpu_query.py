"""Range queries on resident split trees: the values of [a, b), regenerated
from the overlapping leaves only, equal the oracle's range query and the
slice of the full GPU sample, bit for bit, for every sample kind; ranges
inside one leaf, across two, across many, at leaf edges, clamped at both
ends, empty; the capacity error reports the count."""
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


def _query(rs, tree, a, b, cap):
    out = torch.full((max(cap, 1),), -1, dtype=torch.int64, device="cuda")
    rc, cnt = rs.rs_tree_query(tree, a, b, out, cap, check=False)
    return rc, cnt, out.cpu().numpy().view(np.uint64)[: min(cnt, cap)].copy()


def _leaf_edges(N, D):
    """0-based start positions of the 2^D leaves (split at floor(S/2))."""
    ranges = [(0, N)]
    for _ in range(D):
        nxt = []
        for lo, S in ranges:
            K = S // 2
            nxt += [(lo, K), (lo + K, S - K)]
        ranges = nxt
    return [lo for lo, _ in ranges]


def _ranges(N, D, rng, k=24):
    """Query ranges [a, b) of values: random ones plus leaf-edge, clamped and empty ones."""
    edges = _leaf_edges(N, D)
    out = [(0, N + 5), (1, N + 1), (0, 1), (N, N + 1), (5, 5), (7, 3), (N + 3, N + 9)]
    if len(edges) > 2:
        e = edges[len(edges) // 2]
        out += [(e + 1, e + 2), (e, e + 1), (e + 1, edges[len(edges) // 2 + 1] + 1),
                (edges[1] + 1, edges[-1] + 1), (edges[1], edges[-1] + 2)]
    for _ in range(k):
        a = int(rng.integers(0, N + 2))
        w = int(np.exp(rng.uniform(0, np.log(N + 2))))
        out.append((a, a + w))
    return out


CASES = [
    # (n, N, seed, n0, kind)
    (20000, 10**7, 11, 256, 0),
    (3000, 3000, 12, 64, 0),       # dense: complement / bitmap leaves
    (2900, 3000, 13, 64, 0),
    (50000, 2**62, 14, 512, 0),    # 64-bit leaves
    (30000, 5000, 15, 128, 1),     # with replacement, repeats
    (20000, 2**40, 16, 256, 1),
    (20000, 10**8, 17, 256, 2),    # Algorithm B leaves
    (1, 10**9, 18, 4096, 0),
    (7, 7, 19, 4, 0),
]


@pytest.mark.parametrize("case", CASES, ids=[f"n{c[0]}_N{c[1]}_k{c[4]}" for c in CASES])
def test_query_matches_oracle(rs, ctx, oracle, case):
    n, N, seed, n0, kind = case
    tree = rs.rs_tree_create(ctx, n, N, seed, n0, kind)
    D, maxc = rs.rs_tree_info(tree)
    assert D == oracle.depth(n, N, n0)
    full = oracle.sample(n, N, seed, n0, kind)
    rng = np.random.default_rng(seed)
    for a, b in _ranges(N, D, rng):
        lo, hi = np.searchsorted(full, a, "left"), np.searchsorted(full, b, "left")
        want = full[lo:hi] if a < b else full[:0]
        rc, cnt, got = _query(rs, tree, a, b, n)
        assert rc == rs.RS_OK, (a, b, rc)
        assert cnt == len(want), (a, b, cnt, len(want))
        assert np.array_equal(got, want), (a, b)
        if a < b and len(want) < 3000:
            assert np.array_equal(oracle.range_query(n, N, seed, n0, kind, a, b), want)
    tree.close()


def test_query_capacity_and_arguments(rs, ctx, oracle):
    n, N, seed, n0 = 20000, 10**7, 21, 256
    tree = rs.rs_tree_create(ctx, n, N, seed, n0, 0)
    full = oracle.sample(n, N, seed, n0)
    a, b = 2 * 10**6, 5 * 10**6
    want = int(np.searchsorted(full, b) - np.searchsorted(full, a))
    rc, cnt, _ = _query(rs, tree, a, b, want - 1)
    assert rc == rs.RS_ECAPACITY and cnt == want
    rc, cnt, got = _query(rs, tree, a, b, want)
    assert rc == rs.RS_OK and cnt == want
    assert np.array_equal(got, full[np.searchsorted(full, a):np.searchsorted(full, b)])
    rc, cnt = rs.rs_tree_query(tree, a, b, None, 0, check=False)
    assert rc == rs.RS_ECAPACITY and cnt == want
    with pytest.raises(rs.RSError):
        rs.rs_tree_create(ctx, 11, 10, 1, 4, 0)
    with pytest.raises(rs.RSError):
        rs.rs_tree_create(ctx, 5, 10, 1, 0, 0)
    empty = rs.rs_tree_create(ctx, 0, 10, 1, 4, 0)
    rc, cnt, _ = _query(rs, empty, 0, 100, 4)
    assert rc == rs.RS_OK and cnt == 0
    empty.close()
    tree.close()


@pytest.mark.parametrize("kind,N", [(0, 10**9), (0, 2**56), (1, 2**40), (2, 2**50)])
def test_query_is_slice_of_gpu_sample(rs, ctx, kind, N):
    """Larger trees (hundreds of leaves): queries equal slices of the GPU's
    own full sample of the same arguments."""
    n, seed, n0 = 10**6, 31 + kind, 4096
    full_t = torch.empty(n, dtype=torch.int64, device="cuda")
    call = {0: rs.rs_sample, 1: rs.rs_sample_with_replacement, 2: rs.rs_sample_b}[kind]
    call(ctx, n, N, seed, n0, full_t)
    assert rs.rs_sync(ctx) == rs.RS_OK
    full = full_t.cpu().numpy().view(np.uint64)
    tree = rs.rs_tree_create(ctx, n, N, seed, n0, kind)
    rng = np.random.default_rng(kind)
    for _ in range(20):
        a = int(rng.integers(1, N))
        w = int(N * 10 ** rng.uniform(-6, -0.3))
        b = a + w
        lo, hi = np.searchsorted(full, a), np.searchsorted(full, b)
        rc, cnt, got = _query(rs, tree, a, b, int(hi - lo) + 16)
        assert rc == rs.RS_OK and cnt == hi - lo
        assert np.array_equal(got, full[lo:hi]), (a, b)
    rc, cnt, got = _query(rs, tree, 0, N + 1, n)
    assert rc == rs.RS_OK and cnt == n and np.array_equal(got, full)
    tree.close()
