"""Parity of the CUDA path (through the C ABI) with the CPU oracle: bit-exact
for every output (integers), on the same seeded inputs, at sizes the oracle
finishes in seconds (several leaves and ragged tails), plus edge cases
(empty, single element, full range, complement leaves, 64-bit leaves,
the general path for oversized leaves)."""
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


def run(rs, ctx, fn, n, N, seed, n0):
    out = torch.full((max(n, 1),), -1, dtype=torch.int64, device="cuda")
    fn(ctx, n, N, seed, n0, out)
    rc = rs.rs_sync(ctx)
    assert rc == rs.RS_OK, rs.strerror(rc)
    return out[:n].cpu().numpy().view(np.uint64)


def assert_same(got, want, what):
    assert got.shape == want.shape, (what, got.shape, want.shape)
    if not np.array_equal(got, want):
        bad = int(np.argmax(got != want))
        raise AssertionError(f"{what}: first mismatch at {bad}: gpu {got[bad]} oracle {want[bad]}")


H_CASES = [
    (10**6, 10**9, 1, 4096),            # n = 10^6 from N = 10^9 (the small workload)
    (1, 1, 5, 4),
    (5, 5, 1, 1),
    (1000, 1000, 2, 16),                # every leaf full: complement path
    (999, 1000, 3, 16),
    (600, 1000, 4, 64),
    (501, 1000, 7, 1024),
    (4096, 10**9, 9, 4096),             # one leaf, k = n0
    (7000, 10**4, 17, 4096),            # complement leaves with many duplicate draws
    (10**5, 2**62, 11, 4096),           # 64-bit candidates and keys
    (3 * 10**5, 3 * 2**40 + 7, 13, 1024),
    (10**5, 2**32 + 12345, 12, 512),
    (2 * 10**5, 2**33, 14, 4096),
    (10**6, 2**33 + 1, 15, 2),          # tiny leaves
    (100, 150, 16, 1),                  # depth capped by N
    (123457, 3906250 * 3 + 17, 21, 333),
    (8191, 2**20, 22, 8191),            # one leaf near the shared-memory capacity
    (2 * 10**5, (2**31 + 12345) * 64, 31, 4096),   # leaves just above 2^31: half the candidates void
    (4000, 2**61 + 999, 33, 4096),                 # one leaf, 64-bit candidates, an eighth void
    (256000, 20480000, 41, 4096),                  # leaves of 320000 positions: ~25 repeats each
    (256000, (2**22 + 12345) * 64, 43, 4096),      # ~4 void candidates and ~2 repeats per leaf
]


@pytest.mark.parametrize("n,N,seed,n0", H_CASES)
def test_sample_matches_oracle(rs, ctx, oracle, n, N, seed, n0):
    got = run(rs, ctx, rs.rs_sample, n, N, seed, n0)
    assert_same(got, oracle.sample(n, N, seed, n0, oracle.KIND_H), (n, N, seed, n0))


def test_sample_empty(rs, ctx):
    out = torch.full((4,), -1, dtype=torch.int64, device="cuda")
    rs.rs_sample(ctx, 0, 10, 1, 4, out)
    assert rs.rs_sync(ctx) == rs.RS_OK
    assert out.cpu().tolist() == [-1] * 4


WR_CASES = [
    (10**6, 2**40, 1, 4096),
    (10**5, 1000, 2, 512),               # n > N
    (50, 3, 3, 4),
    (10**5, 2**62, 4, 4096),
    (77777, 10**9 + 7, 5, 100),
    (10**5, (2**31 + 777) * 32, 6, 4096),   # half the candidates void
]


@pytest.mark.parametrize("n,N,seed,n0", WR_CASES)
def test_with_replacement_matches_oracle(rs, ctx, oracle, n, N, seed, n0):
    got = run(rs, ctx, rs.rs_sample_with_replacement, n, N, seed, n0)
    assert_same(got, oracle.sample(n, N, seed, n0, oracle.KIND_WR), (n, N, seed, n0))


B_CASES = [
    (10**5, 10**8, 1, 4096),
    (999, 1000, 2, 16),
    (300, 10**12, 3, 64),
    (20000, 2**62, 4, 2048),
    (5000, 6000, 5, 128),
]


@pytest.mark.parametrize("n,N,seed,n0", B_CASES)
def test_leaf_b_matches_oracle(rs, ctx, oracle, n, N, seed, n0):
    got = run(rs, ctx, rs.rs_sample_b, n, N, seed, n0)
    assert_same(got, oracle.sample(n, N, seed, n0, oracle.KIND_B), (n, N, seed, n0))


@pytest.mark.parametrize("n,N,seed,n0", B_CASES)
def test_leaf_b_exact_skips_match_oracle(rs, oracle, n, N, seed, n0):
    """With every geometric skip evaluated in FP64 (rs_set_exact_deviates),
    leaf B gives the oracle's sample too, so both settings give it."""
    c = rs.rs_create(0)
    try:
        rs.rs_set_exact_deviates(c, True)
        got = run(rs, c, rs.rs_sample_b, n, N, seed, n0)
    finally:
        c.close()
    assert_same(got, oracle.sample(n, N, seed, n0, oracle.KIND_B), (n, N, seed, n0))


@pytest.mark.parametrize("cap", [64, 1000])
def test_general_leaf_path_matches_oracle(rs, oracle, cap):
    """Leaves whose selection exceeds the capacity take the global-memory
    path; forcing a tiny capacity must not change a single value."""
    c = rs.rs_create(0)
    try:
        rs.rs_set_leaf_capacity(c, cap)
        for fn, kind, n, N, seed, n0 in [(rs.rs_sample, oracle.KIND_H, 20000, 10**8, 18, 4096),
                                         (rs.rs_sample, oracle.KIND_H, 3000, 5000, 19, 4096),
                                         (rs.rs_sample, oracle.KIND_H, 5000, 2**50, 20, 8192),
                                         (rs.rs_sample_with_replacement, oracle.KIND_WR, 9000, 5000, 21, 4096)]:
            got = run(rs, c, fn, n, N, seed, n0)
            assert_same(got, oracle.sample(n, N, seed, n0, kind), (cap, n, N))
    finally:
        c.close()


TREE_CASES = [
    (10**6, 10**9, 1, 4096, 0),
    (10**9, 2**50, 1, 4096, 0),          # the large workload: all 2^18 leaf records
    (10**9, 2**40, 1, 4096, 1),          # with replacement: binomial splits
    (999, 1000, 3, 3, 0),
    (5000, 77, 16, 16, 1),
    (10**5, 2**62, 4, 4096, 0),
]


@pytest.mark.parametrize("n,N,seed,n0,kind", TREE_CASES)
def test_split_tree_matches_oracle(rs, ctx, oracle, n, N, seed, n0, kind):
    want, D = oracle.tree(n, N, seed, n0, kind)
    recs = torch.zeros(4 * len(want), dtype=torch.int64, device="cuda")
    rs.rs_split_tree(ctx, n, N, seed, n0, kind, recs, len(want))
    assert rs.rs_sync(ctx) == rs.RS_OK
    got = recs.cpu().numpy().view(np.uint64).reshape(-1, 4)
    assert_same(got.ravel(), want.ravel(), (n, N, kind))


GUARD_CASES = TREE_CASES + [
    (7 * 10**8, 3 * 2**47 + 5, 11, 1000, 0),   # ragged sizes, deeper tree
    (123456789, 987654321012, 12, 300, 1),
    (2**40, 2**45, 13, 2**22, 0),              # a shallow tree of huge counts
]


@pytest.mark.parametrize("n,N,seed,n0,kind", GUARD_CASES)
def test_split_tree_guard_equals_fp64(rs, n, N, seed, n0, kind):
    """The single-precision guard of the ratio-of-uniforms tests only
    decides trials far from the boundary: the whole tree is the same bits
    with the guard and with every test evaluated in FP64."""
    D = rs.rs_plan(n, N, n0)
    recs = []
    for exact in (False, True):
        c = rs.rs_create(0)
        try:
            rs.rs_set_exact_deviates(c, exact)
            r = torch.zeros(4 << D, dtype=torch.int64, device="cuda")
            rs.rs_split_tree(c, n, N, seed, n0, kind, r, 1 << D)
            assert rs.rs_sync(c) == rs.RS_OK
            recs.append(r.cpu().numpy())
        finally:
            c.close()
    assert np.array_equal(recs[0], recs[1]), (n, N, kind)


BERN_CASES = [
    (1e-4, 2**28, 7, 4096),
    (1e-2, 2**24, 7, 4096),
    (0.5, 2**20, 7, 4096),
    (0.3, 10**6 + 7, 8, 64),
    (0.999, 5000, 9, 16),
    (1e-15, 2**62, 5, 4096),
]


@pytest.mark.parametrize("p,N,seed,n0", BERN_CASES)
def test_bernoulli_matches_oracle(rs, ctx, oracle, p, N, seed, n0):
    want = oracle.bernoulli(p, N, seed, n0)
    cap = len(want) + 16
    out = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
    rc, cnt = rs.rs_bernoulli(ctx, p, N, seed, n0, 0, N, out, cap)
    assert rs.rs_sync(ctx) == rs.RS_OK
    assert cnt == len(want)
    assert_same(out[:cnt].cpu().numpy().view(np.uint64), want, (p, N))


@pytest.mark.parametrize("p,N,seed,n0", BERN_CASES)
def test_bernoulli_exact_skips_match_oracle(rs, oracle, p, N, seed, n0):
    """Every skip in FP64 (rs_set_exact_deviates): the oracle's positions,
    as with the guarded skips above."""
    want = oracle.bernoulli(p, N, seed, n0)
    cap = len(want) + 16
    out = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
    c = rs.rs_create(0)
    try:
        rs.rs_set_exact_deviates(c, True)
        rc, cnt = rs.rs_bernoulli(c, p, N, seed, n0, 0, N, out, cap)
        assert rs.rs_sync(c) == rs.RS_OK
    finally:
        c.close()
    assert cnt == len(want)
    assert_same(out[:cnt].cpu().numpy().view(np.uint64), want, (p, N))


@pytest.mark.parametrize("limit,slots", [(0, 0), (16 << 30, 8), (16 << 30, 4000)])
def test_bernoulli_two_walks_and_restaged_chunks(rs, ctx, oracle, limit, slots):
    """Without staging (two walks per chunk), and with too few staging slots
    for most chunks (those walk again for the copy): the same positions."""
    try:
        rs.rs_set_bernoulli_staging(ctx, limit, slots)
        for p, N, seed, n0 in BERN_CASES[:4]:
            want = oracle.bernoulli(p, N, seed, n0)
            cap = len(want) + 16
            out = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
            rc, cnt = rs.rs_bernoulli(ctx, p, N, seed, n0, 0, N, out, cap)
            assert rs.rs_sync(ctx) == rs.RS_OK
            assert cnt == len(want)
            assert_same(out[:cnt].cpu().numpy().view(np.uint64), want, (p, N, limit, slots))
    finally:
        rs.rs_set_bernoulli_staging(ctx)


def test_bernoulli_windows_degenerate_and_capacity(rs, ctx, oracle):
    p, N, seed, n0 = 0.01, 10**7 + 123, 7, 1024
    C = 1 << oracle.bern_chunk_log2(p, n0)
    for a, b in [(0, C), (C, 5 * C), (3 * C, N), ((N // C) * C, N)]:
        want = oracle.bernoulli(p, N, seed, n0, a, b)
        out = torch.empty(len(want) + 8, dtype=torch.int64, device="cuda")
        rc, cnt = rs.rs_bernoulli(ctx, p, N, seed, n0, a, b, out, len(want) + 8)
        assert cnt == len(want)
        assert_same(out[:cnt].cpu().numpy().view(np.uint64), want, (a, b))
    out = torch.empty(1000, dtype=torch.int64, device="cuda")
    rc, cnt = rs.rs_bernoulli(ctx, 1.0, 1000, 1, 16, 0, 1000, out, 1000)
    assert cnt == 1000 and out.cpu().tolist() == list(range(1, 1001))
    rc, cnt = rs.rs_bernoulli(ctx, 0.0, 1000, 1, 16, 0, 1000, out, 1000)
    assert cnt == 0
    want = oracle.bernoulli(0.5, 1000, 1, 16)
    rc, cnt = rs.rs_bernoulli(ctx, 0.5, 1000, 1, 16, 0, 1000, out, 10, check=False)
    assert rc == rs.RS_ECAPACITY and cnt == len(want)
    assert_same(out[:10].cpu().numpy().view(np.uint64), want[:10], "capped")
    rc, _ = rs.rs_bernoulli(ctx, 0.5, 1000, 1, 16, 3, 1000, out, 1000, check=False)
    assert rc == rs.RS_EINVAL


SIZE_CASES = [(0.3, 1000, 1), (1e-2, 2**36, 7), (0.5, 2**36, 7), (0.8, 10**6, 3), (1e-15, 2**62, 5),
              (0.0, 100, 1), (1.0, 100, 1), (0.5, 2**62, 9), (2e-6, 10**7, 4)]


@pytest.mark.parametrize("p,N,seed", SIZE_CASES)
def test_bernoulli_size_matches_oracle(rs, ctx, oracle, p, N, seed):
    """The BIN(N, p) size of the sample drawn by its size: the device's
    deviate equals the oracle's (inversion and ratio-of-uniforms, p > 1/2 by
    the complement)."""
    assert rs.rs_bernoulli_size(ctx, p, N, seed) == oracle.bernoulli_size(p, N, seed)


BY_SIZE_CASES = [(0.3, 10**6 + 7, 8, 64), (1e-2, 2**24, 7, 4096), (0.5, 2**20, 7, 4096), (0.9, 5000, 9, 16),
                 (1e-4, 2**30, 3, 4096)]


@pytest.mark.parametrize("p,N,seed,n0", BY_SIZE_CASES)
def test_bernoulli_by_size_matches_oracle(rs, ctx, oracle, p, N, seed, n0):
    """Bernoulli sampling by its size: the whole range (rs_sample of the
    size) and windows with any ends (range queries of that sample) equal the
    oracle's, with the same counts."""
    want, tot = oracle.bernoulli_by_size(p, N, seed, n0)
    cap = len(want) + 16
    out = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
    rc, cnt, tot2 = rs.rs_bernoulli_by_size(ctx, p, N, seed, n0, 0, N, out, cap)
    assert rs.rs_sync(ctx) == rs.RS_OK
    assert tot2 == tot and cnt == len(want)
    assert_same(out[:cnt].cpu().numpy().view(np.uint64), want, ("whole", p, N))
    for a, b in [(0, N // 3), (N // 7 + 1, N // 2 + 3), (N - N // 5 - 1, N), (5, 5)]:
        w, _ = oracle.bernoulli_by_size(p, N, seed, n0, a, b)
        rc, cnt, tot3 = rs.rs_bernoulli_by_size(ctx, p, N, seed, n0, a, b, out, cap)
        assert tot3 == tot and cnt == len(w), (a, b)
        assert_same(out[:cnt].cpu().numpy().view(np.uint64), w, ("window", p, N, a, b))
    rc, cnt, _ = rs.rs_bernoulli_by_size(ctx, p, N, seed, n0, 0, N, out, 3, check=False)
    if tot > 3:
        assert rc == rs.RS_ECAPACITY and cnt == tot
    assert rs.rs_bernoulli_by_size(ctx, p, N, seed, n0, 7, 3, out, cap, check=False)[0] == rs.RS_EINVAL


def test_argument_errors(rs, ctx):
    out = torch.empty(16, dtype=torch.int64, device="cuda")
    assert rs.rs_sample(ctx, 11, 10, 1, 4, out, check=False) == rs.RS_EINVAL
    assert rs.rs_sample(ctx, 1, 10, 1, 0, out, check=False) == rs.RS_EINVAL
    assert rs.rs_sample(ctx, 1, 0, 1, 4, out, check=False) == rs.RS_EINVAL
    assert rs.rs_sample(ctx, 1, 2**62 + 1, 1, 4, out, check=False) == rs.RS_EINVAL
    assert rs.rs_sample(ctx, 1, 10, 1, 4, None, check=False) == rs.RS_EINVAL
    assert rs.rs_sample(ctx, 1, 10, 1, 4, out.data_ptr() + 4, check=False) == rs.RS_EINVAL
    assert rs.rs_sample_with_replacement(ctx, 11, 10, 1, 4, out, check=False) == rs.RS_OK
    assert rs.rs_sync(ctx) == rs.RS_OK


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_pipelined_tree_matches_oracle(rs, ctx, oracle, kind):
    """Subtrees built on the tree stream while earlier subtrees' leaves run:
    the same output as the sequential schedule and as the oracle."""
    n, seed, n0 = 4 * 10**6, 77 + kind, 1024         # depth 12: 8 subtrees of 512 leaves
    N = 2**40 if kind == 1 else 2**50
    call = {0: rs.rs_sample, 1: rs.rs_sample_with_replacement, 2: rs.rs_sample_b}[kind]
    try:
        rs.rs_set_pipeline(ctx, 3, 3)
        got = run(rs, ctx, call, n, N, seed, n0)
        rs.rs_set_pipeline(ctx, 0, 0)
        seq = run(rs, ctx, call, n, N, seed, n0)
    finally:
        rs.rs_set_pipeline(ctx, 0, 3)
    assert_same(got, seq, ("pipelined vs sequential", kind))
    assert_same(got, oracle.sample(n, N, seed, n0, kind), (n, N, seed, n0, kind))


@pytest.mark.parametrize("kind,N", [(0, 2**47), (0, 2**44), (0, 10**9 + 7), (1, 2**40), (0, 2**60)])
def test_large_leaf_shape_matches_oracle(rs, ctx, oracle, kind, N):
    """Leaves averaging about 6,000 samples take the 512-thread leaf kernel
    with room for 9,728 values: every sampled leaf equals the oracle's."""
    n, seed, n0 = 2 * 10**7, 91 + kind, 8192           # depth 12, ~4,900 samples per leaf
    n, n0 = (6 * 10**7, 8192) if N == 2**47 else (n, n0)   # depth 13, ~7,300 per leaf
    call = {0: rs.rs_sample, 1: rs.rs_sample_with_replacement}[kind]
    got = run(rs, ctx, call, n, N, seed, n0)
    recs, D = oracle.tree(n, N, seed, n0, kind)
    rng = np.random.default_rng(seed)
    for i in sorted(set(rng.integers(0, len(recs), 24).tolist()) | {0, len(recs) - 1}):
        lo, s, c, off = (int(x) for x in recs[i])
        want = oracle.leaf(seed, kind, D, i, recs[i])
        assert_same(got[off:off + c], want, ("leaf", i, n, N, kind))


@pytest.mark.parametrize("kind,n,N,n0,pinned", [(0, 10**6, 10**9, 4096, True), (1, 10**6, 2**40, 4096, True),
                                                (2, 10**5, 10**8, 4096, False), (0, 3000, 10**6, 4096, True),
                                                (0, 6 * 10**6, 2**50, 1024, False)])
def test_sample_to_host_matches_device_sample(rs, ctx, oracle, kind, n, N, n0, pinned):
    """The sample copied to host memory piece by piece while it is made equals
    the device sample and the oracle's."""
    seed = 57 + kind
    out = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    host = torch.full((n,), -1, dtype=torch.int64, pin_memory=pinned)
    rs.rs_sample_to_host(ctx, kind, n, N, seed, n0, out, host)
    assert rs.rs_sync(ctx) == rs.RS_OK
    got = host.numpy().view(np.uint64)
    assert np.array_equal(got, out.cpu().numpy().view(np.uint64))
    if n <= 10**6:
        assert_same(got, oracle.sample(n, N, seed, n0, kind), ("to host", kind, n, N))
