"""Parity at the full sizes the benchmark times, in the same launch
configuration (one call of the C ABI over the whole workload): the oracle
cannot produce 10^9 values in seconds, so sampled parts of the output are
recomputed one by one by the oracle (whole leaves, at the leaf records the
oracle's own split tree gives), and the rest is checked by properties that
hold at any size (order, range, count), on the device."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SAMPLED_LEAVES = 40


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


def _check_leaves(got_dev, oracle, seed, kind, n, N, n0):
    recs, D = oracle.tree(n, N, seed, n0, kind)
    assert int(recs[-1][3]) + int(recs[-1][2]) == n
    rng = np.random.default_rng(seed + 1000 * kind)
    picks = set(rng.integers(0, len(recs), SAMPLED_LEAVES).tolist()) | {0, len(recs) // 2, len(recs) - 1}
    for i in sorted(picks):
        lo, s, c, off = (int(x) for x in recs[i])
        want = oracle.leaf(seed, kind, D, i, recs[i])
        got = got_dev[off:off + c].cpu().numpy().view(np.uint64)
        if not np.array_equal(got, want):
            bad = int(np.argmax(got != want))
            raise AssertionError(f"leaf {i} of {len(recs)} (kind {kind}): first mismatch at {bad}: "
                                 f"gpu {got[bad]} oracle {want[bad]}")


@pytest.mark.parametrize("kind,n,N", [(0, 10**9, 2**50), (1, 10**9, 2**40), (2, 10**9, 2**50)])
def test_full_size_samples(rs, ctx, oracle, kind, n, N):
    """n = 1e9 sorted from 2^50 (Algorithm H leaves), with replacement from
    2^40, and with Algorithm B leaves: sampled leaves equal the oracle's,
    the whole output is sorted (strictly without replacement) inside 1..N."""
    seed, n0 = 1, 4096
    call = {0: rs.rs_sample, 1: rs.rs_sample_with_replacement, 2: rs.rs_sample_b}[kind]
    out = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    call(ctx, n, N, seed, n0, out)
    assert rs.rs_sync(ctx) == rs.RS_OK
    assert int(out[0]) >= 1 and int(out[-1]) <= N
    if kind == 1:
        assert bool(torch.all(out[1:] >= out[:-1]))
    else:
        assert bool(torch.all(out[1:] > out[:-1]))
    _check_leaves(out, oracle, seed, kind, n, N, n0)
    del out
    torch.cuda.empty_cache()


def test_full_size_bernoulli(rs, ctx, oracle):
    """Bernoulli p = 1e-2 over 2^36 positions, the whole range in one call:
    the count is within 6 sigma of N p, positions increase strictly inside
    1..N, and chunk-aligned slices equal the oracle's windows."""
    p, N, seed, n0 = 1e-2, 2**36, 7, 4096
    mean = N * p
    cap = int(mean + 10 * np.sqrt(mean)) + 1024
    out = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
    rc, cnt = rs.rs_bernoulli(ctx, p, N, seed, n0, 0, N, out, cap)
    assert rs.rs_sync(ctx) == rs.RS_OK
    assert abs(cnt - mean) < 6 * np.sqrt(mean * (1 - p))
    got = out[:cnt]
    assert int(got[0]) >= 1 and int(got[-1]) <= N
    assert bool(torch.all(got[1:] > got[:-1]))
    C = 1 << oracle.bern_chunk_log2(p, n0)
    nch = N // C
    rng = np.random.default_rng(seed)
    for c0 in sorted(set(rng.integers(0, nch - 2, 6).tolist()) | {0, nch - 2}):
        a, b = c0 * C, (c0 + 2) * C
        want = oracle.bernoulli(p, N, seed, n0, a, b)
        lo = int(torch.searchsorted(got, torch.tensor([a + 1], dtype=torch.int64, device="cuda")))
        sl = got[lo:lo + len(want)].cpu().numpy().view(np.uint64)
        assert np.array_equal(sl, want), (a, b)
        if lo + len(want) < cnt:
            assert int(got[lo + len(want)]) > b
    del out, got
    torch.cuda.empty_cache()


def _with_exact(rs, exact, fn):
    c = rs.rs_create(0)
    try:
        rs.rs_set_exact_deviates(c, exact)
        return fn(c)
    finally:
        c.close()


@pytest.mark.parametrize("p", [1e-2, 1e-4])
def test_full_size_bernoulli_guard_equals_fp64(rs, p):
    """Bernoulli over 2^36 positions (6.9e8 skips at p = 1e-2): the guarded
    skips and the FP64 definition give the same positions, compared on the
    device."""
    N, seed, n0 = 2**36, 7, 4096
    cap = int(N * p + 10 * np.sqrt(N * p)) + 1024
    outs = []
    for exact in (False, True):
        out = torch.full((cap,), -1, dtype=torch.int64, device="cuda")

        def call(c):
            rc, cnt = rs.rs_bernoulli(c, p, N, seed, n0, 0, N, out, cap)
            assert rs.rs_sync(c) == rs.RS_OK
            return cnt
        outs.append((_with_exact(rs, exact, call), out))
    assert outs[0][0] == outs[1][0]
    assert torch.equal(outs[0][1], outs[1][1])
    del outs
    torch.cuda.empty_cache()


def test_full_size_leaf_b_guard_equals_fp64(rs):
    """Algorithm B leaves at n = 1e9 from 2^50 (skips of mean 1.1e6 for
    leaves of 2^32 positions): guarded and FP64 skips give the same sample."""
    n, N, seed, n0 = 10**9, 2**50, 1, 4096
    outs = []
    for exact in (False, True):
        out = torch.full((n,), -1, dtype=torch.int64, device="cuda")

        def call(c):
            rs.rs_sample_b(c, n, N, seed, n0, out)
            assert rs.rs_sync(c) == rs.RS_OK
        _with_exact(rs, exact, call)
        outs.append(out)
    assert torch.equal(outs[0], outs[1])
    del outs
    torch.cuda.empty_cache()


def test_full_size_batch(rs, ctx, oracle):
    """The 100,000-request batch the benchmark times (7.19e9 values), as a
    graph-replayed run after the eager one and a tuning pass: every request
    succeeds, every request's values increase strictly inside 1..N (checked
    on the device), and sampled requests equal the oracle's samples."""
    from paper_1610_05141_gb300.workloads import batch_requests
    n, N, seeds, off, n0, total = batch_requests(R=100000)
    kinds = np.zeros(len(n), dtype=np.uint32)
    plan = rs.rs_batch_plan(ctx, rs.requests_array(n, N, seeds, off, n0, kinds))
    pool = torch.full((total,), -1, dtype=torch.int64, device="cuda")
    status = torch.empty(len(n), dtype=torch.int32, device="cuda")
    try:
        rs.rs_batch_run(plan, pool, status)
        rs.rs_batch_tune(plan, pool, status)
        rs.rs_batch_run(plan, pool, status)
        torch.cuda.synchronize()
        assert bool((status == 0).all())
        # order inside each request: the value steps up everywhere except at a
        # request's first value, which is at least 1; the last value of each
        # request is at most its N
        starts = torch.zeros(total, dtype=torch.bool, device="cuda")
        starts[torch.as_tensor(off.astype(np.int64), device="cuda")] = True
        step_ok = (pool[1:] > pool[:-1]) | starts[1:]
        assert bool(step_ok.all()) and bool((pool[starts] >= 1).all())
        last = torch.as_tensor((off + n - 1).astype(np.int64), device="cuda")
        assert bool((pool[last] <= torch.as_tensor(N.astype(np.int64), device="cuda")).all())
        rng = np.random.default_rng(20161017)
        for i in sorted(set(rng.integers(0, len(n), 24).tolist()) | {0, len(n) - 1, int(np.argmax(n))}):
            ni = int(n[i])
            want = oracle.sample(ni, int(N[i]), int(seeds[i]), int(n0[i]), 0)
            got = pool[int(off[i]):int(off[i]) + ni].cpu().numpy().view(np.uint64)
            assert np.array_equal(got, want), (i, ni, int(N[i]))
    finally:
        plan.close()
        del pool, status
        torch.cuda.empty_cache()


def test_full_size_bernoulli_by_size(rs, ctx, oracle):
    """Bernoulli p = 1e-2 over 2^36 positions drawn by its size, the whole
    range in one call: the size equals the oracle's, positions increase
    strictly inside 1..N, and slices at sampled windows equal the oracle's
    range queries of the same sample."""
    p, N, seed, n0 = 1e-2, 2**36, 7, 4096
    tot = oracle.bernoulli_size(p, N, seed)
    cap = tot + 1024
    out = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
    rc, cnt, tot2 = rs.rs_bernoulli_by_size(ctx, p, N, seed, n0, 0, N, out, cap)
    assert rs.rs_sync(ctx) == rs.RS_OK
    assert tot2 == tot and cnt == tot
    got = out[:cnt]
    assert int(got[0]) >= 1 and int(got[-1]) <= N and bool(torch.all(got[1:] > got[:-1]))
    rng = np.random.default_rng(seed)
    for a in sorted(int(x) for x in rng.integers(0, N - 2**22, 6)):
        b = a + 2**22 + 12345
        want, _ = oracle.bernoulli_by_size(p, N, seed, n0, a, b)
        lo = int(torch.searchsorted(got, torch.tensor([a + 1], dtype=torch.int64, device="cuda")))
        sl = got[lo:lo + len(want)].cpu().numpy().view(np.uint64)
        assert np.array_equal(sl, want), (a, b)
    del out, got
    torch.cuda.empty_cache()

