"""Batches (many independent requests in one device run): every request's
output equals its own single-call output, bit for bit -- against the oracle
for a mixed batch, and against the single GPU calls for a slice of the large
synthetic batch workload; eager and graph-replayed runs agree; bad requests
get their own status without disturbing the others."""
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


def _mixed_requests():
    rng = np.random.default_rng(5)
    reqs = []
    for i in range(160):
        kind = int(rng.integers(0, 3))
        n = int(np.exp(rng.uniform(0, np.log(60000))))
        if kind == 1:
            N = int(np.exp(rng.uniform(0, np.log(2**62))))
        else:
            N = n + int(np.exp(rng.uniform(0, np.log(2**62 - n))))
        n0 = int(rng.choice([64, 512, 4096]))
        reqs.append((n, N, 1000 + i, n0, kind))
    # edge cases: empty, full range, complement leaves, tiny with replacement, invalid ones
    reqs += [(0, 10, 1, 4, 0), (1000, 1000, 2, 16, 0), (999, 1000, 3, 16, 0), (50, 3, 4, 4, 1),
             (5000, 6000, 5, 128, 2), (11, 10, 6, 4, 0), (5, 10, 7, 0, 0), (5, 2**62 + 1, 8, 4, 0),
             (8191, 2**20, 9, 8191, 0)]
    return reqs


def _run(rs, ctx, reqs, runs=2):
    n = [r[0] for r in reqs]
    off = np.zeros(len(reqs), dtype=np.uint64)
    off[1:] = np.cumsum(n)[:-1]
    arr = rs.requests_array(n, [r[1] for r in reqs], [r[2] for r in reqs], off, [r[3] for r in reqs],
                            [r[4] for r in reqs])
    plan = rs.rs_batch_plan(ctx, arr)
    pool = torch.full((max(1, int(sum(n))),), -1, dtype=torch.int64, device="cuda")
    status = torch.full((len(reqs),), -7, dtype=torch.int32, device="cuda")
    results = []
    for _ in range(runs):
        pool.fill_(-1)
        rs.rs_batch_run(plan, pool, status)
        torch.cuda.synchronize()
        results.append((pool.cpu().numpy().view(np.uint64).copy(), status.cpu().numpy().copy()))
    plan.close()
    return off, results


def test_batch_matches_oracle_per_request(rs, ctx, oracle):
    reqs = _mixed_requests()
    off, results = _run(rs, ctx, reqs, runs=2)
    (pool0, st0), (pool1, st1) = results
    assert np.array_equal(pool0, pool1) and np.array_equal(st0, st1)   # eager run == graph replay
    for i, (n, N, seed, n0, kind) in enumerate(reqs):
        rc = oracle.sample_rc(n, N, seed, n0, kind) if n <= (1 << 20) else None
        if rc not in (None, oracle.OK):
            assert st0[i] == rs.RS_EINVAL, (i, reqs[i])
            continue
        assert st0[i] == rs.RS_OK, (i, reqs[i], st0[i])
        want = oracle.sample(n, N, seed, n0, kind)
        got = pool0[int(off[i]): int(off[i]) + n]
        assert np.array_equal(got, want), (i, reqs[i])


def test_batch_workload_slice_matches_single_calls(rs, ctx):
    from paper_1610_05141_gb300.workloads import batch_requests
    n, N, seeds, _, n0, _ = batch_requests(R=600, seed=20161017)
    reqs = [(int(n[i]), int(N[i]), int(seeds[i]), int(n0[i]), 0) for i in range(len(n))]
    off, results = _run(rs, ctx, reqs, runs=2)
    pool, st = results[1]
    assert (st == rs.RS_OK).all()
    for i, (ni, Ni, si, n0i, _) in enumerate(reqs):
        out = torch.empty(ni, dtype=torch.int64, device="cuda")
        rs.rs_sample(ctx, ni, Ni, si, n0i, out)
        assert rs.rs_sync(ctx) == rs.RS_OK
        assert np.array_equal(pool[int(off[i]): int(off[i]) + ni], out.cpu().numpy().view(np.uint64)), i


def test_batch_one_shot_device_requests_and_tune(rs, ctx, oracle):
    reqs = [(3000, 10**9, 11, 512, 0), (2000, 77, 12, 64, 1), (4000, 10**6, 13, 1024, 2)]
    n = [r[0] for r in reqs]
    off = np.zeros(len(reqs), dtype=np.uint64)
    off[1:] = np.cumsum(n)[:-1]
    arr = rs.requests_array(n, [r[1] for r in reqs], [r[2] for r in reqs], off, [r[3] for r in reqs],
                            [r[4] for r in reqs])
    raw = np.frombuffer(arr.tobytes(), dtype=np.uint8)
    reqs_dev = torch.from_numpy(raw.copy()).to("cuda")
    pool = torch.empty(sum(n), dtype=torch.int64, device="cuda")
    status = torch.empty(len(reqs), dtype=torch.int32, device="cuda")
    rs.rs_batch(ctx, reqs_dev, len(reqs), pool, status)
    got = pool.cpu().numpy().view(np.uint64)
    assert (status.cpu().numpy() == rs.RS_OK).all()
    for i, (ni, Ni, si, n0i, k) in enumerate(reqs):
        assert np.array_equal(got[int(off[i]): int(off[i]) + ni], oracle.sample(ni, Ni, si, n0i, k))
    plan = rs.rs_batch_plan(ctx, arr)
    rs.rs_batch_run(plan, pool, status)
    rs.rs_batch_tune(plan, pool, status)
    pool.fill_(0)
    rs.rs_batch_run(plan, pool, status)
    torch.cuda.synchronize()
    assert np.array_equal(pool.cpu().numpy().view(np.uint64), got)
    assert rs.rs_batch_launch_count(plan) > 0
    plan.close()


def _large_class_requests():
    """Requests of both size classes and both key widths: leaves averaging
    ~1,000 to ~8,000 values (n0 up to 8192), with and without replacement,
    sizes that are and are not powers of two."""
    rng = np.random.default_rng(17)
    reqs = []
    for i in range(48):
        kind = int(rng.integers(0, 2))
        n0 = int(rng.choice([1024, 4096, 6000, 8192]))
        n = int(n0 * rng.uniform(0.6, 1.0) * (1 << int(rng.integers(0, 4))))
        N = int(rng.choice([2**31 + 12345, 2**33, 3 * 2**40 + 7, 10**9])) * (1 << int(rng.integers(0, 3)))
        reqs.append((n, max(N, n), 3000 + i, n0, kind))
    return reqs


def test_batch_leaf_shapes_and_blocks_do_not_change_output(rs, ctx, oracle):
    """rs_batch_tune's knobs are output-invariant: every leaf shape of either
    size class (256 or 512 threads) and any blocks per SM give the same pool,
    which equals the oracle's samples."""
    reqs = _large_class_requests()
    n = [r[0] for r in reqs]
    off = np.zeros(len(reqs), dtype=np.uint64)
    off[1:] = np.cumsum(n)[:-1]
    arr = rs.requests_array(n, [r[1] for r in reqs], [r[2] for r in reqs], off, [r[3] for r in reqs],
                            [r[4] for r in reqs])
    plan = rs.rs_batch_plan(ctx, arr)
    pool = torch.empty(int(sum(n)), dtype=torch.int64, device="cuda")
    status = torch.empty(len(reqs), dtype=torch.int32, device="cuda")
    pools = []
    try:
        for small, large, per in [(0, 0, 0), (256, 256, 0), (512, 512, 0), (512, 256, 2), (256, 512, 1)]:
            rs.rs_batch_set_leaf_launch(plan, small, large, per)
            for _ in range(2):   # eager and graph replay
                pool.fill_(-1)
                rs.rs_batch_run(plan, pool, status)
                torch.cuda.synchronize()
                assert (status.cpu().numpy() == rs.RS_OK).all(), (small, large, per)
                pools.append(pool.cpu().numpy().view(np.uint64).copy())
        rs.rs_batch_tune(plan, pool, status)
        pool.fill_(-1)
        rs.rs_batch_run(plan, pool, status)
        torch.cuda.synchronize()
        pools.append(pool.cpu().numpy().view(np.uint64).copy())
        with pytest.raises(rs.RSError):
            rs.rs_batch_set_leaf_launch(plan, 300, 0, 0)
    finally:
        plan.close()
    for p in pools[1:]:
        assert np.array_equal(p, pools[0])
    for i in range(0, len(reqs), 5):
        ni, Ni, si, n0i, k = reqs[i]
        assert np.array_equal(pools[0][int(off[i]): int(off[i]) + ni], oracle.sample(ni, Ni, si, n0i, k)), i
