"""Failure paths, reached without faulting the GPU.

The method's loops have caps (the ratio-of-uniforms trials and inversion
restarts of a split deviate, Sec. 3.1; the Philox blocks of a candidate or
skip stream; the attempts of an Algorithm B leaf, Sec. 2).  A host-set
testing knob lowers them; a loop that reaches its cap must end with the
status RS_EITER as a normal return -- through rs_sync, a batch request's
status, a server job's result -- and the same context must sample correctly
once the caps are back.  The server's admission is made to fail as if host
memory ran out: those jobs finish with RS_ENOMEM and later jobs are served."""
import time

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


@pytest.fixture
def caps(rs):
    yield rs.rs_set_iteration_caps
    rs.rs_set_iteration_caps()   # the defaults again, whatever the test did


def _sample(rs, ctx, fn, n, N, seed, n0):
    out = torch.full((max(n, 1),), -1, dtype=torch.int64, device="cuda")
    fn(ctx, n, N, seed, n0, out)
    return rs.rs_sync(ctx), out[:n].cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("what", ["rou_trials", "inv_restarts", "stream_blocks", "b_attempts"])
def test_cap_ends_with_eiter_then_context_works(rs, ctx, oracle, caps, what):
    # (call, n, N, seed, n0, kind) whose run reaches the cap: split deviates by
    # ratio-of-uniforms (n = 1e6 from 1e9) or by inversion (small counts per
    # node), complement leaves drawn in rounds, Algorithm B leaves
    case = {"rou_trials": (rs.rs_sample, 10**6, 10**9, 1, 4096, oracle.KIND_H),
            "inv_restarts": (rs.rs_sample, 300, 10**6, 2, 8, oracle.KIND_H),
            "stream_blocks": (rs.rs_sample, 5000, 6000, 3, 128, oracle.KIND_H),
            "b_attempts": (rs.rs_sample_b, 10**5, 10**9, 4, 4096, oracle.KIND_B)}[what]
    fn, n, N, seed, n0, kind = case
    caps(**{what: 0 if what != "rou_trials" else 1})
    rc, _ = _sample(rs, ctx, fn, n, N, seed, n0)
    assert rc == rs.RS_EITER, rs.strerror(rc)
    caps()
    rc, got = _sample(rs, ctx, fn, n, N, seed, n0)
    assert rc == rs.RS_OK, rs.strerror(rc)
    assert np.array_equal(got, oracle.sample(n, N, seed, n0, kind))


def test_bernoulli_stream_cap(rs, ctx, oracle, caps):
    p, N, seed, n0 = 0.5, 2**20, 9, 4096
    out = torch.empty(N, dtype=torch.int64, device="cuda")
    caps(stream_blocks=1)   # two 64-bit values per chunk: every chunk runs out
    rc, _ = rs.rs_bernoulli(ctx, p, N, seed, n0, 0, N, out, N, check=False)
    rc2 = rs.rs_sync(ctx)
    assert rs.RS_EITER in (rc, rc2), (rc, rc2)
    caps()
    _, cnt = rs.rs_bernoulli(ctx, p, N, seed, n0, 0, N, out, N)
    assert rs.rs_sync(ctx) == rs.RS_OK
    assert np.array_equal(out[:cnt].cpu().numpy().view(np.uint64), oracle.bernoulli(p, N, seed, n0))


def test_batch_request_statuses(rs, ctx, oracle, caps):
    # requests with a split tree hit the one-trial cap; single-leaf requests
    # (n <= n0) do not, and keep their values
    reqs = [(10**6, 10**9, 11, 4096, 0), (3000, 10**9, 12, 4096, 0), (2**20, 2**40, 13, 4096, 1), (50, 10**4, 14, 64, 0)]
    n = [r[0] for r in reqs]
    off = np.zeros(len(reqs), dtype=np.uint64)
    off[1:] = np.cumsum(n)[:-1]
    arr = rs.requests_array(n, [r[1] for r in reqs], [r[2] for r in reqs], off, [r[3] for r in reqs],
                            [r[4] for r in reqs])
    plan = rs.rs_batch_plan(ctx, arr)
    pool = torch.full((int(sum(n)),), -1, dtype=torch.int64, device="cuda")
    status = torch.full((len(reqs),), -7, dtype=torch.int32, device="cuda")
    try:
        caps(rou_trials=1)
        rs.rs_batch_run(plan, pool, status)
        torch.cuda.synchronize()
        st = status.cpu().numpy()
        assert st[0] == rs.RS_EITER and st[2] == rs.RS_EITER, st
        assert st[1] == rs.RS_OK, st
        got = pool.cpu().numpy().view(np.uint64)
        assert np.array_equal(got[off[1]:off[1] + n[1]], oracle.sample(*reqs[1][:4], 0))
        caps()
        rs.rs_batch_run(plan, pool, status)
        torch.cuda.synchronize()
        assert (status.cpu().numpy() == rs.RS_OK).all()
        got = pool.cpu().numpy().view(np.uint64)
        for i, (nn, N, seed, n0, kind) in enumerate(reqs):
            assert np.array_equal(got[off[i]:off[i] + nn], oracle.sample(nn, N, seed, n0, kind)), i
    finally:
        plan.close()


def _drain(server, tickets, timeout_s=60.0):
    got = {}
    t_end = time.time() + timeout_s
    while len(got) < len(tickets):
        assert time.time() < t_end, "server did not finish"
        for r in server.poll(wait_us=20000):
            got[r.ticket] = r
    return got


def test_server_admission_out_of_memory_then_serves(rs, ctx, oracle):
    server = rs.rs_server_create(ctx, arena_bytes=1 << 26, lanes=2)
    try:
        server.fail_next_plans(1)
        t1 = server.submit(rs.sample_job(20000, 10**9, 21, 4096))
        r1 = _drain(server, [t1])[t1]
        assert r1.status == rs.RS_ENOMEM
        server.release(t1)
        tickets = [server.submit(rs.sample_job(20000 + i, 10**9, 22 + i, 4096)) for i in range(3)]
        res = _drain(server, tickets)
        for i, t in enumerate(tickets):
            r = res[t]
            assert r.status == rs.RS_OK, rs.strerror(r.status)
            got = rs.device_view(r.out_dev, r.count).cpu().numpy().view(np.uint64)
            assert np.array_equal(got, oracle.sample(20000 + i, 10**9, 22 + i, 4096))
            server.release(t)
    finally:
        server.close()


def test_server_job_reports_eiter(rs, ctx, oracle, caps):
    server = rs.rs_server_create(ctx, arena_bytes=1 << 26, lanes=2)
    try:
        caps(rou_trials=1)
        t1 = server.submit(rs.sample_job(10**6, 10**9, 31, 4096))
        r1 = _drain(server, [t1])[t1]
        assert r1.status == rs.RS_EITER
        server.release(t1)
        caps()
        t2 = server.submit(rs.sample_job(10**6, 10**9, 31, 4096))
        r2 = _drain(server, [t2])[t2]
        assert r2.status == rs.RS_OK
        got = rs.device_view(r2.out_dev, r2.count).cpu().numpy().view(np.uint64)
        assert np.array_equal(got, oracle.sample(10**6, 10**9, 31, 4096))
        server.release(t2)
    finally:
        server.close()
