"""Serving with continuous batching: every job's values equal its single
call's (the oracle, rs_sample*, rs_tree_query), whether it ran alone or in
a mix; jobs submitted while a group runs start before it ends; admission by
arena memory never exceeds the arena; jobs that can never fit, or have bad
arguments, complete at once with their error."""
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


def _drain(rs, server, tickets, timeout_s=60.0, on_result=None):
    """Polls until every ticket has a result; returns {ticket: Result}."""
    got = {}
    t_end = time.time() + timeout_s
    while len(got) < len(tickets):
        assert time.time() < t_end, f"server did not finish: {len(got)} of {len(tickets)}"
        for r in server.poll(wait_us=20000):
            got[r.ticket] = r
            if on_result:
                on_result(r)
    return got


def _values(rs, r):
    return rs.device_view(r.out_dev, r.count).cpu().numpy().view(np.uint64).copy()


def _solo(rs, ctx, n, N, seed, n0, kind):
    out = torch.empty(max(n, 1), dtype=torch.int64, device="cuda")
    call = {0: rs.rs_sample, 1: rs.rs_sample_with_replacement, 2: rs.rs_sample_b}[kind]
    call(ctx, n, N, seed, n0, out)
    assert rs.rs_sync(ctx) == rs.RS_OK
    return out[:n].cpu().numpy().view(np.uint64).copy()


def _solo_query(rs, tree, a, b, cap):
    out = torch.empty(max(cap, 1), dtype=torch.int64, device="cuda")
    rc, cnt = rs.rs_tree_query(tree, a, b, out, cap, check=False)
    return rc, cnt, out[: min(cnt, cap)].cpu().numpy().view(np.uint64).copy()


def test_mix_equals_solo(rs, ctx, oracle):
    rng = np.random.default_rng(77)
    trees = [rs.rs_tree_create(ctx, 10**6, 2**56, 901, 4096, 0),
             rs.rs_tree_create(ctx, 200000, 2**40, 902, 1024, 1),
             rs.rs_tree_create(ctx, 100000, 10**8, 903, 512, 2)]
    jobs = []
    for i in range(240):
        if rng.random() < 0.25:
            t = trees[int(rng.integers(0, 3))]
            a = int(rng.integers(1, t.N))
            b = a + int(t.N * 10 ** rng.uniform(-5, -0.5))
            jobs.append(("q", t, a, b, int(t.n)))
        else:
            kind = int(rng.integers(0, 3))
            n = int(np.exp(rng.uniform(0, np.log(3 * 10**5))))
            N = int(np.exp(rng.uniform(np.log(max(n, 2)), np.log(2**56)))) if kind != 1 else \
                int(np.exp(rng.uniform(0, np.log(2**50))))
            N = max(N, n) if kind != 1 else max(N, 1)
            jobs.append(("s", n, N, 5000 + i, int(rng.choice([256, 4096])), kind))
    server = rs.Server(ctx, arena_bytes=64 << 20, lanes=4)
    own = {}   # jobs with their own output tensors
    tickets = []
    for idx, j in enumerate(jobs):
        use_own = idx % 3 == 0
        if j[0] == "s":
            _, n, N, seed, n0, kind = j
            out = torch.empty(max(n, 1), dtype=torch.int64, device="cuda") if use_own else None
            job = rs.sample_job(n, N, seed, n0, kind, out)
        else:
            _, t, a, b, cap = j
            out = torch.empty(cap, dtype=torch.int64, device="cuda") if use_own else None
            job = rs.query_job(t, a, b, cap, out)
        tk = server.submit(job)
        tickets.append(tk)
        if out is not None:
            own[tk] = out
        if idx % 40 == 39:
            time.sleep(0.002)   # let some groups start before the next arrivals
    results = {}

    def keep(r):
        vals = _values(rs, r) if r.status == rs.RS_OK else None
        results[r.ticket] = (r.status, r.count, vals)
        if r.ticket not in own:
            server.release(r.ticket)

    _drain(rs, server, tickets, on_result=keep)
    stats = server.stats()
    assert stats["completed"] == len(jobs)
    assert stats["groups"] >= 2
    assert stats["arena_bytes_in_use"] == 0
    for tk, j in zip(tickets, jobs):
        st, cnt, vals = results[tk]
        if j[0] == "s":
            _, n, N, seed, n0, kind = j
            assert st == rs.RS_OK and cnt == n, (j, st)
            want = oracle.sample(n, N, seed, n0, kind) if n <= 20000 else _solo(rs, ctx, n, N, seed, n0, kind)
            assert np.array_equal(vals, want), j
        else:
            _, t, a, b, cap = j
            rc, c2, want = _solo_query(rs, t, a, b, cap)
            assert st == rc == rs.RS_OK and cnt == c2, (j, st, rc)
            assert np.array_equal(vals, want), j
    server.close()
    for t in trees:
        t.close()


def test_jobs_start_while_a_group_runs(rs, ctx):
    """A long job goes out first; jobs submitted right after it start (on
    other lanes) before it finishes."""
    server = rs.Server(ctx, arena_bytes=1 << 20, lanes=4)
    big = torch.empty(5 * 10**8, dtype=torch.int64, device="cuda")
    t_big = server.submit(rs.sample_job(5 * 10**8, 2**50, 1, 4096, 0, big))
    time.sleep(0.001)   # the worker issues it alone; it runs for several milliseconds
    small = [server.submit(rs.sample_job(1000, 10**9, 100 + i, 4096, 0)) for i in range(16)]
    res = _drain(rs, server, [t_big] + small, on_result=lambda r: None)
    rb = res[t_big]
    assert rb.status == rs.RS_OK
    overlapped = [res[t] for t in small if rb.launch_ms < res[t].launch_ms < rb.done_ms]
    assert overlapped, [(res[t].launch_ms, rb.launch_ms, rb.done_ms) for t in small]
    for t in small:
        assert res[t].status == rs.RS_OK
        server.release(t)
    server.release(t_big)
    server.close()


def test_admission_by_memory(rs, ctx, oracle):
    arena = 2 << 20
    server = rs.Server(ctx, arena_bytes=arena, lanes=2)
    specs = [(60000, 10**9, 700 + i, 4096, i % 3) for i in range(30)]
    tickets = [server.submit(rs.sample_job(*s)) for s in specs]
    ok = {}

    def check(r):
        i = tickets.index(r.ticket)
        assert r.status == rs.RS_OK
        ok[i] = np.array_equal(_values(rs, r), oracle.sample(*specs[i][:4], kind=specs[i][4]))
        server.release(r.ticket)

    _drain(rs, server, tickets, on_result=check)
    assert all(ok.values()) and len(ok) == len(specs)
    stats = server.stats()
    assert 0 < stats["peak_arena_bytes"] <= arena
    assert stats["arena_bytes_in_use"] == 0
    # a job larger than the arena, a bad one, an empty one: completed at once
    t1 = server.submit(rs.sample_job(10**6, 10**9, 1, 4096, 0))
    t2 = server.submit(rs.sample_job(11, 10, 1, 4096, 0))
    t3 = server.submit(rs.sample_job(0, 10, 1, 4096, 0))
    res = _drain(rs, server, [t1, t2, t3])
    assert res[t1].status == rs.RS_ECAPACITY
    assert res[t2].status == rs.RS_EINVAL
    assert res[t3].status == rs.RS_OK and res[t3].count == 0
    for t in (t1, t2, t3):
        server.release(t)
    with pytest.raises(rs.RSError):
        server.release(t1)
    server.close()
