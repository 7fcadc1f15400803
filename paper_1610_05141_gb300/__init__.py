"""GB300 divide-and-conquer random sampler: thin Python binding of include/rs.h.

Every function here only marshals arguments (torch tensors -> device
pointers, the current torch stream -> cudaStream_t) and calls the C ABI of
_build/librs_gb300.so; all sampling runs in the library's CUDA kernels.
There is no fallback: importing fails loudly if the library is missing.
Build it with ``python -m paper_1610_05141_gb300.build`` (or
``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librs_gb300.so")

RS_OK, RS_EINVAL, RS_ECAPACITY, RS_ENOMEM, RS_ECUDA, RS_ETIMEOUT, RS_EITER = range(7)
RS_KIND_H, RS_KIND_WR, RS_KIND_B = 0, 1, 2


class RSError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {code} ({strerror(code) if _lib else code})")


RS_OP_SAMPLE, RS_OP_QUERY = 0, 1


class Job(ctypes.Structure):
    """rs_job."""
    _fields_ = [("op", ctypes.c_uint32), ("kind", ctypes.c_uint32), ("n", ctypes.c_uint64),
                ("N", ctypes.c_uint64), ("seed", ctypes.c_uint64), ("n0", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("tree", ctypes.c_void_p), ("a", ctypes.c_uint64),
                ("b", ctypes.c_uint64), ("cap", ctypes.c_uint64), ("out_dev", ctypes.c_void_p)]


class Result(ctypes.Structure):
    """rs_result."""
    _fields_ = [("ticket", ctypes.c_uint64), ("status", ctypes.c_int32), ("reserved", ctypes.c_uint32),
                ("count", ctypes.c_uint64), ("out_dev", ctypes.c_void_p), ("submit_ms", ctypes.c_double),
                ("launch_ms", ctypes.c_double), ("done_ms", ctypes.c_double)]


class ServerConfig(ctypes.Structure):
    """rs_server_config."""
    _fields_ = [("arena_bytes", ctypes.c_uint64), ("max_inflight", ctypes.c_uint32), ("lanes", ctypes.c_uint32),
                ("max_group", ctypes.c_uint32), ("reserved", ctypes.c_uint32), ("lane_bytes", ctypes.c_uint64)]


class ServerStats(ctypes.Structure):
    """rs_server_stats."""
    _fields_ = [(k, ctypes.c_uint64) for k in ("submitted", "completed", "groups", "launches", "max_group_seen",
                                               "peak_inflight", "peak_arena_bytes", "arena_bytes_in_use")]


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads the library (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"sampler library not built: {path} is missing "
                           "(run python -m paper_1610_05141_gb300.build)")
    lib = ctypes.CDLL(path)
    u64, u32, i32, vp, dbl = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_void_p, ctypes.c_double
    sig = {
        "rs_create": (i32, [ctypes.POINTER(vp), i32]),
        "rs_destroy": (i32, [vp]),
        "rs_plan": (i32, [u64, u64, u32, ctypes.POINTER(i32)]),
        "rs_sample": (i32, [vp, u64, u64, u64, u32, vp, vp]),
        "rs_sample_with_replacement": (i32, [vp, u64, u64, u64, u32, vp, vp]),
        "rs_sample_b": (i32, [vp, u64, u64, u64, u32, vp, vp]),
        "rs_split_tree": (i32, [vp, u64, u64, u64, u32, i32, vp, u64, vp]),
        "rs_bernoulli": (i32, [vp, dbl, u64, u64, u32, u64, u64, vp, u64, ctypes.POINTER(u64), vp]),
        "rs_sync": (i32, [vp, vp]),
        "rs_strerror": (ctypes.c_char_p, [i32]),
        "rs_set_leaf_capacity": (i32, [vp, u32]),
        "rs_set_exact_deviates": (i32, [vp, i32]),
        "rs_set_iteration_caps": (i32, [u64, u64, u64, u64]),
        "rs_set_profiling": (i32, [vp, i32]),
        "rs_phase_totals": (i32, [vp, ctypes.POINTER(dbl), ctypes.POINTER(dbl), ctypes.POINTER(u64)]),
        "rs_launch_count": (i32, [vp, ctypes.POINTER(u64)]),
        "rs_set_pipeline": (i32, [vp, i32, i32]),
        "rs_set_bernoulli_staging": (i32, [vp, u64, u64]),
        "rs_bernoulli_size": (i32, [vp, dbl, u64, u64, ctypes.POINTER(u64), vp]),
        "rs_bernoulli_by_size": (i32, [vp, dbl, u64, u64, u32, u64, u64, vp, u64, ctypes.POINTER(u64),
                                       ctypes.POINTER(u64), vp]),
        "rs_union_key": (u64, [u64, u32]),
        "rs_points": (i32, [vp, u32, vp, u64, u64, u32, vp, vp]),
        "rs_peel_create": (i32, [vp, u64, u64, u64, u32, u32, ctypes.POINTER(vp)]),
        "rs_peel_next": (i32, [vp, vp, u64, ctypes.POINTER(u64), ctypes.POINTER(u32), vp]),
        "rs_peel_state": (i32, [vp, ctypes.POINTER(u64), ctypes.POINTER(u64), ctypes.POINTER(u64)]),
        "rs_peel_destroy": (i32, [vp]),
        "rs_union_counts": (i32, [vp, vp, u32, u64, u64, vp, vp]),
        "rs_union_sample": (i32, [vp, vp, u32, u64, u64, u32, vp, vp, vp]),
        "rs_sample_to_host": (i32, [vp, i32, u64, u64, u64, u32, vp, vp, vp]),
        "rs_sample_static": (i32, [u64, u64, u64, u32, vp, vp]),
        "rs_batch_plan": (i32, [vp, vp, u32, ctypes.POINTER(vp)]),
        "rs_batch_run": (i32, [vp, vp, vp, vp]),
        "rs_batch_tune": (i32, [vp, vp, vp, vp]),
        "rs_batch_launch_count": (i32, [vp, ctypes.POINTER(u64)]),
        "rs_batch_set_leaf_launch": (i32, [vp, i32, i32, i32]),
        "rs_batch_destroy": (i32, [vp]),
        "rs_batch": (i32, [vp, vp, u32, vp, vp, vp]),
        "rs_tree_create": (i32, [vp, u64, u64, u64, u32, i32, vp, ctypes.POINTER(vp)]),
        "rs_tree_query": (i32, [vp, u64, u64, vp, u64, ctypes.POINTER(u64), vp]),
        "rs_tree_info": (i32, [vp, ctypes.POINTER(i32), ctypes.POINTER(u64)]),
        "rs_tree_destroy": (i32, [vp]),
        "rs_server_create": (i32, [vp, ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]),
        "rs_server_submit": (i32, [vp, ctypes.POINTER(Job), ctypes.POINTER(u64)]),
        "rs_server_poll": (i32, [vp, ctypes.POINTER(Result), u32, ctypes.POINTER(u32), u32]),
        "rs_server_release": (i32, [vp, u64]),
        "rs_server_stats_get": (i32, [vp, ctypes.POINTER(ServerStats)]),
        "rs_server_fail_next_plans": (i32, [vp, u32]),
        "rs_server_destroy": (i32, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def strerror(code: int) -> str:
    return load().rs_strerror(code).decode()


def _ptr(t) -> int:
    """Device pointer of a tensor (or an int address, or None)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(rc: int, where: str) -> int:
    if rc != RS_OK:
        raise RSError(rc, where)
    return rc


class Context:
    """Owns an rs_ctx (scratch memory and status word on one device)."""

    def __init__(self, device: int = 0):
        h = ctypes.c_void_p()
        _check(load().rs_create(ctypes.byref(h), device), "rs_create")
        self.handle = h
        self.device = device

    def close(self):
        if self.handle:
            load().rs_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rs_create(device: int = 0) -> Context:
    return Context(device)


def rs_destroy(ctx: Context) -> None:
    ctx.close()


def rs_plan(n: int, N: int, n0: int) -> int:
    d = ctypes.c_int(0)
    _check(load().rs_plan(n, N, n0, ctypes.byref(d)), "rs_plan")
    return d.value


def rs_sample(ctx: Context, n, N, seed, n0, out, stream=None, check=True) -> int:
    rc = load().rs_sample(ctx.handle, n, N, seed, n0, _ptr(out), _stream(stream))
    return _check(rc, "rs_sample") if check else rc


def rs_sample_with_replacement(ctx: Context, n, N, seed, n0, out, stream=None, check=True) -> int:
    rc = load().rs_sample_with_replacement(ctx.handle, n, N, seed, n0, _ptr(out), _stream(stream))
    return _check(rc, "rs_sample_with_replacement") if check else rc


def rs_sample_b(ctx: Context, n, N, seed, n0, out, stream=None, check=True) -> int:
    rc = load().rs_sample_b(ctx.handle, n, N, seed, n0, _ptr(out), _stream(stream))
    return _check(rc, "rs_sample_b") if check else rc


def rs_sample_to_host(ctx: Context, kind, n, N, seed, n0, out, out_host, stream=None, check=True) -> int:
    """out_host: a pinned torch CPU tensor (or a host address)."""
    rc = load().rs_sample_to_host(ctx.handle, kind, n, N, seed, n0, _ptr(out), _ptr(out_host), _stream(stream))
    return _check(rc, "rs_sample_to_host") if check else rc


def rs_split_tree(ctx: Context, n, N, seed, n0, kind, recs, max_leaves, stream=None, check=True) -> int:
    rc = load().rs_split_tree(ctx.handle, n, N, seed, n0, kind, _ptr(recs), max_leaves, _stream(stream))
    return _check(rc, "rs_split_tree") if check else rc


def rs_bernoulli(ctx: Context, p, N, seed, n0, a, b, out, cap, stream=None, check=True):
    """Returns (rc, count)."""
    cnt = ctypes.c_uint64(0)
    rc = load().rs_bernoulli(ctx.handle, float(p), N, seed, n0, a, b, _ptr(out), cap, ctypes.byref(cnt),
                             _stream(stream))
    if check and rc != RS_OK:
        raise RSError(rc, "rs_bernoulli")
    return rc, cnt.value


def rs_bernoulli_size(ctx: Context, p, N, seed, stream=None) -> int:
    """BIN(N, p) size of the Bernoulli sample drawn by its size."""
    cnt = ctypes.c_uint64(0)
    _check(load().rs_bernoulli_size(ctx.handle, float(p), N, seed, ctypes.byref(cnt), _stream(stream)),
           "rs_bernoulli_size")
    return cnt.value


def rs_bernoulli_by_size(ctx: Context, p, N, seed, n0, a, b, out, cap, stream=None, check=True):
    """Returns (rc, count in [a, b), total size)."""
    cnt, tot = ctypes.c_uint64(0), ctypes.c_uint64(0)
    rc = load().rs_bernoulli_by_size(ctx.handle, float(p), N, seed, n0, a, b, _ptr(out), cap, ctypes.byref(cnt),
                                     ctypes.byref(tot), _stream(stream))
    if check and rc != RS_OK:
        raise RSError(rc, "rs_bernoulli_by_size")
    return rc, cnt.value, tot.value


def rs_union_key(seed, i) -> int:
    return int(load().rs_union_key(seed, i))


def _segments(L):
    import numpy as np
    L = np.ascontiguousarray(L, dtype=np.uint64)
    return L, np.zeros(max(len(L), 1), dtype=np.uint64)


def rs_union_counts(ctx: Context, L, n, seed, stream=None):
    """Samples per segment of a sample of n from the union of segments of sizes L."""
    L, counts = _segments(L)
    _check(load().rs_union_counts(ctx.handle, L.ctypes.data, len(L), n, seed, counts.ctypes.data, _stream(stream)),
           "rs_union_counts")
    return counts[: len(L)]


def rs_union_sample(ctx: Context, L, n, seed, n0, out, stream=None):
    """Writes the union's sample (segment after segment, positions within the
    segment) to out[0..n); returns the counts per segment."""
    L, counts = _segments(L)
    _check(load().rs_union_sample(ctx.handle, L.ctypes.data, len(L), n, seed, n0, _ptr(out), counts.ctypes.data,
                                  _stream(stream)), "rs_union_sample")
    return counts[: len(L)]


def rs_points(ctx: Context, E, n, seed, n0, out, stream=None):
    """n points uniform in the box [0, E_0) x ... into out (n * d int64, point-major)."""
    import numpy as np
    E = np.ascontiguousarray(E, dtype=np.uint64)
    _check(load().rs_points(ctx.handle, len(E), E.ctypes.data, n, seed, n0, _ptr(out), _stream(stream)), "rs_points")


class Peel:
    """Iterator over a sample in increasing order, batch by batch (rs_peel_*)."""

    def __init__(self, handle):
        self.handle = handle

    def next(self, out, cap, stream=None, check=True):
        """Returns (rc, values written, batches made)."""
        cnt, nb = ctypes.c_uint64(0), ctypes.c_uint32(0)
        rc = load().rs_peel_next(self.handle, _ptr(out), cap, ctypes.byref(cnt), ctypes.byref(nb), _stream(stream))
        if check and rc != RS_OK:
            raise RSError(rc, "rs_peel_next")
        return rc, cnt.value, nb.value

    def state(self):
        a, b, c = ctypes.c_uint64(0), ctypes.c_uint64(0), ctypes.c_uint64(0)
        _check(load().rs_peel_state(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "rs_peel_state")
        return a.value, b.value, c.value

    def close(self):
        if self.handle:
            load().rs_peel_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rs_peel_create(ctx: Context, n, N, seed, n0, max_batches=256) -> Peel:
    h = ctypes.c_void_p()
    _check(load().rs_peel_create(ctx.handle, n, N, seed, n0, max_batches, ctypes.byref(h)), "rs_peel_create")
    return Peel(h.value)


def rs_sync(ctx: Context, stream=None) -> int:
    return load().rs_sync(ctx.handle, _stream(stream))


def rs_strerror(code: int) -> str:
    return strerror(code)


def rs_set_leaf_capacity(ctx: Context, cap: int) -> int:
    return _check(load().rs_set_leaf_capacity(ctx.handle, cap), "rs_set_leaf_capacity")


def rs_set_exact_deviates(ctx: Context, on: bool) -> int:
    return _check(load().rs_set_exact_deviates(ctx.handle, 1 if on else 0), "rs_set_exact_deviates")


def rs_set_iteration_caps(rou_trials=None, inv_restarts=None, stream_blocks=None, b_attempts=None) -> int:
    """Testing knob (current device, process-wide): None keeps a default."""
    keep = (1 << 64) - 1
    args = [keep if v is None else int(v) for v in (rou_trials, inv_restarts, stream_blocks, b_attempts)]
    return _check(load().rs_set_iteration_caps(*args), "rs_set_iteration_caps")


def rs_set_profiling(ctx: Context, on: bool) -> int:
    return _check(load().rs_set_profiling(ctx.handle, 1 if on else 0), "rs_set_profiling")


def rs_phase_totals(ctx: Context):
    """(tree_ms, leaf_ms, calls) summed over the profiled sampling calls."""
    t, l, c = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_uint64(0)
    _check(load().rs_phase_totals(ctx.handle, ctypes.byref(t), ctypes.byref(l), ctypes.byref(c)), "rs_phase_totals")
    return t.value, l.value, c.value


def rs_set_bernoulli_staging(ctx: Context, max_bytes: int = 16 << 30, slots_per_chunk: int = 0) -> int:
    return _check(load().rs_set_bernoulli_staging(ctx.handle, max_bytes, slots_per_chunk),
                  "rs_set_bernoulli_staging")


def rs_set_pipeline(ctx: Context, log2_parts: int, leaf_blocks_per_sm: int = 3) -> int:
    return _check(load().rs_set_pipeline(ctx.handle, log2_parts, leaf_blocks_per_sm), "rs_set_pipeline")


def rs_launch_count(ctx: Context) -> int:
    c = ctypes.c_uint64(0)
    _check(load().rs_launch_count(ctx.handle, ctypes.byref(c)), "rs_launch_count")
    return c.value


def rs_sample_static(n, N, seed, n0, out, stream=None) -> int:
    """rs_sample without device allocation (static scratch); returns the
    call's device status after waiting for the stream."""
    return load().rs_sample_static(n, N, seed, n0, _ptr(out), _stream(stream))


REQUEST_DTYPE = [("n", "<u8"), ("N", "<u8"), ("seed", "<u8"), ("out_off", "<u8"), ("n0", "<u4"), ("kind", "<u4")]


def requests_array(n, N, seed, out_off, n0, kind):
    """rs_request records (a numpy structured array with the C layout)."""
    import numpy as np
    a = np.zeros(len(n), dtype=np.dtype(REQUEST_DTYPE))
    a["n"], a["N"], a["seed"], a["out_off"] = n, N, seed, out_off
    a["n0"], a["kind"] = n0, kind
    return a


class BatchPlan:
    """Owns an rs_batch plan."""

    def __init__(self, ctx: Context, reqs):
        h = ctypes.c_void_p()
        _check(load().rs_batch_plan(ctx.handle, reqs.ctypes.data, len(reqs), ctypes.byref(h)), "rs_batch_plan")
        self.handle = h
        self.ctx = ctx   # the context must outlive the plan

    def close(self):
        if self.handle:
            load().rs_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rs_batch_plan(ctx: Context, reqs) -> BatchPlan:
    return BatchPlan(ctx, reqs)


def rs_batch_run(plan: BatchPlan, out_pool, status, stream=None) -> int:
    return _check(load().rs_batch_run(plan.handle, _ptr(out_pool), _ptr(status), _stream(stream)), "rs_batch_run")


def rs_batch_tune(plan: BatchPlan, out_pool, status, stream=None) -> int:
    return _check(load().rs_batch_tune(plan.handle, _ptr(out_pool), _ptr(status), _stream(stream)), "rs_batch_tune")


def rs_batch_set_leaf_launch(plan: BatchPlan, small_threads=0, large_threads=0, blocks_per_sm=0) -> int:
    return _check(load().rs_batch_set_leaf_launch(plan.handle, small_threads, large_threads, blocks_per_sm),
                  "rs_batch_set_leaf_launch")


def rs_batch_launch_count(plan: BatchPlan) -> int:
    c = ctypes.c_uint64(0)
    _check(load().rs_batch_launch_count(plan.handle, ctypes.byref(c)), "rs_batch_launch_count")
    return c.value


def rs_batch(ctx: Context, reqs_dev, R, out_pool, status, stream=None) -> int:
    return _check(load().rs_batch(ctx.handle, _ptr(reqs_dev), R, _ptr(out_pool), _ptr(status), _stream(stream)),
                  "rs_batch")


class Tree:
    """Owns an rs_tree (the resident leaf records of one sample's split tree)."""

    def __init__(self, ctx: Context, n, N, seed, n0, kind=RS_KIND_H, stream=None):
        h = ctypes.c_void_p()
        _check(load().rs_tree_create(ctx.handle, n, N, seed, n0, kind, _stream(stream), ctypes.byref(h)),
               "rs_tree_create")
        self.handle = h
        self.ctx = ctx   # the context must outlive the tree
        self.n, self.N, self.seed, self.n0, self.kind = n, N, seed, n0, kind

    def close(self):
        if self.handle:
            load().rs_tree_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rs_tree_create(ctx: Context, n, N, seed, n0, kind=RS_KIND_H, stream=None) -> Tree:
    return Tree(ctx, n, N, seed, n0, kind, stream)


def rs_tree_destroy(tree: Tree) -> None:
    tree.close()


def rs_tree_query(tree: Tree, a, b, out, cap, stream=None, check=True):
    """Returns (rc, count)."""
    cnt = ctypes.c_uint64(0)
    rc = load().rs_tree_query(tree.handle, a, b, _ptr(out), cap, ctypes.byref(cnt), _stream(stream))
    if check and rc != RS_OK:
        raise RSError(rc, "rs_tree_query")
    return rc, cnt.value


def rs_tree_info(tree: Tree):
    """(depth, largest leaf count)."""
    d, m = ctypes.c_int(0), ctypes.c_uint64(0)
    _check(load().rs_tree_info(tree.handle, ctypes.byref(d), ctypes.byref(m)), "rs_tree_info")
    return d.value, m.value


def sample_job(n, N, seed, n0, kind=RS_KIND_H, out=None) -> Job:
    return Job(op=RS_OP_SAMPLE, kind=kind, n=n, N=N, seed=seed, n0=n0, out_dev=_ptr(out))


def query_job(tree: Tree, a, b, cap, out=None) -> Job:
    return Job(op=RS_OP_QUERY, tree=tree.handle, a=a, b=b, cap=cap, out_dev=_ptr(out))


class Server:
    """Owns an rs_server (worker thread, output arena, lanes)."""

    def __init__(self, ctx: Context, arena_bytes=1 << 30, max_inflight=0, lanes=0, max_group=0, lane_bytes=0):
        cfg = ServerConfig(arena_bytes=arena_bytes, max_inflight=max_inflight, lanes=lanes, max_group=max_group,
                           lane_bytes=lane_bytes)
        h = ctypes.c_void_p()
        _check(load().rs_server_create(ctx.handle, ctypes.byref(cfg), ctypes.byref(h)), "rs_server_create")
        self.handle = h
        self.ctx = ctx
        self._buf = (Result * 1024)()

    def submit(self, job: Job) -> int:
        t = ctypes.c_uint64(0)
        _check(load().rs_server_submit(self.handle, ctypes.byref(job), ctypes.byref(t)), "rs_server_submit")
        return t.value

    def poll(self, wait_us=0, max_results=1024):
        """Completed jobs' results (a list of Result copies)."""
        got = ctypes.c_uint32(0)
        n = min(max_results, len(self._buf))
        _check(load().rs_server_poll(self.handle, self._buf, n, ctypes.byref(got), wait_us), "rs_server_poll")
        out = []
        for i in range(got.value):
            r = Result()
            ctypes.pointer(r)[0] = self._buf[i]
            out.append(r)
        return out

    def release(self, ticket: int) -> None:
        _check(load().rs_server_release(self.handle, ticket), "rs_server_release")

    def fail_next_plans(self, count: int) -> None:
        """Testing knob: the next `count` group plans fail as if host memory ran out."""
        _check(load().rs_server_fail_next_plans(self.handle, count), "rs_server_fail_next_plans")

    def stats(self) -> dict:
        s = ServerStats()
        _check(load().rs_server_stats_get(self.handle, ctypes.byref(s)), "rs_server_stats_get")
        return {k: getattr(s, k) for k, _ in ServerStats._fields_}

    def close(self):
        if self.handle:
            load().rs_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rs_server_create(ctx: Context, **cfg) -> Server:
    return Server(ctx, **cfg)


class _DeviceArray:
    """__cuda_array_interface__ of n uint64 at a raw device address (read as int64)."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<i8", "data": (ptr, False), "version": 2}


def device_view(ptr: int, n: int):
    """A torch int64 tensor viewing n values at a device address (e.g. a
    server result in the arena); no copy."""
    import torch
    if n == 0:
        return torch.empty(0, dtype=torch.int64, device="cuda")
    return torch.as_tensor(_DeviceArray(ptr, n), device="cuda")
