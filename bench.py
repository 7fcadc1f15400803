#!/usr/bin/env python3
"""Benchmark: sorted sampling without replacement, n = 10^9 distinct values
from 1..2^50 (n0 = 4096: 2^18 leaves of 2^32 positions), on one GB300.

One step = one whole pass of the sampler: split tree (2^18 - 1 hypergeometric
deviates) + every leaf (selection, sort, write-out of 8 GB of uint64).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  `value` is samples/s over the device-timed steps
(output buffer resident; the 8 GB output exceeds the 129 MB L2, so no flush
is needed); `e2e` is the same through rs_sample_to_host, which also copies
each step's sample into pinned host memory (piece by piece while the next
pieces are made).  `batch` and `serve` measure the batched and served paths
against one call per request.  `roofline` relates the leaf kernel's algorithmic write
bytes (8 B per sample) per launch to its CUDA-event duration on its own
stream.  Under torchrun with N > 1, every rank runs an independent replica
(seed + rank) on its own GPU: the path does not shard.
`--impl reference` times the CPU oracle on a bounded sample of the same
workload (rank 0 only).
"""
import argparse
import hashlib
import re

import numpy as np
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_SAMPLES = 10**9
UNIVERSE = 2**50
N0 = 4096
SEED = 1
BYTES_PER_SAMPLE = 8
WORKLOAD = "sorted sampling without replacement: n=1e9 distinct uint64 from 1..2^50, n0=4096 (2^18 leaves)"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_PATH = os.path.join(ROOT, "profiles", "leaf_kernel_traffic.json")
LEAF_SOURCES = ["rs_leaf.cu", "rs_hash_leaf.cuh", "rs_big_leaf.cuh", "rs_leaf.cuh", "rs_block.cuh", "rs_rng.cuh",
                "rs_common.cuh", "rs_internal.h"]


def set_workload(n, log2N, n0=None):
    """Smaller cases of the same shape (used for ncu captures of a few GB)."""
    global N_SAMPLES, UNIVERSE, WORKLOAD, N0
    if n is None and log2N is None and n0 is None:
        return
    N_SAMPLES = n if n is not None else N_SAMPLES
    UNIVERSE = 2**log2N if log2N is not None else UNIVERSE
    N0 = n0 if n0 is not None else N0
    WORKLOAD = (f"sorted sampling without replacement: n={N_SAMPLES} distinct uint64 from 1..2^{UNIVERSE.bit_length() - 1}"
                f", n0={N0} (reduced case)")


def hbm_peak():
    try:
        with open(PEAKS_PATH) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _code_only(text):
    """Source text without comments and trailing blanks: the hash follows the code."""
    text = re.sub(rb"/\*.*?\*/", b"", text, flags=re.S)
    text = re.sub(rb"//[^\n]*", b"", text)
    return b"\n".join(line.rstrip() for line in text.split(b"\n") if line.strip())


def leaf_source_hash(read=None):
    """Hash of the leaf kernel's sources (code only, comments left out);
    read(name) -> bytes overrides reading the working tree."""
    h = hashlib.sha256()
    for name in LEAF_SOURCES:
        if read is None:
            with open(os.path.join(ROOT, "paper_1610_05141_gb300", "csrc", name), "rb") as f:
                data = f.read()
        else:
            data = read(name)
        h.update(_code_only(data))
    return h.hexdigest()[:16]


def leaf_traffic():
    """DRAM bytes per launch of the leaf kernel from the committed ncu
    summary, scaled to this workload, or None if the kernel changed since."""
    try:
        with open(TRAFFIC_PATH) as f:
            t = json.load(f)
    except Exception:
        return None
    if t.get("source_hash") != leaf_source_hash():
        return None
    return t["dram_bytes_per_sample"] * N_SAMPLES


class ClockSampler:
    """nvidia-smi clock/throttle samples every 50 ms while running."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0=None, t1=None):
        """Median SM clock and throttle reasons of the samples taken between
        the wall-clock times t0 and t1 (all samples if not given)."""
        import datetime
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) < 9:
                        continue
                    try:
                        ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                    except ValueError:
                        continue
                    if (t0 is None or ts >= t0) and (t1 is None or ts <= t1):
                        rows.append(parts)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples in the timed region"],
                    "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        mhz = []
        for r in rows:
            try:
                mhz.append(float(r[1]))
            except ValueError:
                pass
            for name, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        try:
            max_mhz = float(rows[0][2])
        except ValueError:
            max_mhz = None
        power = []
        for r in rows:
            try:
                power.append(float(r[3]))
            except ValueError:
                pass
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": max_mhz,
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max(power) if power else None}


def cpu_baseline(budget_s=15.0):
    """The oracle, as it stands, on one host core: the full split tree plus
    leaves in order until the time budget is spent."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    recs, D = oracle.tree(N_SAMPLES, UNIVERSE, SEED, N0, oracle.KIND_H)
    samples = 0
    leaves = 0
    while time.perf_counter() - t0 < budget_s and leaves < len(recs):
        samples += len(oracle.leaf(SEED, oracle.KIND_H, D, leaves, recs[leaves]))
        leaves += 1
    dt = time.perf_counter() - t0
    return {"value": samples / dt, "unit": "samples/s", "cores": 1, "kind": "oracle",
            "sample": f"full split tree (2^18 leaf records) + the first {leaves} leaves ({samples} samples) "
                      f"in {dt:.1f} s on one core"}


def _oracle_leaf_worker(job):
    """One host process of the leaf-parallel oracle run: the split tree, then
    the leaves w, w + P, w + 2P, ... until its time budget is spent."""
    w, P, budget_s = job
    import oracle
    recs, D = oracle.tree(N_SAMPLES, UNIVERSE, SEED, N0, oracle.KIND_H)
    t0 = time.perf_counter()
    samples, i = 0, w
    while time.perf_counter() - t0 < budget_s and i < len(recs):
        samples += len(oracle.leaf(SEED, oracle.KIND_H, D, i, recs[i]))
        i += P
    return samples, time.perf_counter() - t0


def cpu_baseline_parallel(budget_s=2.0):
    """The oracle's leaves spread over every host core (one process each,
    started by spawn), each process with its own copy of the split tree."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    P = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(P) as pool:
        res = pool.map(_oracle_leaf_worker, [(w, P, budget_s) for w in range(P)])
    samples = sum(r[0] for r in res)
    dt = max(r[1] for r in res)
    return {"value": samples / dt, "unit": "samples/s", "cores": P, "kind": "oracle",
            "sample": f"leaves i = w mod {P} on {P} processes for {dt:.1f} s each ({samples} samples), "
                      f"after each built the full split tree"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    # each step: the full split tree plus a slice of leaves, sized so that the
    # whole run stays within about two and a half minutes
    budget = 150.0 / max(1, args.steps + args.warmup)
    t0 = time.perf_counter()
    recs, D = oracle.tree(N_SAMPLES, UNIVERSE, SEED, N0, oracle.KIND_H)
    t_tree = time.perf_counter() - t0
    t0 = time.perf_counter()
    for i in range(50):
        oracle.leaf(SEED, oracle.KIND_H, D, i, recs[i])
    t_leaf = (time.perf_counter() - t0) / 50
    leaves_per_step = int(min(len(recs) - 1, 4000, max(20, (budget - t_tree) / t_leaf)))

    def step(k):
        t0 = time.perf_counter()
        r, d = oracle.tree(N_SAMPLES, UNIVERSE, SEED + k, N0, oracle.KIND_H)
        s = 0
        first = (k * leaves_per_step) % max(1, len(r) - leaves_per_step)
        for i in range(first, first + leaves_per_step):
            s += len(oracle.leaf(SEED + k, oracle.KIND_H, d, i, r[i]))
        return s, time.perf_counter() - t0

    for k in range(args.warmup):
        step(k)
    tot_s, tot_t = 0, 0.0
    for k in range(args.steps):
        s, t = step(args.warmup + k)
        tot_s += s
        tot_t += t
    value = tot_s / tot_t
    line = {"impl": "reference", "metric": "sorted samples/s", "value": value, "unit": "samples/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * tot_t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": N_SAMPLES, "N": UNIVERSE, "n0": N0},
            "cpu_baseline": {"value": value, "unit": "samples/s", "cores": 1, "kind": "oracle",
                             "sample": f"per step: full split tree + {leaves_per_step} leaves "
                                       f"(~{tot_s // max(args.steps, 1)} samples), one core"},
            "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_batch(rs, ctx, stream, args):
    """Batched requests (100k independent samples in one graph-replayed run)
    against one rs_sample launch per request on the same GPU and stream."""
    import torch
    from paper_1610_05141_gb300.workloads import batch_requests
    n, N, seeds, off, n0, total = batch_requests(R=args.batch_requests)
    kinds = np.zeros(len(n), dtype=np.uint32)
    arr = rs.requests_array(n, N, seeds, off, n0, kinds)
    t0 = time.perf_counter()
    plan = rs.rs_batch_plan(ctx, arr)
    plan_s = time.perf_counter() - t0
    pool = torch.empty(total, dtype=torch.int64, device="cuda")
    status = torch.empty(len(n), dtype=torch.int32, device="cuda")
    rs.rs_batch_run(plan, pool, status, stream)        # eager run
    rs.rs_batch_tune(plan, pool, status, stream)
    for _ in range(2):
        rs.rs_batch_run(plan, pool, status, stream)    # graph capture + replay
    stream.synchronize()
    if not bool((status == 0).all()):
        raise RuntimeError("batch request failed")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    runs = args.batch_runs
    e0.record(stream)
    for _ in range(runs):
        rs.rs_batch_run(plan, pool, status, stream)
    e1.record(stream)
    stream.synchronize()
    batch_ms = e0.elapsed_time(e1) / runs
    launches = rs.rs_batch_launch_count(plan)
    plan.close()
    del pool
    # unbatched: the first `m` requests, one call (and its launches) each
    m = min(args.unbatched_requests, len(n))
    outs = torch.empty(int(n[:m].sum()), dtype=torch.int64, device="cuda")
    for i in range(min(m, 50)):   # warm-up
        rs.rs_sample(ctx, int(n[i]), int(N[i]), int(seeds[i]), int(n0[i]), outs[int(off[i]):], stream)
    stream.synchronize()
    e0.record(stream)
    for i in range(m):
        rs.rs_sample(ctx, int(n[i]), int(N[i]), int(seeds[i]), int(n0[i]), outs[int(off[i]):], stream)
    e1.record(stream)
    stream.synchronize()
    single_ms = e0.elapsed_time(e1)
    # the same slice batched
    plan = rs.rs_batch_plan(ctx, rs.requests_array(n[:m], N[:m], seeds[:m], off[:m], n0[:m], kinds[:m]))
    st2 = torch.empty(m, dtype=torch.int32, device="cuda")
    for _ in range(3):
        rs.rs_batch_run(plan, outs, st2, stream)
    stream.synchronize()
    e0.record(stream)
    for _ in range(runs):
        rs.rs_batch_run(plan, outs, st2, stream)
    e1.record(stream)
    stream.synchronize()
    slice_ms = e0.elapsed_time(e1) / runs
    plan.close()
    return {
        "workload": f"{len(n)} requests, n log-uniform in [1,1e6), N log-uniform in [n,2^48], n0=4096, "
                    "PCG64 seed 20161017",
        "requests": len(n), "samples": total, "ms_per_run": batch_ms,
        "req_per_s": len(n) / (batch_ms / 1000), "samples_per_s": total / (batch_ms / 1000),
        "write_gbs": 8 * total / (batch_ms / 1000) / 1e9,
        "request_latency_ms": batch_ms,
        "request_latency_note": "a run is one graph replay: every request's values are complete when the run "
                                "ends, so each request's latency is the run's time (no per-request spread)",
        "kernel_launches_per_run": launches, "plan_s": plan_s,
        "unbatched": {"requests": m, "req_per_s": m / (single_ms / 1000),
                      "batched_same_requests_req_per_s": m / (slice_ms / 1000),
                      "speedup": single_ms / slice_ms},
    }


def run_rows(rs, ctx, stream, args):
    """The other rows of the method at their configurations' sizes: sampling
    with replacement (n = 1e9 from 2^40, binomial splits), Algorithm B as the
    base case (n = 1e9 from 2^50), and Bernoulli sampling of 2^36 positions
    with p = 1e-4 and 1e-2 (whole range in one call) and p = 0.5 (the whole
    range as 8 chunk-aligned windows of 2^33 positions into one reusable
    34 GB buffer: the whole output would be 275 GB).  Device-timed (CUDA
    events on the stream), a few steps each after one warm-up call."""
    import torch
    peak, _ = hbm_peak()
    out = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, steps):
        fn()
        stream.synchronize()
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1) / steps

    rows = set(args.rows.split(","))

    def want(name):
        return name in rows

    K = args.row_scale_log2   # profiling cases only: n and N of a5/a7 and N of a6 divided by 2^K
    n_rows = 10**9 >> K
    NB = 2**36 >> K
    buf = torch.empty(n_rows, dtype=torch.int64, device="cuda")
    for name, call, N, steps in (("a5_with_replacement", rs.rs_sample_with_replacement, 2**40 >> K, args.row_steps),
                                 ("a7_leaf_b", rs.rs_sample_b, 2**50 >> K, max(1, args.row_steps // 3))):
        if not want(name.split("_")[0]):
            continue
        rs.rs_set_profiling(ctx, True)
        ms = timed(lambda: call(ctx, n_rows, N, 3, N0, buf, stream), steps)
        tree_ms, leaf_ms, calls = rs.rs_phase_totals(ctx)
        rs.rs_set_profiling(ctx, False)
        if rs.rs_sync(ctx, stream) != rs.RS_OK:
            raise RuntimeError(f"{name} failed")
        leaf = leaf_ms / calls
        out[name] = {"workload": f"n={n_rows:.3g} from 1..2^{N.bit_length() - 1}, n0={N0}", "ms_per_step": ms,
                     "samples_per_s": n_rows / (ms / 1000),
                     "phases_ms": {"split_tree": tree_ms / calls, "leaves": leaf},
                     "leaf_write_gbs": 8 * n_rows / (leaf / 1000) / 1e9,
                     "leaf_frac_of_hbm": 8 * n_rows / (leaf / 1000) / 1e9 / peak}
    if want("a6"):
        bern = {}
        for p, windows, steps in ((1e-4, 1, args.row_steps), (1e-2, 1, args.row_steps), (0.5, 8, 2)):
            if windows > 1 and K:   # scaled profiling runs stop before the 34 GB buffer
                continue
            if windows > 1:   # p = 0.5: a 34 GB buffer reused by every window, and room to stage its positions
                del buf
                torch.cuda.empty_cache()
                buf = torch.empty((1 << 32) + (1 << 20), dtype=torch.int64, device="cuda")
                rs.rs_set_bernoulli_staging(ctx, 48 << 30)
            cap = buf.numel()
            width = NB // windows
            holder = {"rc": rs.RS_OK, "count": 0}

            def call_b():
                total = 0
                for w in range(windows):
                    rc, c = rs.rs_bernoulli(ctx, p, NB, 5, N0, w * width, (w + 1) * width, buf, cap, stream,
                                            check=False)
                    if rc != rs.RS_OK:
                        holder["rc"] = rc
                    total += c
                holder["count"] = total

            ms = timed(call_b, steps)
            if holder["rc"] != rs.RS_OK:
                raise RuntimeError(f"bernoulli p={p} failed: {holder['rc']}")
            cnt = holder["count"]
            bern[f"p={p:g}"] = {"positions": NB, "windows": windows, "emitted": cnt, "ms_per_call": ms,
                                "emitted_per_s": cnt / (ms / 1000), "positions_per_s": NB / (ms / 1000),
                                "write_gbs": 8 * cnt / (ms / 1000) / 1e9,
                                "note": "whole range: per window one walk with staged positions, the scan of the "
                                        "counts, the copy into place, and the count read back"}
        rs.rs_set_bernoulli_staging(ctx)
        out["a6_bernoulli"] = {"N": NB, "n0": N0, "by_p": bern}
    if want("f2"):
        if buf.numel() < (1 << 32):   # p = 0.5: windows of 2^32 expected values
            del buf
            torch.cuda.empty_cache()
            buf = torch.empty((1 << 32) + (1 << 20), dtype=torch.int64, device="cuda")
        # the next row (f2): Bernoulli sampling by its size (Sec. 4.7) -- the
        # BIN(N, p) size, then the sample without replacement of that size; p =
        # 0.5 as a resident split tree and 8 window queries into the same buffer
        cap = buf.numel()
        by_size = {}
        for p, windows, steps in ((1e-4, 1, args.row_steps), (1e-2, 1, args.row_steps), (0.5, 8, 2)):
            holder = {"count": 0}

            def call_s():
                if windows == 1:
                    rc, cnt, _ = rs.rs_bernoulli_by_size(ctx, p, 2**36, 5, N0, 0, 2**36, buf, cap, stream)
                    holder["count"] = cnt
                    return
                n = rs.rs_bernoulli_size(ctx, p, 2**36, 5, stream)
                tree = rs.rs_tree_create(ctx, n, 2**36, 5, N0, rs.RS_KIND_H, stream)
                width = 2**36 // windows
                total = 0
                for w in range(windows):
                    _, c = rs.rs_tree_query(tree, w * width + 1, (w + 1) * width + 1, buf, cap, stream)
                    total += c
                tree.close()
                holder["count"] = total

            ms = timed(call_s, steps)
            if rs.rs_sync(ctx, stream) != rs.RS_OK:
                raise RuntimeError(f"bernoulli by size p={p} failed")
            cnt = holder["count"]
            by_size[f"p={p:g}"] = {"positions": 2**36, "windows": windows, "emitted": cnt, "ms_per_call": ms,
                                   "emitted_per_s": cnt / (ms / 1000), "write_gbs": 8 * cnt / (ms / 1000) / 1e9,
                                   "note": "whole call: the size (read back), then rs_sample of that size, or the "
                                           "split tree and one range query per window"}
        out["f2_bernoulli_by_size"] = {"N": 2**36, "n0": N0, "by_p": by_size}
    if want("f3"):
        # the next row (f3): a sample of 1e8 from the union of 4096 segments of
        # uneven sizes (Sec. 4.3): the count tree, then the segments' samples as
        # one batch
        from paper_1610_05141_gb300.workloads import union_segments
        L = union_segments()
        n_u = 10**8
        ms_counts = timed(lambda: rs.rs_union_counts(ctx, L, n_u, 5, stream), args.row_steps)
        ms_union = timed(lambda: rs.rs_union_sample(ctx, L, n_u, 5, N0, buf, stream), args.row_steps)
        out["f3_union"] = {"workload": f"n=1e8 from the union of {len(L)} segments of sizes log-uniform in "
                                       f"2^20..2^40 (total {int(L.sum()):.3e}), n0={N0}",
                           "ms_per_call": ms_union, "samples_per_s": n_u / (ms_union / 1000),
                           "count_tree_ms": ms_counts,
                           "note": "whole call: sizes to the device, the count tree, counts read back, the "
                                   "segments' batch planned and run, statuses read back"}
    if want("f1"):
        # the next row (f1): online sorted sampling by peeling (Sec. 4.1), n = 1e7
        # from 2^50 in batches of about n0 = 4096 values
        n_p, N_p = 10**7, 2**50
        peel = {}
        for B in (1, 256):
            it = rs.rs_peel_create(ctx, n_p, N_p, 5, N0, B)
            calls, made, t0 = 0, 0, time.perf_counter()
            first = None
            while True:
                _, cnt, nb = it.next(buf, 1 << 21, stream)
                if first is None:
                    first = (time.perf_counter() - t0) * 1e3
                if nb == 0:
                    break
                calls += 1
                made += cnt
                if B == 1 and calls == 400:
                    break
            ms = (time.perf_counter() - t0) * 1e3
            it.close()
            peel[f"batches_per_call={B}"] = {"calls": calls, "values": made, "ms": ms, "ms_per_call": ms / calls,
                                            "first_call_ms": first, "values_per_s": made / (ms / 1000)}
        out["f1_peel"] = {"workload": f"n=1e7 from 1..2^50 in batches of about n0={N0}", "by_batches": peel,
                          "note": "host wall time of synchronous calls: the chain of hypergeometric deviates "
                                  "(one thread), the counts read back, one leaf launch for the call's batches"}
    if want("f4"):
        # the next row (f4): 1e8 points uniform in the square [0, 2^31)^2, with
        # replacement, by bisection (Sec. 4.6)
        n_pts = 10**8
        ms_pts = timed(lambda: rs.rs_points(ctx, [2**31, 2**31], n_pts, 5, N0, buf, stream), args.row_steps)
        if rs.rs_sync(ctx, stream) != rs.RS_OK:
            raise RuntimeError("points failed")
        out["f4_points"] = {"workload": f"n=1e8 points in [0, 2^31)^2 with replacement, n0={N0}",
                            "ms_per_call": ms_pts, "points_per_s": n_pts / (ms_pts / 1000),
                            "write_gbs": 16 * n_pts / (ms_pts / 1000) / 1e9,
                            "note": "whole call: box tree, leaf records and their largest volume and count (read "
                                    "back), leaf WR indices, decode to coordinates"}
    del buf
    return out


def _pct(x, q):
    return float(np.percentile(np.asarray(x, dtype=np.float64), q)) if len(x) else None


def run_serve(rs, ctx, stream, args):
    """Serving: a Poisson stream of sampling jobs (n log-uniform in
    [1e2, 1e8), N log-uniform in [n, 2^56]) and range queries (20%, 1e3..1e5
    expected hits) on resident trees, through the server's continuous
    batching with a 64 GB output arena.  Capacity = completion rate with the
    queue kept full; then open-loop runs at fractions of it give p50/p99
    latency (submit to completion, server clock).  The same jobs, one call
    each on one stream, give the unbatched rate."""
    import torch
    from paper_1610_05141_gb300.workloads import serve_jobs, serve_trees
    tspec = serve_trees()
    trees = [rs.rs_tree_create(ctx, n, N, seed, N0, rs.RS_KIND_H, stream) for (n, N, seed) in tspec]
    server = rs.Server(ctx, arena_bytes=args.serve_arena_gb << 30, max_inflight=4096, lanes=4, max_group=4096)

    def job(J, i):
        if J["op"][i] == 0:
            return rs.sample_job(int(J["n"][i]), int(J["N"][i]), int(J["seed"][i]), N0, rs.RS_KIND_H)
        return rs.query_job(trees[int(J["tree"][i])], int(J["a"][i]), int(J["b"][i]), int(J["cap"][i]))

    def finish(results, r, J=None, idx=None):
        results.append(r)
        if r.status != rs.RS_OK:
            raise RuntimeError(f"serve job failed: status {r.status}")
        server.release(r.ticket)

    def drain(results, want, timeout_s=120.0):
        t_end = time.time() + timeout_s
        while len(results) < want:
            if time.time() > t_end:
                raise RuntimeError("server did not drain")
            for r in server.poll(wait_us=2000):
                finish(results, r)

    def summarize(results, t_first, wall_s=None):
        lat = [r.done_ms - r.submit_ms for r in results]
        span_ms = max(r.done_ms for r in results) - t_first
        return {"jobs": len(results), "req_per_s": len(results) / (span_ms / 1000),
                "latency_ms": {"p50": _pct(lat, 50), "p99": _pct(lat, 99), "max": max(lat)},
                "queue_ms_p99": _pct([r.launch_ms - r.submit_ms for r in results], 99)}

    # warm-up (kernel attributes, lanes)
    W = serve_jobs(200, tspec, seed=4)
    res = []
    for i in range(200):
        server.submit(job(W, i))
    drain(res, 200)
    # capacity: everything queued at once
    C = serve_jobs(args.serve_capacity_jobs, tspec, seed=5)
    res = []
    st0 = server.stats()
    for i in range(len(C["op"])):
        server.submit(job(C, i))
    drain(res, len(C["op"]))
    t_first = min(r.submit_ms for r in res)
    cap = summarize(res, t_first)
    st1 = server.stats()
    capacity = cap["req_per_s"]
    samples_cap = int(sum(r.count for r in res))
    cap["samples_per_s"] = samples_cap / ((max(r.done_ms for r in res) - t_first) / 1000)
    cap["groups"] = st1["groups"] - st0["groups"]
    cap["kernel_launches"] = st1["launches"] - st0["launches"]
    # open loop at fractions of capacity
    loads = {}
    for k, frac in enumerate((0.25, 0.5, 0.8)):
        lam = frac * capacity
        count = max(50, int(lam * args.serve_seconds))
        J = serve_jobs(count, tspec, seed=50 + k)
        arrivals = np.cumsum(np.random.Generator(np.random.PCG64(500 + k)).exponential(1.0 / lam, count))
        res = []
        lag = []
        t0 = time.perf_counter()
        i = 0
        while i < count:
            now = time.perf_counter() - t0
            if now >= arrivals[i]:
                server.submit(job(J, i))
                lag.append(1000 * (now - arrivals[i]))
                i += 1
                continue
            for r in server.poll(wait_us=0):
                finish(res, r)
        drain(res, count)
        t_first = min(r.submit_ms for r in res)
        out = summarize(res, t_first)
        out["offered_req_per_s"] = lam
        out["submit_lag_ms_p99"] = _pct(lag, 99)
        loads[str(frac)] = out
    stats = server.stats()
    # exactness spot check: jobs of the mix (own buffers) against solo calls
    chk = serve_jobs(64, tspec, seed=6, log10_n_max=6.0)
    bufs, tks = {}, []
    for i in range(64):
        sz = int(chk["n"][i]) if chk["op"][i] == 0 else int(chk["cap"][i])
        bufs[i] = torch.empty(max(sz, 1), dtype=torch.int64, device="cuda")
        if chk["op"][i] == 0:
            tks.append(server.submit(rs.sample_job(int(chk["n"][i]), int(chk["N"][i]), int(chk["seed"][i]), N0,
                                                   rs.RS_KIND_H, bufs[i])))
        else:
            tks.append(server.submit(rs.query_job(trees[int(chk["tree"][i])], int(chk["a"][i]), int(chk["b"][i]),
                                                  int(chk["cap"][i]), bufs[i])))
    res = []
    drain(res, 64)
    counts = {r.ticket: r.count for r in res}
    server.close()
    exact = 0
    for i in range(64):
        cnt = counts[tks[i]]
        solo = torch.empty_like(bufs[i])
        if chk["op"][i] == 0:
            rs.rs_sample(ctx, int(chk["n"][i]), int(chk["N"][i]), int(chk["seed"][i]), N0, solo, stream)
            stream.synchronize()
        else:
            _, c2 = rs.rs_tree_query(trees[int(chk["tree"][i])], int(chk["a"][i]), int(chk["b"][i]), solo,
                                     int(chk["cap"][i]), stream)
            if c2 != cnt:
                raise RuntimeError("served query count differs from the solo call")
        if not torch.equal(solo[:cnt], bufs[i][:cnt]):
            raise RuntimeError(f"served job {i} differs from its solo call")
        exact += 1
    # unbatched: the capacity mix's first jobs, one call each on one stream
    m = min(args.serve_unbatched_jobs, len(C["op"]))
    big = torch.empty(int(max(C["n"][:m].max(), C["cap"][:m].max())), dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(m):
        if C["op"][i] == 0:
            rs.rs_sample(ctx, int(C["n"][i]), int(C["N"][i]), int(C["seed"][i]), N0, big, stream)
        else:
            rs.rs_tree_query(trees[int(C["tree"][i])], int(C["a"][i]), int(C["b"][i]), big, int(C["cap"][i]), stream)
    stream.synchronize()
    single_s = time.perf_counter() - t0
    if rs.rs_sync(ctx, stream) != rs.RS_OK:
        raise RuntimeError("unbatched serve jobs failed")
    del big
    for t in trees:
        t.close()
    return {
        "workload": "Poisson arrivals; 80% sampling jobs n log-uniform [1e2,1e8), N log-uniform [n,2^56], "
                    "20% range queries on 8 resident trees (n=1e8, N log-uniform [1e8,2^56]) with 1e3..1e5 "
                    f"expected hits; arena {args.serve_arena_gb} GB, 4 lanes, PCG64 seeds 4-6, 50-52",
        "capacity": cap, "loads": loads,
        "groups": stats["groups"], "max_group": stats["max_group_seen"], "peak_inflight": stats["peak_inflight"],
        "peak_arena_gb": stats["peak_arena_bytes"] / 2**30,
        "exact_vs_solo": f"{exact}/64 jobs bit-identical to their single calls",
        "unbatched": {"jobs": m, "req_per_s": m / single_s,
                      "note": "same jobs, one rs_sample / rs_tree_query call each, one stream"},
        "speedup_vs_unbatched": capacity / (m / single_s),
    }


def combine_over_ranks(dist, ms_per_step, e2e_step, launches, device):
    """Replicas: the job's step time is the slowest rank's (max), its launch
    count the sum over ranks."""
    import torch
    t = torch.tensor([ms_per_step, e2e_step], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    lt = torch.tensor([launches], dtype=torch.int64, device=device)
    dist.all_reduce(lt)
    ms, e2e = t.tolist()
    return ms, e2e, int(lt.item())


def run_ours(args):
    import torch
    import paper_1610_05141_gb300 as rs
    from paper_1610_05141_gb300 import build as rs_build

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or world == 1:
        rs_build.build()
    if dist is not None:
        dist.barrier()
    rs.load()
    ctx = rs.rs_create(local)
    if args.pipeline is not None:
        log2_parts, blocks = (int(x) for x in args.pipeline.split(","))
        rs.rs_set_pipeline(ctx, log2_parts, blocks)
    stream = torch.cuda.Stream()
    out = torch.empty(N_SAMPLES, dtype=torch.int64, device="cuda")
    seed = SEED + rank

    def barrier():
        if dist is not None:
            dist.barrier()

    with ClockSampler(local) as clocks, torch.cuda.stream(stream):
        for _ in range(args.warmup):
            rs.rs_sample(ctx, N_SAMPLES, UNIVERSE, seed, N0, out, stream)
        stream.synchronize()
        rc = rs.rs_sync(ctx, stream)
        if rc != rs.RS_OK:
            raise RuntimeError(f"device status {rc}: {rs.strerror(rc)}")
        # device-timed steps
        rs.rs_set_profiling(ctx, True)
        launches0 = rs.rs_launch_count(ctx)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        wall0 = time.time()
        ev0.record(stream)
        for _ in range(args.steps):
            rs.rs_sample(ctx, N_SAMPLES, UNIVERSE, seed, N0, out, stream)
        ev1.record(stream)
        stream.synchronize()
        torch.cuda.synchronize()
        wall1 = time.time()
        barrier()
        launches = rs.rs_launch_count(ctx) - launches0
        ms_total = ev0.elapsed_time(ev1)
        tree_ms, leaf_ms, calls = rs.rs_phase_totals(ctx)
        rs.rs_set_profiling(ctx, False)
        rc = rs.rs_sync(ctx, stream)
        if rc != rs.RS_OK:
            raise RuntimeError(f"device status {rc}: {rs.strerror(rc)}")
        # end to end: sample + copy of the sample into pinned host memory
        e2e_steps = max(1, min(args.steps, 10))
        host = torch.empty(N_SAMPLES, dtype=torch.int64, pin_memory=True)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(e2e_steps):   # the sample goes to host memory piece by piece while it is made
            rs.rs_sample_to_host(ctx, rs.RS_KIND_H, N_SAMPLES, UNIVERSE, seed, N0, out, host, stream)
        e1.record(stream)
        stream.synchronize()
        barrier()
        e2e_ms = e0.elapsed_time(e1) / e2e_steps
        e2e_wall_ms = 1000 * (time.perf_counter() - t0) / e2e_steps
        del host
        batch = None
        serve = None
        if not args.no_batch:
            del out
            torch.cuda.empty_cache()
            batch = run_batch(rs, ctx, stream, args)
        if not args.no_serve:
            out = None
            torch.cuda.empty_cache()
            serve = run_serve(rs, ctx, stream, args)
        rows = None
        if not args.no_rows:
            out = None
            torch.cuda.empty_cache()
            rows = run_rows(rs, ctx, stream, args)
    clk = clocks.summary(wall0, wall1)

    ms_per_step = ms_total / args.steps
    e2e_step = max(e2e_ms, e2e_wall_ms)
    if dist is not None:
        ms_per_step, e2e_step, launches = combine_over_ranks(dist, ms_per_step, e2e_step, launches, "cuda")
    value = world * N_SAMPLES / (ms_per_step / 1000)
    leaf_avg_ms = leaf_ms / calls
    peak, peak_kind = hbm_peak()
    achieved = BYTES_PER_SAMPLE * N_SAMPLES / (leaf_avg_ms / 1000) / 1e9
    line = {
        "metric": "sorted samples/s", "value": value, "unit": "samples/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N_SAMPLES, "N": UNIVERSE, "n0": N0, "seed": SEED,
                   "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": "no flush: each step writes 8 GB, 62x the 129 MB L2"},
        "write_gbs": BYTES_PER_SAMPLE * N_SAMPLES / (ms_per_step / 1000) / 1e9,
        "phases_ms": {"split_tree": tree_ms / calls, "leaves": leaf_avg_ms},
        "roofline": {"bound": "hbm", "kernel": "leaf_kernel<uint32,H>", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind + " (MEASURED_PEAKS hbm_gbs)",
                     "traffic": leaf_traffic()},
        "e2e": {"value": world * N_SAMPLES / (e2e_step / 1000), "unit": "samples/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": BYTES_PER_SAMPLE * N_SAMPLES, "ms_per_step": e2e_step,
                "h2d_note": "a step's inputs are four scalars (n, N, seed, n0) passed by value: there is no input "
                            "array to copy; the whole sample is copied to pinned host memory"},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if batch is not None:
        line["batch"] = batch
    if serve is not None:
        line["serve"] = serve
    if rows is not None:
        line["rows"] = rows
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        single = cpu_baseline(8.0)
        line["cpu_baseline"] = cpu_baseline_parallel()
        line["cpu_baseline"]["one_core"] = {"value": single["value"], "sample": single["sample"]}
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


def run_tree_only(args):
    """The split tree of the workload alone (rs_split_tree into a record
    buffer of 32 B per leaf), device-timed: a small footprint for profiling
    the tree kernels."""
    import torch
    import paper_1610_05141_gb300 as rs
    from paper_1610_05141_gb300 import build as rs_build
    rs_build.build()
    rs.load()
    ctx = rs.rs_create(0)
    D = rs.rs_plan(N_SAMPLES, UNIVERSE, N0)
    recs = torch.zeros(4 << D, dtype=torch.int64, device="cuda")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for k in range(args.warmup):
            rs.rs_split_tree(ctx, N_SAMPLES, UNIVERSE, SEED + k, N0, 0, recs, 1 << D, stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(args.steps):
            rs.rs_split_tree(ctx, N_SAMPLES, UNIVERSE, SEED + k, N0, 0, recs, 1 << D, stream)
        e1.record(stream)
        stream.synchronize()
    rc = rs.rs_sync(ctx, stream)
    if rc != rs.RS_OK:
        raise RuntimeError(f"device status {rc}: {rs.strerror(rc)}")
    print(json.dumps({"metric": "split tree ms", "value": e0.elapsed_time(e1) / max(args.steps, 1), "unit": "ms",
                      "higher_is_better": False, "config": {"workload": WORKLOAD, "depth": D}}))
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-requests measurement")
    ap.add_argument("--batch-requests", type=int, default=100_000)
    ap.add_argument("--batch-runs", type=int, default=5)
    ap.add_argument("--unbatched-requests", type=int, default=10000)
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-rows", action="store_true", help="skip with-replacement, leaf B and Bernoulli")
    ap.add_argument("--rows", default="a5,a7,a6,f2,f3,f1,f4",
                    help="which of the other rows to run (comma-separated: a5,a7,a6,f2,f3,f1,f4)")
    ap.add_argument("--row-steps", type=int, default=6)
    ap.add_argument("--row-scale-log2", type=int, default=0,
                    help="divide the a5/a7 sizes and the a6 range by 2^K (profiling cases only)")
    ap.add_argument("--serve-seconds", type=float, default=3.0, help="length of each open-loop serving run")
    ap.add_argument("--serve-capacity-jobs", type=int, default=4000)
    ap.add_argument("--serve-unbatched-jobs", type=int, default=1000)
    ap.add_argument("--serve-arena-gb", type=int, default=64)
    ap.add_argument("--n", "--n-samples", dest="n", type=int, default=None, help="smaller n (profiling cases only)")
    ap.add_argument("--log2N", type=int, default=None, help="smaller universe 2^log2N (profiling cases only)")
    ap.add_argument("--n0", type=int, default=None, help="other leaf size (profiling cases only)")
    ap.add_argument("--tree-only", action="store_true", help="time the split tree alone (profiling)")
    ap.add_argument("--pipeline", default=None,
                    help="LOG2_PARTS,LEAF_BLOCKS_PER_SM for rs_set_pipeline (default: the library's)")
    args = ap.parse_args()
    set_workload(args.n, args.log2N, args.n0)
    if args.tree_only:
        run_tree_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
