"""Host-side inputs and bookkeeping, no GPU: the seeded workload generators
(their ranges, distributions and determinism), the request record layout
shared with the C ABI, and the bench's rule for when a stored DRAM-traffic
figure still applies."""
import ctypes
import json
import os

import numpy as np
import pytest

from paper_1610_05141_gb300 import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_batch_requests_ranges_and_layout():
    n, N, seeds, off, n0, total = workloads.batch_requests(R=20000)
    assert len(n) == len(N) == len(seeds) == len(off) == len(n0) == 20000
    assert n.min() >= 1 and n.max() < 10**6
    assert np.all(N >= n) and N.max() <= 2**48
    assert total == int(n.sum())
    assert off[0] == 0 and np.array_equal(off[1:], np.cumsum(n)[:-1])   # packed back to back
    assert np.array_equal(seeds, np.arange(1, 20001))
    assert np.all(n0 == 4096)
    # n is log-uniform: log10 n roughly uniform on [0, 6)
    h, _ = np.histogram(np.log10(n.astype(float)), bins=6, range=(0, 6))
    assert h.min() > 0.8 * h.mean() and h.max() < 1.2 * h.mean()


def test_batch_requests_deterministic():
    a = workloads.batch_requests(R=1000)
    b = workloads.batch_requests(R=1000)
    for x, y in zip(a[:5], b[:5]):
        assert np.array_equal(x, y)
    c = workloads.batch_requests(R=1000, seed=7)
    assert not np.array_equal(a[0], c[0])


def test_serve_mix():
    trees = workloads.serve_trees()
    assert len(trees) == 8 and all(t[0] == 10**8 and 10**8 <= t[1] <= 2**56 for t in trees)
    J = workloads.serve_jobs(40000, trees)
    q = J["op"] == 1
    assert abs(q.mean() - 0.2) < 0.01
    s = ~q
    assert J["n"][s].min() >= 100 and J["n"][s].max() < 10**8
    assert np.all(J["N"][s] >= J["n"][s]) and J["N"][s].max() <= 2**56
    assert abs(J["n"][s].mean() / 7.24e6 - 1) < 0.1     # log-uniform on [1e2, 1e8): mean (1e8 - 1e2) / ln 1e6
    # queries: expected hits (b - a) n / N in [1e3, 1e5], inside the tree's range, capacity above the mean
    tn = np.array([t[0] for t in trees], dtype=float)[J["tree"][q]]
    tN = np.array([t[1] for t in trees], dtype=float)[J["tree"][q]]
    hits = (J["b"][q] - J["a"][q]).astype(float) * tn / tN
    assert hits.min() > 0.9e3 and hits.max() < 1.1e5
    assert np.all(J["a"][q] >= 1) and np.all(J["b"][q] <= tN + 1)
    assert np.all(J["cap"][q] > hits)


def test_request_record_layout_matches_header():
    import paper_1610_05141_gb300 as rs

    class Req(ctypes.Structure):     # rs_request as declared in include/rs.h
        _fields_ = [("n", ctypes.c_uint64), ("N", ctypes.c_uint64), ("seed", ctypes.c_uint64),
                    ("out_off", ctypes.c_uint64), ("n0", ctypes.c_uint32), ("kind", ctypes.c_uint32)]
    dt = np.dtype(rs.REQUEST_DTYPE)
    assert dt.itemsize == ctypes.sizeof(Req)
    for name, _ in Req._fields_:
        assert dt.fields[name][1] == getattr(Req, name).offset
    a = rs.requests_array([5, 6], [10, 11], [1, 2], [0, 5], [4, 4], [0, 1])
    assert a["n"].tolist() == [5, 6] and a["kind"].tolist() == [0, 1]


def test_job_and_result_records_match_header():
    import paper_1610_05141_gb300 as rs
    # rs_job: two u32, three u64, two u32, a pointer, three u64, a pointer
    assert ctypes.sizeof(rs.Job) == 4 + 4 + 3 * 8 + 4 + 4 + 8 + 3 * 8 + 8
    assert rs.Job.tree.offset == 40 and rs.Job.out_dev.offset == 72
    assert ctypes.sizeof(rs.Result) == 8 + 4 + 4 + 8 + 8 + 3 * 8
    assert ctypes.sizeof(rs.ServerConfig) == 8 + 4 + 4 + 4 + 4 + 8


def test_bench_traffic_record_tracks_leaf_sources():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    with open(bench.TRAFFIC_PATH) as f:
        rec = json.load(f)
    # every source of the leaf kernel is part of the hash, and the record is for the current sources
    srcs = os.listdir(os.path.join(ROOT, "paper_1610_05141_gb300", "csrc"))
    for name in ("rs_leaf.cu", "rs_hash_leaf.cuh", "rs_big_leaf.cuh"):
        assert name in bench.LEAF_SOURCES and name in srcs
    if rec["source_hash"] == bench.leaf_source_hash():
        assert bench.leaf_traffic() == pytest.approx(rec["dram_bytes_per_sample"] * bench.N_SAMPLES)
    else:
        assert bench.leaf_traffic() is None
    assert 7.0 < rec["dram_bytes_per_sample"] <= 8.5


def test_leaf_hash_follows_code_not_comments():
    """The traffic record is keyed to the leaf sources' code: a comment edit
    keeps the hash, a code edit changes it."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    csrc = os.path.join(ROOT, "paper_1610_05141_gb300", "csrc")

    def read(name):
        with open(os.path.join(csrc, name), "rb") as f:
            return f.read()

    base = bench.leaf_source_hash(read)
    assert base == bench.leaf_source_hash()
    first = bench.LEAF_SOURCES[0]
    commented = lambda name: read(name) + (b"\n// a note\n/* and a\n block */\n" if name == first else b"")
    assert bench.leaf_source_hash(commented) == base
    edited = lambda name: read(name) + (b"\nint rs_extra_symbol;\n" if name == first else b"")
    assert bench.leaf_source_hash(edited) != base
