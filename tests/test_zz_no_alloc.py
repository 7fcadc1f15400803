"""rs_sample_static, the entry point for callers that cannot allocate device
memory while they run (an allocator that owns the whole device, a host
application that forbids cudaMalloc after start-up, a loop that cannot take
the device-wide stall of cudaMalloc/cudaFree), gives the oracle's sample.

The calls run in a fresh child process that never creates a context, so
nothing the context path builds can stand in for the static array's own
set-up; the child calls each case twice in a row (the array keeps the
previous call's contents) and reports the device's free memory around the
second call, which must not move.  Kept in a file of its own, collected
last, so that it also runs after every other GPU test."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (n, N, seed, n0): 32-bit keys with void candidates (leaves of 3,906,250
# positions), complement leaves (bitmap path), 64-bit keys, the 512-thread
# leaf shape (about 8,192 samples per leaf of 2^32 positions)
CASES = [(10**6, 10**9, 1, 4096), (5000, 6000, 7, 128), (123457, 2**62, 3, 512), (8192 * 64, 2**38, 5, 8192)]
# one leaf selecting 2^17 values: above the static general-path pool of 2^16
CAPACITY_CASE = (2**17, 2**40, 1, 2**17)

_CHILD = r"""
import ctypes, json, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import paper_1610_05141_gb300 as rs
lib = rs.load()   # the library only: no context is created in this process
cases, cap_case, outdir = json.loads(sys.argv[2]), json.loads(sys.argv[3]), sys.argv[4]
torch.cuda.set_device(0)
stream = torch.cuda.current_stream().cuda_stream

def call(n, N, seed, n0, out):
    return int(lib.rs_sample_static(ctypes.c_uint64(n), ctypes.c_uint64(N), ctypes.c_uint64(seed),
                                    ctypes.c_uint32(n0), ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream)))

report = {"cases": [], "capacity": None}
for i, (n, N, seed, n0) in enumerate(cases):
    runs = []
    for rep in range(2):
        out = torch.full((n,), -1, dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        rc = call(n, N, seed, n0, out)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        np.save(f"{outdir}/case{i}_{rep}.npy", out.cpu().numpy())
        runs.append([rc, free0, free1])
    report["cases"].append(runs)
n, N, seed, n0 = cap_case
out = torch.empty(n, dtype=torch.int64, device="cuda")
report["capacity"] = call(n, N, seed, n0, out)
print(json.dumps(report))
"""


@pytest.fixture(scope="module")
def child_report(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_05141_gb300 import build
    build.build()
    outdir = tmp_path_factory.mktemp("static")
    p = subprocess.run([sys.executable, "-c", _CHILD, ROOT, json.dumps(CASES), json.dumps(CAPACITY_CASE),
                        str(outdir)], capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    return json.loads(p.stdout.strip().splitlines()[-1]), outdir


@pytest.mark.parametrize("i", range(len(CASES)))
def test_static_matches_oracle_on_two_calls(child_report, oracle, i):
    import paper_1610_05141_gb300 as rs
    report, outdir = child_report
    n, N, seed, n0 = CASES[i]
    want = oracle.sample(n, N, seed, n0, oracle.KIND_H)
    for rep, (rc, free0, free1) in enumerate(report["cases"][i]):
        assert rc == rs.RS_OK, (rep, rs.strerror(rc))
        got = np.load(outdir / f"case{i}_{rep}.npy").view(np.uint64)
        assert np.array_equal(got, want), (CASES[i], rep, int(np.argmax(got != want)))
    # the second call allocates nothing: the device's free memory does not move
    _, free0, free1 = report["cases"][i][1]
    assert free0 == free1, (free0, free1)


def test_static_leaf_over_its_pool_reports_capacity(child_report):
    import paper_1610_05141_gb300 as rs
    report, _ = child_report
    assert report["capacity"] == rs.RS_ECAPACITY


def test_static_rejects_sizes_beyond_its_limit():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import ctypes

    import paper_1610_05141_gb300 as rs
    lib = rs.load()
    out = torch.empty(8, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    # n = n0 * 2^16 + 1 needs depth 17
    rc = lib.rs_sample_static(ctypes.c_uint64(4096 * 2**16 + 1), ctypes.c_uint64(2**40), ctypes.c_uint64(1),
                              ctypes.c_uint32(4096), ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
    assert rc == rs.RS_ECAPACITY
    rc = lib.rs_sample_static(ctypes.c_uint64(11), ctypes.c_uint64(10), ctypes.c_uint64(1), ctypes.c_uint32(4),
                              ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
    assert rc == rs.RS_EINVAL
