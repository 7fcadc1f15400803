"""The allocation-free entry point rs_sample_static, for callers that cannot
allocate device memory while they run, gives the same sample as rs_sample.

Kept in a file of its own, collected last: it must pass in a fresh process
and after the other GPU tests (its static scratch persists between calls)."""
import ctypes

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


CASES = [(10**6, 10**9, 1, 4096), (5000, 6000, 7, 128), (123457, 2**62, 3, 512)]


def test_static_matches_sample_on_two_calls(rs):
    lib = rs.load()
    assert hasattr(lib, "rs_sample_static")
    ctx = rs.rs_create(0)
    try:
        stream = torch.cuda.current_stream().cuda_stream
        for n, N, seed, n0 in CASES:
            ref = torch.empty(n, dtype=torch.int64, device="cuda")
            rs.rs_sample(ctx, n, N, seed, n0, ref)
            assert rs.rs_sync(ctx) == rs.RS_OK
            want = ref.cpu().numpy()
            for _ in range(2):   # the static scratch keeps the previous call's contents
                out = torch.full((n,), -1, dtype=torch.int64, device="cuda")
                rc = lib.rs_sample_static(ctypes.c_uint64(n), ctypes.c_uint64(N), ctypes.c_uint64(seed),
                                          ctypes.c_uint32(n0), ctypes.c_void_p(out.data_ptr()),
                                          ctypes.c_void_p(stream))
                assert rc == rs.RS_OK, rs.strerror(rc)
                assert np.array_equal(out.cpu().numpy(), want), (n, N, seed)
    finally:
        ctx.close()


def test_static_rejects_sizes_beyond_its_limit(rs):
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
