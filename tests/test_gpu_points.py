"""GPU parity of sampling with replacement from a d-dimensional box by
bisection (Sec. 4.6): the device's points equal the oracle's bit for bit
(deep trees, odd and unit extents, 64-bit leaf volumes, one to four
dimensions, one leaf), one dimension equals the sampler with replacement,
and at the size the benchmark times every coordinate lies in its extent."""
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


@pytest.fixture(scope="module")
def oracle():
    import oracle as o
    o.build()
    return o


def _points(rs, ctx, E, n, seed, n0):
    out = torch.full((max(n * len(E), 1),), -1, dtype=torch.int64, device="cuda")
    rs.rs_points(ctx, E, n, seed, n0, out)
    assert rs.rs_sync(ctx) == rs.RS_OK
    return out[: n * len(E)].cpu().numpy().view(np.uint64).reshape(n, len(E))


CASES = [
    ([7, 5], 10000, 11, 16),
    ([2**31, 2**31], 200000, 3, 4096),          # leaf volumes of 2^56: 64-bit keys
    ([2**20, 3, 2**20], 300000, 4, 1024),
    ([1, 1], 50, 1, 8),                         # one point, many draws
    ([6, 5, 4], 3000, 9, 4096),                 # one leaf
    ([2**15] * 4, 100000, 5, 512),
    ([3, 1000003], 20000, 8, 100),
    ([2**16, 2**16], 20000000, 6, 4096),        # 2^13 leaves of 2^19 positions (32-bit keys)
    ([2**31 - 1, 2**31 - 1], 300000, 13, 4096),  # odd extents near 2^31 in every leaf
    ([3, 2**60 + 1], 100000, 14, 4096),         # odd extents near 2^55 after halving
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_points_match_oracle(rs, ctx, oracle, case):
    E, n, seed, n0 = CASES[case]
    got = _points(rs, ctx, E, n, seed, n0)
    want = oracle.points(n, E, seed, n0)
    if not np.array_equal(got, want):
        bad = int(np.argmax((got != want).any(axis=1)))
        raise AssertionError(f"case {case}: first mismatch at point {bad}: gpu {got[bad]} oracle {want[bad]}")


def test_one_dimension_is_with_replacement(rs, ctx):
    n, N, seed, n0 = 100000, 10**9, 2, 256
    got = _points(rs, ctx, [N], n, seed, n0)[:, 0]
    wr = torch.empty(n, dtype=torch.int64, device="cuda")
    rs.rs_sample_with_replacement(ctx, n, N, seed, n0, wr)
    assert rs.rs_sync(ctx) == rs.RS_OK
    assert np.array_equal(got, wr.cpu().numpy().view(np.uint64) - 1)


def test_points_invalid(rs, ctx):
    out = torch.empty(8, dtype=torch.int64, device="cuda")
    for E in ([3, 0], [2**31, 2**31, 2], [1, 1, 1, 1, 1]):
        with pytest.raises(rs.RSError):
            rs.rs_points(ctx, E, 2, 1, 8, out)
    rs.rs_points(ctx, [3, 4], 0, 1, 8, None)


def test_points_bench_size(rs, ctx):
    """1e8 points in [0, 2^31)^2 with n0 = 4096, as the benchmark times it:
    every coordinate inside its extent and both marginals uniform by
    sixteenths."""
    E, n = [2**31, 2**31], 10**8
    out = torch.full((2 * n,), -1, dtype=torch.int64, device="cuda")
    rs.rs_points(ctx, E, n, 5, 4096, out)
    assert rs.rs_sync(ctx) == rs.RS_OK
    P = out.view(n, 2)
    assert bool((P >= 0).all()) and bool((P < 2**31).all())
    for k in range(2):
        h = torch.bincount(P[:, k] >> 27, minlength=16).double()
        assert float(((h - n / 16) ** 2 / (n / 16)).sum()) < 60   # chi^2 with 15 degrees of freedom
    del out, P
    torch.cuda.empty_cache()
