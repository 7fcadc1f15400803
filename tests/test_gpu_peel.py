"""GPU parity of online sorted sampling by peeling (Sec. 4.1): the
iterator's batches, concatenated, equal the oracle's sample bit for bit,
and the batches per call follow the oracle's batch counts, for several
batch limits and buffer sizes; including complement leaves, 64-bit leaf
ranges, n = N, n = 0, one batch (n0 >= n), the largest universe, a buffer
too small for the next batch, and the size the benchmark times."""
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


def _drain(rs, ctx, n, N, seed, n0, B, cap):
    it = rs.rs_peel_create(ctx, n, N, seed, n0, B)
    buf = torch.full((max(cap, 1),), -1, dtype=torch.int64, device="cuda")
    vals, per_call = [], []
    try:
        while True:
            _, cnt, nb = it.next(buf, cap)
            if nb == 0:
                assert cnt == 0
                break
            vals.append(buf[:cnt].cpu().numpy().view(np.uint64).copy())
            per_call.append((nb, cnt))
        assert it.state()[0] == 0
    finally:
        it.close()
    return (np.concatenate(vals) if vals else np.zeros(0, dtype=np.uint64)), per_call


CASES = [
    (20, 1000, 3, 4, 1, 64),
    (100000, 2**50, 1, 4096, 256, 1 << 20),
    (20000, 10**12, 17, 500, 7, 1 << 16),
    (900, 1000, 5, 64, 4, 4096),               # complement leaves
    (30000, 2**62, 6, 1000, 64, 1 << 18),      # the largest universe, 64-bit leaf ranges
    (37, 37, 2, 8, 3, 64),                     # n = N
    (300, 10**9, 3, 4096, 16, 4096),           # n0 >= n: one batch
    (5000, 2**40, 9, 100, 1, 256),             # one batch per call
    (50000, 2**33, 10, 2048, 100, 5000),       # the buffer limits the batches per call
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_peel_matches_oracle(rs, ctx, oracle, case):
    n, N, seed, n0, B, cap = CASES[case]
    got, per_call = _drain(rs, ctx, n, N, seed, n0, B, cap)
    want, counts = oracle.peel_sample(n, N, seed, n0)
    assert got.shape == want.shape
    if not np.array_equal(got, want):
        bad = int(np.argmax(got != want))
        raise AssertionError(f"case {case}: first mismatch at {bad}: gpu {got[bad]} oracle {want[bad]}")
    # the batches per call: a prefix of the oracle's batches that fits cap
    t = 0
    for nb, cnt in per_call:
        assert nb <= B and cnt == int(counts[t:t + nb].sum()) and cnt <= cap
        if t + nb < len(counts):
            assert nb == B or cnt + int(counts[t + nb]) > cap
        t += nb
    assert t == len(counts)


def test_peel_empty_and_capacity(rs, ctx, oracle):
    it = rs.rs_peel_create(ctx, 0, 100, 1, 4)
    assert it.next(None, 0) == (rs.RS_OK, 0, 0)
    it.close()
    n, N, seed, n0 = 5000, 2**40, 4, 512
    _, counts = oracle.peel_sample(n, N, seed, n0)
    it = rs.rs_peel_create(ctx, n, N, seed, n0, 8)
    buf = torch.full((1024,), -1, dtype=torch.int64, device="cuda")
    rc, need, nb = it.next(buf, 10, check=False)
    assert rc == rs.RS_ECAPACITY and nb == 0 and need == int(counts[0])
    assert it.state() == (n, N, 0)
    rc, cnt, nb = it.next(buf, 1024)
    assert rc == rs.RS_OK and nb == 1 and cnt == int(counts[0])
    it.close()
    with pytest.raises(rs.RSError):
        rs.rs_peel_create(ctx, 5, 4, 1, 2)


def test_peel_bench_size(rs, ctx, oracle):
    """n = 1e7 from 2^50, n0 = 4096, 256 batches per call, as the benchmark
    runs it: the whole sample equals the oracle's."""
    n, N, seed, n0 = 10**7, 2**50, 5, 4096
    got, per_call = _drain(rs, ctx, n, N, seed, n0, 256, 1 << 21)
    want, counts = oracle.peel_sample(n, N, seed, n0)
    assert np.array_equal(got, want)
    assert sum(nb for nb, _ in per_call) == len(counts)
