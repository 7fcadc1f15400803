"""The oracle's deviates against their plain definitions.

The oracle evaluates the split deviates (Sec. 3.1: hypergeometric; Sec.
4.6: binomial) and the geometric skips (Sec. 2 Algorithm B, Sec. 4.7) in
FP64 with its own choices of evaluation: a table-driven logarithm, Newton
reciprocals, a division-free ln(1 + z), the logarithms of each ratio-of-
uniforms difference's fixed end taken once per node, ln U times a rounded
reciprocal for the skips.  Those choices are meant to change an outcome
only where the exact test quantity is within rounding of its boundary.
This file checks that claim on at least 10^5 random parameter sets each,
drawn from the sizes the samplers' trees really produce, against
``plain_deviates`` (exact quotients, 40-digit logarithms of factorials,
nothing hoisted): the outcomes must be equal wherever no decision was
within 1e-12 (relative to the magnitude of its terms) of its boundary, and
the number of such close calls is counted, reported and bounded.
"""
import math
import multiprocessing as mpc
import os
import sys
from concurrent.futures import ProcessPoolExecutor

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)

TAG_BERN = 5
N_HG = 100_000
N_BIN = 100_000
N_SKIP_POSITIONS = 100_000


def _jitter(rng, mean, S):
    """A count near `mean` (the spread of a split count), within [0, S]."""
    c = int(round(mean + rng.normal() * math.sqrt(max(mean, 1.0)) * 0.6))
    return min(max(c, 0), S)


def hg_params(count, seed=20161017):
    """(seed, node, n, K, S) tuples: nodes of the trees of the sampling
    workloads at every level (n = 1e9 from 2^50, n = 1e6 from 1e9, the
    batch's log-uniform sizes), the owners' trees of a union of uneven
    segments and the peeling iterator's splits (K far from S/2), and small
    universes (inversion, every reduction)."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        kind = rng.integers(0, 6)
        if kind == 0:      # n = 1e9 from 2^50, depth 18
            lvl = int(rng.integers(0, 18))
            S = (1 << 50) >> lvl
            n = _jitter(rng, 1e9 / 2**lvl, S)
            K = S // 2
        elif kind == 1:    # n = 1e6 from 1e9, depth 8
            lvl = int(rng.integers(0, 8))
            S = (10**9 >> lvl) + int(rng.integers(0, 2))
            n = _jitter(rng, 1e6 / 2**lvl, S)
            K = S // 2
        elif kind == 2:    # the batch: n log-uniform in [1, 1e6), N log-uniform in [n, 2^48]
            n0 = max(1, int(10 ** (6 * rng.random())))
            N = max(n0, int(math.exp(math.log(n0) + rng.random() * (48 * math.log(2) - math.log(n0)))))
            D = 0
            while n0 > 4096 << D:
                D += 1
            while D > 0 and (1 << D) > N:
                D -= 1
            lvl = int(rng.integers(0, D + 1))
            S = max(1, N >> lvl)
            n = _jitter(rng, n0 / 2**lvl, S)
            K = S // 2
        elif kind == 3:    # union of segments: uneven left sums
            S = int(math.exp(rng.random() * 40 * math.log(2))) + 2
            K = int(rng.integers(1, S))
            n = int(min(S, math.exp(rng.random() * math.log(min(S, 10**9)))))
        elif kind == 4:    # peeling: HG(n_t, ceil(N_t n0 / n_t), N_t)
            N_t = int(math.exp(rng.random() * 50 * math.log(2))) + 1
            n_t = max(1, int(min(N_t, math.exp(rng.random() * math.log(min(N_t, 10**8))))))
            K = min(N_t, -(-N_t * 4096 // n_t))
            S, n = N_t, n_t
        else:              # small universes, every reduction
            S = int(rng.integers(1, 400))
            n = int(rng.integers(0, S + 1))
            K = int(rng.integers(0, S + 1))
        out.append((int(rng.integers(1, 2**63)), int(rng.integers(1, 1 << 24)), n, K, S))
    return out


def bin_params(count, seed=20161018):
    """(seed, node, c, K, S) tuples of the with-replacement trees: n = 1e9
    from 2^40 at every level, the batch's sizes with replacement (n may exceed
    N), the points sampler's boxes (K = floor(e/2) of an extent e), small
    counts (inversion)."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        kind = rng.integers(0, 4)
        if kind == 0:
            lvl = int(rng.integers(0, 18))
            S = (1 << 40) >> lvl
            c = _jitter(rng, 1e9 / 2**lvl, 1 << 62)
            K = S // 2
        elif kind == 1:
            c0 = max(1, int(10 ** (6 * rng.random())))
            N = max(2, int(math.exp(rng.random() * 48 * math.log(2))))
            lvl = int(rng.integers(0, 12))
            S = max(2, N >> lvl)
            c = _jitter(rng, c0 / 2**lvl, 1 << 62)
            K = S // 2
        elif kind == 2:    # a box's halving: ratio floor(e/2) / e for its largest extent e
            e = int(rng.integers(2, 1 << 31))
            S, K = e, e // 2
            c = _jitter(rng, math.exp(rng.random() * math.log(1e8)), 1 << 62)
        else:
            S = int(rng.integers(2, 1000))
            K = int(rng.integers(1, S // 2 + 1))
            c = int(rng.integers(0, 60))
        out.append((int(rng.integers(1, 2**63)), int(rng.integers(1, 1 << 24)), c, K, S))
    return out


def _hg_chunk(params):
    import oracle
    import plain_deviates as pd
    res = []
    for (sd, node, n, K, S) in params:
        got = oracle.hg(sd, node, n, K, S)
        want, amb = pd.plain_hg(sd, node, n, K, S)
        res.append((got, want, amb))
    return res


def _bin_chunk(params):
    import oracle
    import plain_deviates as pd
    res = []
    for (sd, node, c, K, S) in params:
        got = oracle.binom(sd, node, c, K, S)
        want, amb = pd.plain_bin(sd, node, c, K, S)
        res.append((got, want, amb))
    return res


def _skip_chunk(cases):
    import oracle
    import plain_deviates as pd
    res = []
    for (sd, p, chunk) in cases:
        n0 = 256
        cl = oracle.bern_chunk_log2(p, n0)
        C = 1 << cl
        N = 1 << 62
        i = chunk % (N >> cl)
        a, b = i * C, (i + 1) * C
        got = [int(x) - 1 for x in oracle.bernoulli(p, N, sd, n0, a, b)]
        want, first_amb = pd.plain_skips(sd, TAG_BERN, i, p, a, b)
        upto = len(want) if first_amb is None else first_amb
        same = got[:upto] == want[:upto] and (first_amb is not None or len(got) == len(want))
        res.append((same, first_amb is not None, upto))
    return res


def _run(fn, items, chunks=64):
    import oracle
    oracle.build()
    parts = [items[i::chunks] for i in range(chunks)]
    with ProcessPoolExecutor(max_workers=os.cpu_count() or 4, mp_context=mpc.get_context("spawn")) as ex:
        out = []
        for r in ex.map(fn, parts):
            out.extend(r)
    return out


def _summarise(name, res, limit):
    amb = sum(1 for (_, _, a) in res if a)
    bad = [(g, w) for (g, w, a) in res if not a and g != w]
    print(f"\n{name}: {len(res)} deviates, {len(bad)} disagreements away from a boundary, "
          f"{amb} with a decision within 1e-12 of its boundary")
    assert not bad, f"{name}: oracle differs from the plain definition: {bad[:5]}"
    assert amb <= limit, f"{name}: {amb} close calls"


def test_hg_matches_plain_definition():
    _summarise("HG", _run(_hg_chunk, hg_params(N_HG)), N_HG // 1000)


def test_bin_matches_plain_definition():
    _summarise("BIN", _run(_bin_chunk, bin_params(N_BIN)), N_BIN // 1000)


def test_skips_match_plain_definition():
    rng = np.random.default_rng(4711)
    cases = []
    # p log-uniform from 1e-12 to 0.999; each chunk has about 256-512 positions
    while len(cases) * 300 < N_SKIP_POSITIONS:
        p = float(math.exp(rng.uniform(math.log(1e-12), math.log(0.999))))
        cases.append((int(rng.integers(1, 2**63)), p, int(rng.integers(0, 1 << 40))))
    res = _run(_skip_chunk, cases)
    compared = sum(n for (_, _, n) in res)
    amb = sum(1 for (_, a, _) in res if a)
    bad = sum(1 for (ok, _, _) in res if not ok)
    print(f"\nskips: {compared} positions compared in {len(res)} chunks, {bad} chunks differing before a "
          f"close call, {amb} chunks with a skip within 1e-14 of an integer")
    assert compared >= N_SKIP_POSITIONS
    assert bad == 0
    # close calls come from p below about 1e-9, where a skip q exceeds 1e9 and
    # FP64 resolves its floor only to about q 2^-52: a chunk of ~300 such
    # skips then holds one with some probability
    assert amb <= len(res) // 5


def test_comparison_catches_small_changes():
    """The comparison has teeth: the plain definition with a hat that lacks
    its additive constant, or with each skip rounded up instead of down,
    disagrees with the oracle on many cases."""
    import mpmath as mp
    import oracle
    import plain_deviates as pd
    cases = [c for c in hg_params(400, seed=5) if c[2] * c[3] > 64 * c[4]][:150]
    saved = pd.HAT_D2
    try:
        pd.HAT_D2 = mp.mpf(0)
        moved = sum(1 for (sd, node, n, K, S) in cases if pd.plain_hg(sd, node, n, K, S)[0] != oracle.hg(sd, node, n, K, S))
    finally:
        pd.HAT_D2 = saved
    assert moved > len(cases) // 10
    sd, p = 99, 0.013
    want = oracle.bernoulli(p, 1 << 62, sd, 256, 0, 1 << oracle.bern_chunk_log2(p, 256)) - 1
    pos, up = -1, []
    for j in range(len(want) + 5):
        U = ((oracle.value(sd, TAG_BERN, 0, j) >> 11) + 1) / 2.0**53
        pos += math.ceil(math.log(U) / math.log1p(-p)) + 1
        if pos >= 1 << oracle.bern_chunk_log2(p, 256):
            break
        up.append(pos)
    assert list(map(int, want)) != up
