"""Plain-definition evaluation of the split deviates and geometric skips.

Test infrastructure: an independent statement of what the oracle's
hypergeometric and binomial deviates and its Bernoulli skips compute, written
from their definitions with exact quotients and 40-digit logarithms of
factorials (mpmath), with none of the oracle's evaluation choices: no
table-driven logarithm, no Newton reciprocals, no division-free ln(1 + z), no
logarithm taken once per node, no single-precision seeds.

Each function replays the same random values (64-bit values of the keyed
stream, read through the oracle's stream function, whose Philox blocks and
word layout are pinned on their own) and returns the result together with
a flag that says whether some decision on the way was too close to call: a
decision counts as ambiguous when its exact test quantity lies within
``eps`` (relative to the magnitude of the terms that form it) of its
boundary, where the FP64 evaluation of the oracle may legitimately fall on
the other side.

Definitions followed (the paper's split deviates, Sec. 3.1 and Sec. 4.6, and
its geometric skips, Sec. 2 Algorithm B and Sec. 4.7):

* HG(n, K, S), successes among n draws without replacement from S items of
  which K are successes.  Reductions K -> S - K when 2K > S and n -> S - n
  when 2n > S; a = min(n, K), b = max(n, K), mean a b / S.  Below mean 16:
  inversion, the least k with u < F(k), F the exact distribution function,
  u the [0, 1) uniform of value 0.  Otherwise ratio-of-uniforms with the
  table-mountain hat: trial i draws U in (0, 1] (value 2i) and V in [0, 1)
  (value 2i + 1), X = (mean + 1/2) + h (V - 1/2) / U with
  h = 2 sqrt(2/e) sqrt(var + 1/2) + 3 - 2 sqrt(3/e), rejected outside
  [0, a + 1), else k = floor(X) is accepted when 2 ln U <= ln f(k) - ln f(M),
  M = floor((a + 1)(b + 1) / (S + 2)).  The result is un-reduced.
* BIN(c, K/S), p = K / S <= 1/2: the same with the binomial pmf, mean c p,
  var = c p (1 - p), M = floor((c + 1) K / S), rejection above c + 1.
* Skips over [start, end) with probability p: the j-th value's U in (0, 1],
  skip floor(ln U / ln(1 - p)); a skip of 2^62 or more ends the range.
"""
from __future__ import annotations

import mpmath as mp

import oracle

mp.mp.dps = 40
TAG_SPLIT = 1
TWO53 = mp.mpf(2) ** 53
HAT_D1 = 2 * mp.sqrt(2 / mp.e)
HAT_D2 = 3 - 2 * mp.sqrt(3 / mp.e)
EPS = mp.mpf("1e-12")


def _u_open(x: int):
    return mp.mpf((x >> 11) + 1) / TWO53


def _v_closed(x: int):
    return mp.mpf(x >> 11) / TWO53


def _lf(x: int):
    return mp.loggamma(mp.mpf(x) + 1)


def _near(x, y, scale, eps=EPS) -> bool:
    return abs(x - y) <= eps * scale


def _rou(seed, node, a_top, alpha, h, M_terms, logf_k, eps):
    """Ratio-of-uniforms trials; returns (k, ambiguous).  logf_k(k) returns
    the list of terms whose sum is ln f(k) - ln f(M)."""
    amb = False
    for i in range(1 << 20):
        U = _u_open(oracle.value(seed, TAG_SPLIT, node, 2 * i))
        V = _v_closed(oracle.value(seed, TAG_SPLIT, node, 2 * i + 1))
        t = h * (V - mp.mpf(0.5)) / U
        X = alpha + t
        sx = abs(alpha) + abs(t) + 1
        if _near(X, 0, sx, eps) or _near(X, a_top + 1, sx, eps):
            amb = True
        if X < 0 or X >= a_top + 1:
            continue
        k = int(mp.floor(X))
        if _near(X, k, sx, eps) or _near(X, k + 1, sx, eps):
            amb = True
        terms = logf_k(k)
        T = mp.fsum(terms)
        lhs = 2 * mp.log(U)
        if _near(lhs, T, mp.fsum(abs(x) for x in terms) + abs(lhs) + 1, eps):
            amb = True
        if lhs <= T:
            return k, amb
    raise RuntimeError("no trial accepted")


def _inversion(seed, node, lnp0, mag, ratio, kmax, eps):
    """Least k with u < F(k) where F(0) = e^lnp0 and f(k+1) = f(k) ratio(k);
    ambiguous when u lies within eps * mag (the relative accuracy of an
    FP64 evaluation of lnp0, whose terms have magnitude mag) of some F(k)."""
    u = _v_closed(oracle.value(seed, TAG_SPLIT, node, 0))
    p = mp.exp(lnp0)
    F = mp.mpf(0)
    amb = False
    k = 0
    while True:
        F += p
        if abs(u - F) <= eps * (mag * F + 1):
            amb = True
        if u < F:
            return k, amb
        p = p * ratio(k)
        k += 1
        if k > kmax:
            raise RuntimeError("inversion ran past the support")


def plain_hg(seed: int, node: int, n: int, K: int, S: int, eps=EPS):
    """HG(n, K, S) by its definition; returns (value, ambiguous)."""
    if n == 0 or K == 0:
        return 0, False
    if K == S:
        return n, False
    if n == S:
        return K, False
    n_orig = n
    sK = 2 * K > S
    if sK:
        K = S - K
    sN = 2 * n > S
    if sN:
        n = S - n
    a, b = min(n, K), max(n, K)
    m = S - a - b
    mu = mp.mpf(a) * b / S
    amb = _near(mu, 16, 16, eps)
    if mu < 16:
        sd1 = _lf(S - b) - _lf(S - a - b)
        sd2 = _lf(S) - _lf(S - a)
        Y, amb2 = _inversion(seed, node, sd1 - sd2, abs(sd1) + abs(sd2) + 1,
                             lambda k: mp.mpf((a - k) * (b - k)) / ((k + 1) * (m + k + 1)), a, eps)
    else:
        var = mu * (mp.mpf(S - a) / S) * (mp.mpf(S - b) / (S - 1))
        h = HAT_D1 * mp.sqrt(var + mp.mpf(0.5)) + HAT_D2
        M = ((a + 1) * (b + 1)) // (S + 2)
        f0 = (_lf(M), _lf(a - M), _lf(b - M), _lf(m + M))
        Y, amb2 = _rou(seed, node, a, mu + mp.mpf(0.5), h, f0,
                       lambda k: [f0[0] - _lf(k), f0[1] - _lf(a - k), f0[2] - _lf(b - k), f0[3] - _lf(m + k)], eps)
    if sN:
        Y = K - Y
    if sK:
        Y = n_orig - Y
    return Y, amb or amb2


def plain_bin(seed: int, node: int, c: int, K: int, S: int, eps=EPS):
    """BIN(c, K/S), K/S <= 1/2, by its definition; returns (value, ambiguous)."""
    if c == 0 or K == 0:
        return 0, False
    p = mp.mpf(K) / S
    mu = c * p
    amb = _near(mu, 16, 16, eps)
    r = p / (1 - p)
    if mu < 16:
        lnp0 = c * mp.log1p(-p)
        Y, amb2 = _inversion(seed, node, lnp0, abs(lnp0) + 1, lambda k: (c - k) * r / (k + 1), c, eps)
    else:
        h = HAT_D1 * mp.sqrt(mu * (1 - p) + mp.mpf(0.5)) + HAT_D2
        M = ((c + 1) * K) // S
        logr = mp.log(r)
        f0 = (_lf(M), _lf(c - M))
        Y, amb2 = _rou(seed, node, c, mu + mp.mpf(0.5), h, f0,
                       lambda k: [f0[0] - _lf(k), f0[1] - _lf(c - k), (k - M) * logr], eps)
    return Y, amb or amb2


def plain_skips(seed: int, tag: int, node: int, p: float, start: int, end: int, eps=mp.mpf("1e-14")):
    """0-based positions chosen in [start, end) by geometric skips of the
    (tag, node) stream; returns (positions, index of the first position
    whose skip was within eps of an integer, or None).  The oracle's skip
    ln U * RN(1 / ln(1 - p)) is within a few ulp of the quotient, so its
    floor can differ only inside that zone; positions after a close call may
    all move by one."""
    L = mp.log1p(-mp.mpf(p))
    pos = start - 1
    out = []
    first_amb = None
    two62 = mp.mpf(2) ** 62
    j = 0
    while True:
        U = _u_open(oracle.value(seed, tag, node, j))
        j += 1
        q = mp.mpf(0) if U == 1 else mp.log(U) / L
        sq = abs(q) + 1
        amb = _near(q, two62, sq, eps)
        if q >= two62:
            if amb and first_amb is None:
                first_amb = len(out)
            break
        f = int(mp.floor(q))
        amb = amb or _near(q, f, sq, eps) or _near(q, f + 1, sq, eps)
        if amb and first_amb is None:
            first_amb = len(out)
        pos = pos + f + 1
        if pos >= end:
            break
        out.append(pos)
    return out, first_amb
