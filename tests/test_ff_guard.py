"""The second guard of the split deviates (rs_ff.cuh), checked on the CPU
through a model of its float-float arithmetic: every single-precision
operation of the device code restated with numpy float32 (round to nearest),
fused multiply-adds and conversions by exact rationals, the fixed-point
logarithm by its integer model (qlog_model).

The guard's margins are 2^-36 of the magnitudes involved plus 2^-26; it
rests on its evaluations being far closer than that to the exact values.
Pinned here against mpmath on every argument regime of ln x! - ln y! (the
table, the Stirling form against a table value, the series for ln(1 + d/y)
and the difference of two fixed-point logarithms, up to 2^62) and on the
nodes' parameters (alpha, h, and the binomial log-odds): the evaluations must stay within 2^-40 of their
magnitudes (plus 2^-30 for the single-precision Stirling tails)."""
import math
from fractions import Fraction

import mpmath as mp
import numpy as np
import pytest

from qlog_model import LN2FRAC32, LN2Q57, make_table, qnlog_u57

f32 = np.float32


def rn(x):
    """A rational rounded to the nearest single (ties to even)."""
    x = Fraction(x)
    f = f32(float(x))
    while Fraction(float(f)) > x:
        f = np.nextafter(f, f32(-np.inf))
    while Fraction(float(np.nextafter(f, f32(np.inf)))) <= x:
        f = np.nextafter(f, f32(np.inf))
    lo, hi = f, np.nextafter(f, f32(np.inf))
    dl, dh = x - Fraction(float(lo)), Fraction(float(hi)) - x
    if dl == 0:
        return lo
    if dl != dh:
        return lo if dl < dh else hi
    return lo if (lo.view(np.uint32) & 1) == 0 else hi


def fma(a, b, c):
    return rn(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def fast2(a, b):
    s = f32(a + b)
    return (s, f32(b - f32(s - a)))


def two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    return (s, f32(f32(a - f32(s - bb)) + f32(b - bb)))


def ff_add(x, y):
    s, e = two_sum(x[0], y[0])
    return fast2(s, f32(e + f32(x[1] + y[1])))


def ff_neg(x):
    return (f32(-x[0]), f32(-x[1]))


def ff_sub(x, y):
    return ff_add(x, ff_neg(y))


def ff_mul(x, y):
    p = f32(x[0] * y[0])
    e = f32(fma(x[0], y[0], -p) + f32(f32(x[0] * y[1]) + f32(x[1] * y[0])))
    return fast2(p, e)


def ff_mul_f(x, f):
    p = f32(x[0] * f)
    return fast2(p, f32(fma(x[0], f, -p) + f32(x[1] * f)))


def rcp(x):
    return rn(Fraction(1) / Fraction(float(x)))


def ff_div(x, y):
    r = rcp(y[0])
    q1 = f32(x[0] * r)
    rem = ff_sub(x, ff_mul_f(y, q1))
    return fast2(q1, f32(rem[0] * r))


def ff_sqrt(x):
    s = f32(np.sqrt(x[0]))
    p = f32(s * s)
    d = ff_add(x, (f32(-p), f32(-fma(s, s, -p))))
    return fast2(s, f32(d[0] * f32(f32(0.5) * rcp(s))))


def ff_from_u64(x):
    h = rn(x)
    return (h, rn(x - int(Fraction(float(h)))))


def ff_from_double(d):
    h = f32(d)
    return (h, f32(d - float(h)))


def ff_from_q57(L):
    h = rn(L)
    rest = L - int(Fraction(float(h)))
    return (f32(h * f32(2.0**-57)), f32(rn(rest) * f32(2.0**-57)))


def val(x):
    return Fraction(float(x[0])) + Fraction(float(x[1]))


def ln_q57(m, table):
    return 53 * LN2Q57 + ((53 * LN2FRAC32) >> 32) - qnlog_u57(m, table)


def ff_tail(x):
    r = rcp(rn(x))
    return f32(r * f32(f32(0.083333333) - f32(f32(f32(0.0027777778) * r) * r)))


C7 = (f32(1.428571492e-01), f32(-6.386212004e-09))
C5 = (f32(2.000000030e-01), f32(-2.980232283e-09))
C3 = (f32(3.333333433e-01), f32(-9.934107759e-09))
HL2PI = (f32(9.189385176e-01), f32(1.563417662e-08))


def ff_lfdiff(x, y, lf, table):
    """rs_ff.cuh ff_lfdiff, operation for operation; lf(i) = ln i! as the
    FP64 table holds it."""
    if x < 256:
        a, b = ff_from_double(lf(x)), ff_from_double(lf(y))
        return ff_sub(a, b), float(a[0]) + float(b[0]) + 1
    X = ff_from_u64(x)
    Xh = ff_add(X, (f32(0.5), f32(0)))
    if y < 256:
        lx = ff_from_q57(ln_q57(x, table))
        A = ff_mul(Xh, lx)
        ly = ff_from_double(lf(y))
        mag = float(A[0]) + float(X[0]) + float(ly[0]) + 2
        v = ff_sub(A, X)
        v = ff_add(v, HL2PI)
        v = ff_add(v, (ff_tail(x), f32(0)))
        return ff_sub(v, ly), mag
    d = x - y
    D = ff_from_u64(d)
    lyq = ln_q57(y, table)
    if d < (y >> 5):
        w = ff_div(D, ff_from_u64(2 * y + d))
        w2 = ff_mul(w, w)
        s = ff_add(C7, ff_mul_f(w2, f32(1.111111119e-01)))
        s = ff_add(C5, ff_mul(w2, s))
        s = ff_add(C3, ff_mul(w2, s))
        s = ff_add((f32(1), f32(0)), ff_mul(w2, s))
        l1p = ff_mul_f(ff_mul(w, s), f32(2))
    else:
        l1p = ff_from_q57(ln_q57(x, table) - lyq)
    A = ff_mul(Xh, l1p)
    B = ff_mul(D, ff_from_q57(lyq))
    mag = float(A[0]) + float(B[0]) + float(D[0]) + 1
    v = ff_add(A, B)
    v = ff_sub(v, D)
    return ff_add(v, (f32(ff_tail(x) - ff_tail(y)), f32(0))), mag


@pytest.fixture(scope="module")
def table():
    return make_table()


def _lf(i):
    return float(mp.loggamma(mp.mpf(i) + 1))


def _cases():
    rng = np.random.default_rng(36)
    out = []
    for _ in range(60):                                   # the table
        x = int(rng.integers(1, 256))
        out.append((x, int(rng.integers(0, x))))
    for _ in range(80):                                   # Stirling against a table value
        x = int(np.exp(rng.uniform(np.log(256), np.log(2.0**62))))
        out.append((x, int(rng.integers(0, 256))))
    for _ in range(200):                                  # ln(1 + d/y) by its series
        y = int(np.exp(rng.uniform(np.log(256), np.log(2.0**62))))
        d = int(np.exp(rng.uniform(0, np.log(max(2, y // 32)))))
        out.append((y + d, y))
    for _ in range(120):                                  # by two fixed-point logarithms
        y = int(np.exp(rng.uniform(np.log(256), np.log(2.0**50))))
        d = int(np.exp(rng.uniform(np.log(y / 32 + 1), np.log(8.0 * y))))
        out.append((y + d, y))
    out += [(256, 255), (257, 256), (2**62, 2**62 - 1), (2**40 + 2**35, 2**40), (1000, 256), (2**33, 2**33 - 1)]
    return out


def test_ff_lfdiff_within_its_bound(table):
    mp.mp.dps = 60
    worst = 0.0
    for x, y in _cases():
        v, mag = ff_lfdiff(x, y, _lf, table)
        exact = mp.loggamma(mp.mpf(x) + 1) - mp.loggamma(mp.mpf(y) + 1)
        err = abs(mp.mpf(val(v).numerator) / val(v).denominator - exact)
        bound = mp.mpf(2) ** -40 * mag + mp.mpf(2) ** -30
        worst = max(worst, float(err / bound))
        assert err <= bound, (x, y, float(err), mag)
    # the guard's margin is 2^-36 mag + 2^-26: far above what is seen here
    assert worst < 1.0


def test_ff_node_parameters_within_their_bound():
    """alpha = a b / S + 1/2 and h = D1 sqrt(var + 1/2) + D2 of the
    hypergeometric set-up in float-float (setupff), against exact values."""
    mp.mp.dps = 60
    rng = np.random.default_rng(37)
    d1 = (f32(1.715527773e+00), f32(-2.982028846e-09))
    d2 = (f32(8.989161849e-01), f32(-2.284329170e-08))
    half = (f32(0.5), f32(0))
    for _ in range(300):
        S = int(np.exp(rng.uniform(np.log(40), np.log(2.0**62))))
        a = max(1, int(np.exp(rng.uniform(0, np.log(S / 2)))))
        b = int(rng.integers(a, S // 2 + 1)) if S // 2 >= a else a
        Sf = ff_from_u64(S)
        mu = ff_div(ff_mul(ff_from_u64(a), ff_from_u64(b)), Sf)
        var = ff_mul(ff_mul(mu, ff_div(ff_from_u64(S - a), Sf)), ff_div(ff_from_u64(S - b), ff_from_u64(S - 1)))
        h = ff_add(ff_mul(d1, ff_sqrt(ff_add(var, half))), d2)
        alpha = ff_add(mu, half)
        mu_x = mp.mpf(a) * b / S
        var_x = mu_x * (mp.mpf(S - a) / S) * (mp.mpf(S - b) / (S - 1))
        h_x = 2 * mp.sqrt(2 / mp.e) * mp.sqrt(var_x + mp.mpf(0.5)) + 3 - 2 * mp.sqrt(3 / mp.e)
        for got, want in ((alpha, mu_x + mp.mpf(0.5)), (h, h_x)):
            g = mp.mpf(val(got).numerator) / val(got).denominator
            assert abs(g - want) <= mp.mpf(2) ** -40 * abs(want), (S, a, b, float(g), float(want))


def test_ff_binomial_parameters_within_their_bound(table):
    """alpha, h and ln(p / (1 - p)) of the binomial set-up in float-float
    (ff_bin_params: p = K / S, mean c p, variance c p (1 - p), the log-odds
    as a difference of two fixed-point logarithms), against exact values."""
    mp.mp.dps = 60
    rng = np.random.default_rng(38)
    d1 = (f32(1.715527773e+00), f32(-2.982028846e-09))
    d2 = (f32(8.989161849e-01), f32(-2.284329170e-08))
    half = (f32(0.5), f32(0))
    for _ in range(300):
        S = int(np.exp(rng.uniform(np.log(4), np.log(2.0**62))))
        K = int(rng.integers(1, S // 2 + 1))
        c = max(1, int(np.exp(rng.uniform(0, np.log(2.0**62)))))
        pp = ff_div(ff_from_u64(K), ff_from_u64(S))
        mu = ff_mul(ff_from_u64(c), pp)
        h = ff_add(ff_mul(d1, ff_sqrt(ff_add(ff_mul(mu, ff_sub((f32(1), f32(0)), pp)), half))), d2)
        alpha = ff_add(mu, half)
        logr = (f32(0), f32(0)) if 2 * K == S else ff_from_q57(ln_q57(K, table) - ln_q57(S - K, table))
        p_x = mp.mpf(K) / S
        mu_x = c * p_x
        h_x = 2 * mp.sqrt(2 / mp.e) * mp.sqrt(mu_x * (1 - p_x) + mp.mpf(0.5)) + 3 - 2 * mp.sqrt(3 / mp.e)
        lr_x = mp.log(mp.mpf(K)) - mp.log(mp.mpf(S - K))
        for got, want in ((alpha, mu_x + mp.mpf(0.5)), (h, h_x)):
            g = mp.mpf(val(got).numerator) / val(got).denominator
            assert abs(g - want) <= mp.mpf(2) ** -40 * abs(want), (S, K, c, float(g), float(want))
        g = mp.mpf(val(logr).numerator) / val(logr).denominator
        # the log-odds enter the test times |k - M|; the guard's margin
        # grants 2^-36 |k - M| for their error
        assert abs(g - lr_x) <= mp.mpf(2) ** -44 * (1 + abs(lr_x)), (S, K, float(g), float(lr_x))
