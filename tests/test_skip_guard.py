"""The guarded geometric skip of the CUDA path (rs_bern.cu skip_fast, with
rs_math.cuh qnlog_u57), checked on the CPU through a model of its integer and
single-precision arithmetic.

The skip of a draw is floor(q) for q = RN(ln U * R), R = RN(1 / ln(1 - p))
(Sec. 2 Algorithm B, Sec. 4.7), ln U the FP64 logarithm of the definition.
The CUDA path decides it without FP64 when a bound says the decision is
safe, and evaluates the definition otherwise; both claims behind that are
pinned here:

* the fixed-point logarithm is within 2^-55 of -ln U (exact rational
  reference, every exponent, every table interval and its edges);
* wherever the modelled single-precision decision is taken it equals the
  oracle's floor of q, on random draws and on draws whose q lies within
  2^-30 of an integer, for p from 1e-9 to 0.9;
* the constants in the source are what their comments say.

The model restates the device code's operations one for one (Python
integers for the 64-bit arithmetic, numpy float32 with exact rational
checks for the single-precision steps)."""
import math
import os
import re
from fractions import Fraction

import mpmath
import numpy as np
import pytest

from qlog_model import H, INTERVALS, LN2FRAC32, LN2Q57, M64, make_table, qnlog_u57


def test_constants_match_their_definitions():
    mpmath.mp.dps = 60
    for k in range(3, 7):
        assert abs(H[k] - Fraction(2**32, k)) <= Fraction(1, 2), k
    ln2 = mpmath.log(2) * 2**57
    assert LN2Q57 == int(mpmath.floor(ln2))
    assert abs(LN2FRAC32 - (ln2 - LN2Q57) * 2**32) <= 0.5


def _mulhi(a, b):   # unsigned high 64 bits
    return (a * b) >> 64


@pytest.fixture(scope="module")
def table():
    return make_table()


def _draws():
    rng = np.random.default_rng(57)
    ms = [1, 2, 3, 2**52 - 1, 2**52, 2**52 + 1, 2**53 - 2, 2**53 - 1]
    for t in range(53):
        ms += [int(v) for v in rng.integers(1 << t, 1 << (t + 1), 40, dtype=np.uint64)] if t < 63 else []
    for i in range(INTERVALS):
        for t in (52, 47, 30, 12):
            base = (1 << t) + ((i << t) >> 9)
            ms += [base + d for d in (-2, -1, 0, 1, 2) if 1 <= base + d < 1 << 53]
    return ms


def test_fixed_point_log_within_its_bound(table):
    mpmath.mp.dps = 50
    worst = mpmath.mpf(0)
    for m in _draws():
        exact = -mpmath.log(mpmath.mpf(m) / 2**53) * 2**57
        worst = max(worst, abs(qnlog_u57(m, table) - exact))
    assert worst <= 2.1, float(worst)   # units of 2^-57: the bound 2^-55.9


# --- single precision -------------------------------------------------------

f32 = np.float32


def _round_dir(x: Fraction, up: bool) -> np.float32:
    """x rounded to float32 toward +inf (up) or -inf."""
    f = f32(float(x))
    while Fraction(float(f)) > x:
        f = np.nextafter(f, f32(-np.inf))
    while Fraction(float(np.nextafter(f, f32(np.inf)))) <= x:
        f = np.nextafter(f, f32(np.inf))
    if up and Fraction(float(f)) < x:
        f = np.nextafter(f, f32(np.inf))
    return f


def _rn(x: Fraction) -> np.float32:
    lo = _round_dir(x, False)
    if Fraction(float(lo)) == x:
        return lo
    hi = np.nextafter(lo, f32(np.inf))
    dl, dh = x - Fraction(float(lo)), Fraction(float(hi)) - x
    if dl != dh:
        return lo if dl < dh else hi
    return lo if (lo.view(np.uint32) & 1) == 0 else hi


def skip_params(R):
    a = -R
    rh = f32(a)
    rl = f32(a - float(rh))
    rb = _round_dir(Fraction(a) * Fraction(1, 2**54), True)
    return rh, rl, rb


def skip_fast(x, R, table):
    """The device's decision: skip + 1, or None where it takes FP64."""
    rh, rl, rb = skip_params(R)
    m = (x >> 11) + 1
    if m == 1 << 53:
        return 1
    A = qnlog_u57(m, table)
    if A <= 0:
        return None
    lz = 64 - A.bit_length()
    nn = A << lz
    Lh = f32((nn >> 40) * 2.0 ** (-17 - lz))
    Lm = f32(((nn >> 17) & 0x7FFFFF) * 2.0 ** (-40 - lz))
    p = f32(Lh * rh)
    e0 = _rn(Fraction(float(Lh)) * Fraction(float(rh)) - Fraction(float(p)))
    e = f32(e0 + f32(f32(Lh * rl) + f32(Lm * rh)))
    if not p < f32(2.0**44):
        return None
    fl = f32(math.floor(p))
    r = f32(f32(p - fl) + e)
    b = f32(f32(f32(f32(abs(r) + f32(1)) * f32(2.0**-23)) + f32(p * f32(2.0**-43))) + rb)
    klo = math.floor(_round_dir(Fraction(float(r)) - Fraction(float(b)), False))
    khi = math.floor(_round_dir(Fraction(float(r)) + Fraction(float(b)), True))
    if klo != khi:
        return None
    return int(fl) + klo + 1


def _definition_step(oracle, x, R):
    m = (x >> 11) + 1
    if m == 1 << 53:
        return 1
    q = oracle.log(m * 2.0**-53) * R
    return math.floor(q) + 1


def _near_integer_draws(oracle, R, count, rng):
    """Draws whose q lies within 2^-30 of an integer: U = exp(k / R) for an
    integer k, then the 53-bit draws next to it."""
    out = []
    for _ in range(count):
        k = int(rng.integers(1, max(2, min(10**9, int(40 * abs(R))))))
        u = math.exp(k / R)
        m = int(round(u * 2**53))
        for d in (-1, 0, 1):
            mm = min(max(m + d, 1), 2**53 - 1)
            out.append(((mm - 1) << 11) | int(rng.integers(0, 1 << 11)))
    return out


@pytest.mark.parametrize("p", [0.9, 0.3, 1e-2, 1e-4, 8.9e-7, 1e-9])
def test_guarded_skip_equals_definition(oracle, table, p):
    rng = np.random.default_rng(int(p * 1e9) + 7)
    R = 1.0 / oracle.log1p(-p)
    xs = [int(v) for v in rng.integers(0, 2**63, 3000, dtype=np.uint64)]
    xs += [int(v) << 1 for v in rng.integers(0, 2**63, 3000, dtype=np.uint64)]
    xs += _near_integer_draws(oracle, R, 1000, rng)
    decided = 0
    for x in xs:
        got = skip_fast(x, R, table)
        if got is None:
            continue
        decided += 1
        assert got == _definition_step(oracle, x, R), (p, x)
    # the guard decides nearly all random draws (the near-integer ones not)
    assert decided >= 6000 * 0.99, decided
