"""Pins for the oracle's own FP64 math (log, log1p, exp, ln x!, differences of
ln x!) against high-precision values from mpmath, and of its stored constants
against their mathematical definitions."""
import math
import os
import re
import struct

import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")
mpmath.mp.prec = 160

ORACLE_SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "rs_oracle.c")


def _bits_to_double(b):
    return struct.unpack("<d", struct.pack("<Q", b))[0]


def _ulp(x):
    x = abs(float(x))
    return math.ulp(x) if x != 0 else 2.0**-1074


def _ulp_err(got, exact):
    return abs(mpmath.mpf(got) - exact) / mpmath.mpf(_ulp(exact))


def test_constants_match_definitions():
    """Each stored hex constant is the double its comment defines."""
    src = open(ORACLE_SRC).read()
    consts = dict(re.findall(r"#define (\w+)\s+from_bits\((0x[0-9a-f]+)ull\)", src))
    ln2 = mpmath.log(2)
    want = {
        "LN2_LO": None,   # checked below from LN2_HI
        "INV_LN2": 1 / ln2,
        "HL2PI": mpmath.log(2 * mpmath.pi) / 2,
        "HAT_D1": 2 * mpmath.sqrt(2 / mpmath.e),
        "HAT_D2": 3 - 2 * mpmath.sqrt(3 / mpmath.e),
    }
    got = {k: _bits_to_double(int(v, 16)) for k, v in consts.items()}
    for k, w in want.items():
        if w is not None:
            assert got[k] == float(w), k
    # LN2_HI: ln 2 truncated to 32 significant bits (exact product with any
    # integer k of up to 21 bits); LN2_LO: the rounded remainder.
    hi = got["LN2_HI"]
    m, e = math.frexp(hi)
    assert (m * 2**32) == int(m * 2**32)
    assert mpmath.mpf(hi) <= ln2 < mpmath.mpf(hi) + mpmath.mpf(2) ** (e - 32)
    assert got["LN2_LO"] == float(ln2 - mpmath.mpf(hi))


def _log_args():
    rng = np.random.default_rng(1)
    xs = [1.0, 2.0, 0.5, math.sqrt(2), float.fromhex("0x1.6a09e667f3bcdp+0"), float.fromhex("0x1.6a09e667f3bcep+0"),
          1 + 2**-52, 1 - 2**-53, 2**-1022, 2**1023, 3.0, 10.0, 1e-300, 1e300, 2.0**-53, 1.0 - 2**-30]
    xs += list(np.exp(rng.uniform(-700, 700, 3000)))
    xs += list(1 + rng.uniform(-0.3, 0.45, 2000))
    xs += [float(i) for i in range(1, 2000)]
    xs += list(rng.integers(1, 2**62, 1000).astype(float))
    return xs


def test_log_accuracy(oracle):
    """or_log within 2 ulp of ln x on normals spanning the exponent range."""
    worst = 0
    for x in _log_args():
        got = oracle.log(x)
        exact = mpmath.log(mpmath.mpf(x))
        if exact == 0:
            assert got == 0.0
            continue
        worst = max(worst, _ulp_err(got, exact))
    assert worst <= 2, worst


def test_log_table(oracle):
    """Each interval of the logarithm's table: inv is the double nearest 1/c
    for the interval's centre c, hi + lo is -ln(inv) to double-double
    accuracy, hi is -ln(inv) rounded; the intervals next to 1 use c = 1."""
    with mpmath.workprec(300):
        for i in range(128):
            inv, hi, lo = oracle.log_table_entry(i)
            if i in (0, 127):
                assert (inv, hi, lo) == (1.0, 0.0, 0.0)
                continue
            c = 1 + (2 * i + 1) / 256
            assert inv == 1.0 / c
            exact = -mpmath.log(mpmath.mpf(inv))
            assert abs(mpmath.mpf(hi) + mpmath.mpf(lo) - exact) <= abs(exact) * mpmath.mpf(2) ** -100, i
            assert hi == float(exact), i
            assert abs(lo) <= math.ulp(hi) / 2


def test_log_special_values(oracle):
    assert oracle.log(1.0) == 0.0
    assert oracle.log(2.0) == math.log(2.0)
    assert oracle.log(0.5) == -math.log(2.0)


def test_log1p_accuracy(oracle):
    """Goldberg's log1p within 3 ulp, including |z| far below 2^-53."""
    rng = np.random.default_rng(2)
    zs = [1e-300, -1e-300, 1e-20, -1e-17, 2**-53, -2**-54, 1e-10, -0.5, -0.25, 0.5, 1.0, 1e10, -1 + 2**-53]
    zs += list(-rng.uniform(0, 0.5, 1000)) + list(np.exp(rng.uniform(-60, 25, 1500)))
    zs += list(-np.exp(rng.uniform(-60, math.log(0.999), 1000)))
    worst = 0
    for z in zs:
        got = oracle.log1p(z)
        exact = mpmath.log1p(mpmath.mpf(z))
        worst = max(worst, _ulp_err(got, exact))
    assert worst <= 3, worst


def test_recip_accuracy(oracle):
    """1/x from a single-precision seed and two Newton steps: within 1 ulp
    of the exact reciprocal over the range it serves (uniforms down to 2^-53,
    integers up to 2^64)."""
    rng = np.random.default_rng(6)
    xs = [1.0, 2.0, 3.0, 0.1, 2.0**-53, 2.0**64, 1 + 2**-52, 2 - 2**-52, 12345.0, 2.0**32 - 1]
    xs += list(np.exp(rng.uniform(math.log(2.0**-53), math.log(2.0**64), 3000)))
    xs += [float(v) for v in rng.integers(1, 2**62, 1000)]
    worst = 0
    for x in xs:
        got = oracle.recip(x)
        worst = max(worst, _ulp_err(got, 1 / mpmath.mpf(x)))
    assert worst <= 1, worst
    # the seed alone is far from that: the Newton steps are doing the work
    assert any(float(np.float32(1) / np.float32(x)) != oracle.recip(x) for x in xs[10:50])


def test_log1p_pos_accuracy(oracle):
    """ln(1 + z), z >= 0, by the table logarithm of the rounded 1 + z plus
    the exact rounding error over 1 + z: within 2 ulp from z = 2^-70 (where
    1 + z rounds to 1) to z = 2^40."""
    rng = np.random.default_rng(7)
    zs = [0.0, 2.0**-70, 2.0**-53, 2.0**-52, 1e-10, 2.0**-7, 0.5, 1.0, 3.0, 2.0**40]
    zs += list(np.exp(rng.uniform(math.log(2.0**-70), math.log(2.0**40), 4000)))
    worst = 0
    for z in zs:
        got = oracle.log1p_pos(z)
        if z == 0.0:
            assert got == 0.0
            continue
        worst = max(worst, _ulp_err(got, mpmath.log1p(mpmath.mpf(z))))
    assert worst <= 2, worst


def test_exp_accuracy(oracle):
    """or_exp within 2 ulp on its domain [-708, 0]."""
    rng = np.random.default_rng(3)
    xs = [0.0, -1e-300, -1e-17, -0.5, -1.0, -math.log(2), -40.0, -44.0, -700.0, -708.0]
    xs += list(-rng.uniform(0, 708, 2000)) + list(-np.exp(rng.uniform(-40, 0, 1000)))
    worst = 0
    for x in xs:
        got = oracle.exp(x)
        exact = mpmath.exp(mpmath.mpf(x))
        worst = max(worst, _ulp_err(got, exact))
    assert worst <= 2, worst


def _lf_exact(x):
    return mpmath.loggamma(mpmath.mpf(x) + 1)


def test_lf_accuracy(oracle):
    """ln x! to a relative error below 1e-14 (table below 256, Stirling above)."""
    rng = np.random.default_rng(4)
    xs = list(range(0, 600)) + [int(v) for v in rng.integers(256, 2**62, 500)]
    xs += [int(v) for v in np.exp(rng.uniform(math.log(256), math.log(2**62), 500))]
    for x in xs:
        got = oracle.lf(x)
        exact = _lf_exact(x)
        if x <= 1:
            assert got == 0.0
            continue
        assert abs(mpmath.mpf(got) - exact) <= 1e-14 * abs(exact), x


def test_lfdiff_accuracy(oracle):
    """ln x! - ln y! to a relative error below 1e-13 of the difference, for
    every branch: table, small y, and the cancellation-free form (short differences included)
    at x, y up to 2^62 (where a plain difference of ln x! would lose it)."""
    rng = np.random.default_rng(5)
    pairs = [(5, 5), (10, 3), (255, 0), (300, 295), (300, 292), (300, 291), (1000, 255), (1000, 10),
             (257, 256), (10**6 + 1, 10**6), (10**6 + 8, 10**6), (2**40 + 1, 2**40), (2**61 + 3, 2**61)]
    for _ in range(600):
        y = int(np.exp(rng.uniform(0, math.log(2**61))))
        d = int(np.exp(rng.uniform(0, math.log(max(2, min(y, 2**40))))))
        pairs.append((y + d, y))
    for x, y in pairs:
        got = oracle.lfdiff(x, y)
        exact = _lf_exact(x) - _lf_exact(y)
        if x == y:
            assert got == 0.0
            continue
        assert abs(mpmath.mpf(got) - exact) <= 1e-13 * abs(exact), (x, y, got, float(exact))
        assert oracle.sd(x, y) == got and oracle.sd(y, x) == -got


def test_sd_fixed_accuracy(oracle):
    """The ratio-of-uniforms differences with the node's ln P supplied: ln P! -
    ln Q! to 1e-13 of the difference on every branch (short differences
    included), with P the larger or the smaller end, and equal to or_sd where
    no logarithm is reused."""
    rng = np.random.default_rng(8)
    pairs = [(5, 5), (10, 3), (3, 10), (255, 0), (0, 255), (300, 295), (295, 300), (1000, 255), (255, 1000),
             (1000, 10), (10, 1000), (0, 7)]
    for _ in range(400):
        y = int(np.exp(rng.uniform(0, math.log(2**61))))
        d = int(np.exp(rng.uniform(0, math.log(max(2, min(y, 2**40))))))
        pairs += [(y + d, y), (y, y + d)]
    for P, Q in pairs:
        lnP = oracle.log(float(max(P, 1)))
        got = oracle.sd_fixed(P, Q, lnP)
        exact = _lf_exact(P) - _lf_exact(Q)
        if P == Q:
            assert got == 0.0
            continue
        assert abs(mpmath.mpf(got) - exact) <= 1e-13 * abs(exact), (P, Q, got, float(exact))
        if max(P, Q) < 256:
            assert got == oracle.sd(P, Q)

