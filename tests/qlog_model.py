"""Test infrastructure: a model of the CUDA path's fixed-point logarithm
(rs_math.cuh qnlog_u57) in Python integers, operation for operation, with
its table built as the device builds it, for the tests of the guards that
use it.  Not the oracle: the oracle's logarithm is FP64."""
import os
import re

import mpmath

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MATH = os.path.join(ROOT, "paper_1610_05141_gb300", "csrc", "rs_math.cuh")
M64 = 1 << 64


def _const(name):
    src = open(MATH).read()
    m = re.search(r"constexpr (?:int64_t|uint32_t) %s = (-?\d+)(?:ll|u);" % name, src)
    assert m, name
    return int(m.group(1))


H = {k: _const("kQh%d" % k) for k in range(3, 7)}
LN2Q57 = _const("kLn2Q57")
LN2FRAC32 = _const("kLn2Q57Frac32")
INTERVALS = 512


def _mulhi(a, b):   # unsigned high 64 bits
    return (a * b) >> 64


def make_table():
    """The fixed-point table: inv = ceil(2^64 / c) for the left ends
    c = 1 + i/512, and -ln(inv 2^-64) rounded to Q63 (the device builds it
    from a double-double value; within the same half unit)."""
    mpmath.mp.dps = 50
    inv_q, ln_q = {}, {}
    for i in range(1, INTERVALS):
        inv_q[i] = -(-(1 << 73) // (512 + i))
        assert inv_q[i] * (512 + i) >= 1 << 73 and inv_q[i] < M64
        ln_q[i] = int(mpmath.nint(-mpmath.log(mpmath.mpf(inv_q[i]) / M64) * 2**63))
    return inv_q, ln_q


def qnlog_u57(m, table):
    inv_q, ln_q = table
    t = m.bit_length() - 1
    F = m << (63 - t)
    i = (F >> 54) & (INTERVALS - 1)
    lninv = 0
    if i == 0:
        r64 = (F - (1 << 63)) << 1
    else:
        r64 = (_mulhi(F, inv_q[i]) - (1 << 63)) << 1
        lninv = ln_q[i]
    assert 0 <= r64 < 1 << 55
    r2 = _mulhi(r64, r64)
    r3 = _mulhi(r2, r64)
    r32 = r64 >> 32
    h = H[5] - ((r32 * H[6]) >> 32)
    h = H[4] - ((r32 * h) >> 32)
    h = H[3] - ((r32 * h) >> 32)
    l1p = r64 - (r2 >> 1) + _mulhi(r3, h << 32)
    lnf = lninv + (l1p >> 1)
    assert lnf < 1 << 64
    e = 53 - t
    return e * LN2Q57 + ((e * LN2FRAC32) >> 32) - (lnf >> 6)
