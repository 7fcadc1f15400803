// rs_math.cuh -- the sampler's own FP64 functions on the device.
//
// Built only from IEEE-exact operations (+ - * / sqrt, explicit fused
// multiply-add, conversions, bit manipulation) and compiled with -fmad=false,
// so the results are the same bits on every IEEE machine that evaluates the
// same expressions in the same order.  The split deviates (Sec. 3: hypergeometric, Sec. 4.6: binomial)
// and the geometric skips of Bernoulli sampling (Sec. 4.7) depend on them.
#pragma once
#include "rs_common.cuh"

namespace rs {

RS_DEV double bits_to_double(uint64_t b) { return __longlong_as_double((long long)b); }
RS_DEV uint64_t double_to_bits(double d) { return (uint64_t)__double_as_longlong(d); }

// ln 2 split for exact range reduction: the high part keeps 32 significant
// bits so k * LN2_HI is exact for |k| < 2^21.
#define RS_LN2_HI bits_to_double(0x3fe62e42fee00000ull)
#define RS_LN2_LO bits_to_double(0x3dea39ef35793c76ull)
#define RS_INV_LN2 bits_to_double(0x3ff71547652b82feull)
#define RS_HL2PI bits_to_double(0x3fed67f1c864beb5ull)    // ln(2 pi) / 2
#define RS_HAT_D1 bits_to_double(0x3ffb72cd3f331398ull)   // 2 sqrt(2/e)
#define RS_HAT_D2 bits_to_double(0x3fecc3ebd3bc711aull)   // 3 - 2 sqrt(3/e)

// Double-double arithmetic for building the table: error-free sums (Knuth)
// and products (fused multiply-add), then renormalization.
struct DD {
    double hi, lo;
};
RS_DEV DD dd_fast2(double a, double b) {
    const double s = a + b;
    return DD{s, b - (s - a)};
}
RS_DEV DD dd_two_sum(double a, double b) {
    const double s = a + b;
    const double bb = s - a;
    return DD{s, (a - (s - bb)) + (b - bb)};
}
RS_DEV DD dd_add(DD a, DD b) {
    const DD s = dd_two_sum(a.hi, b.hi);
    const double e = s.lo + (a.lo + b.lo);
    return dd_fast2(s.hi, e);
}
RS_DEV DD dd_mul(DD a, DD b) {
    const double p = a.hi * b.hi;
    double e = __fma_rn(a.hi, b.hi, -p);
    e = e + (a.hi * b.lo + a.lo * b.hi);
    return dd_fast2(p, e);
}
// a / b to double-double precision: three quotient digits.
RS_DEV DD dd_div(DD a, DD b) {
    const double q1 = a.hi / b.hi;
    DD t = dd_mul(b, DD{q1, 0.0});
    DD r = dd_add(a, DD{-t.hi, -t.lo});
    const double q2 = r.hi / b.hi;
    t = dd_mul(b, DD{q2, 0.0});
    r = dd_add(r, DD{-t.hi, -t.lo});
    const double q3 = r.hi / b.hi;
    const DD q = dd_fast2(q1, q2);
    return dd_add(q, DD{q3, 0.0});
}

// Entry i of the logarithm table: interval i of [1, 2) (width 2^-7) has
// centre c = 1 + (2i+1)/256 and inv = RN(1/c); -ln(inv) = -2 atanh(s),
// s = (inv-1)/(inv+1), summed in double-double to s^71/71 (|s| <= 1/3).
// Intervals 0 and 127 use c = 1 (see dlog).
// -ln(x) for x = hi + lo in (1/2, 1] in double-double: -2 atanh(s),
// s = (x - 1)/(x + 1) (|s| < 1/3), summed to s^71/71.
RS_DEV DD dd_neg_log(DD x) {
    const DD s = dd_div(dd_add(x, DD{-1.0, 0.0}), dd_add(x, DD{1.0, 0.0}));
    const DD s2 = dd_mul(s, s);
    DD term = s, sum = s;
    for (int k = 1; k < 36; ++k) {
        term = dd_mul(term, s2);
        sum = dd_add(sum, dd_div(term, DD{(double)(2 * k + 1), 0.0}));
    }
    return DD{-2.0 * sum.hi, -2.0 * sum.lo};
}

// Entry i of the fixed-point table (i = 1 .. 511; entry 0 is unused):
// inv = ceil(2^64 / c) = ceil(2^73 / (512 + i)) exactly, and -ln(inv 2^-64)
// in Q63 from its double-double value (the high part times 2^63 is an
// integer, as the value exceeds 2^-10; the low part is rounded: error at
// most half a unit).
RS_DEV void build_qlog_entry(int i, double* tab) {
    uint64_t* q = reinterpret_cast<uint64_t*>(tab);
    if (i == 0) {
        q[kTabQInv] = 0;
        q[kTabQLn] = 0;
        return;
    }
    const unsigned __int128 num = (unsigned __int128)1 << 73;
    const uint64_t d = 512 + (uint64_t)i;
    const uint64_t inv = (uint64_t)((num + d - 1) / d);
    const double hi = __ull2double_rn(inv) * 0x1p-64;   // inv 2^-64 = hi + lo exactly
    const double lo = (double)(int64_t)(inv - __double2ull_rn(hi * 0x1p64)) * 0x1p-64;
    const DD v = dd_neg_log(DD{hi, lo});
    q[kTabQInv + i] = inv;
    q[kTabQLn + i] = (uint64_t)(__double2ll_rn(v.hi * 0x1p63) + __double2ll_rn(v.lo * 0x1p63));
}

RS_DEV void build_log_entry(int i, double* tab) {
    if (i == 0 || i == 127) {
        tab[kTabInv + i] = 1.0;
        tab[kTabHi + i] = 0.0;
        tab[kTabLo + i] = 0.0;
        return;
    }
    const double c = 1.0 + (double)(2 * i + 1) / 256.0;
    const double inv = 1.0 / c;
    const DD s = dd_div(DD{inv - 1.0, 0.0}, dd_two_sum(inv, 1.0));
    const DD s2 = dd_mul(s, s);
    DD term = s, sum = s;
    for (int k = 1; k < 36; ++k) {
        term = dd_mul(term, s2);
        sum = dd_add(sum, dd_div(term, DD{(double)(2 * k + 1), 0.0}));
    }
    tab[kTabInv + i] = inv;
    tab[kTabHi + i] = -(2.0 * sum.hi);
    tab[kTabLo + i] = -(2.0 * sum.lo);
}

// ln x for a normal x > 0: x = 2^e m, m in [1, 2); the top 7 bits of m pick
// an interval with centre c and inv = RN(1/c), and ln m = -ln(inv) +
// ln(1 + r), r = m inv - 1 (one fused multiply-add, |r| <= 2^-8), ln(1 + r)
// by its Taylor polynomial to r^8/8 (Horner with fused multiply-adds).  The
// two intervals next to 1 use c = 1 and r = m - 1 (or m/2 - 1 with e + 1),
// exact, so that ln x near 1 keeps its relative accuracy; there |r| <= 2^-7.
RS_DEV double dlog(double x, const double* __restrict__ tab) {
    const uint64_t bits = double_to_bits(x);
    int64_t e = (int64_t)((bits >> 52) & 0x7FF) - 1023;
    const int i = (int)((bits >> 45) & 0x7F);
    double m = bits_to_double((bits & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull);
    double r;
    if (i == 127) {
        m = m * 0.5;
        e = e + 1;
        r = m - 1.0;
    } else if (i == 0) {
        r = m - 1.0;
    } else {
        r = __fma_rn(m, __ldg(tab + kTabInv + i), -1.0);
    }
    double q = -1.0 / 8.0;
    q = __fma_rn(q, r, 1.0 / 7.0);
    q = __fma_rn(q, r, -1.0 / 6.0);
    q = __fma_rn(q, r, 1.0 / 5.0);
    q = __fma_rn(q, r, -1.0 / 4.0);
    q = __fma_rn(q, r, 1.0 / 3.0);
    q = __fma_rn(q, r, -0.5);
    const double p = __fma_rn(r * r, q, r);
    const double de = (double)e;
    return (de * RS_LN2_HI + __ldg(tab + kTabHi + i)) + ((de * RS_LN2_LO + __ldg(tab + kTabLo + i)) + p);
}

// -ln U in fixed point for U = m 2^-53, 1 <= m < 2^53 (the uniforms of the
// geometric skips): the result times 2^-57 is within 2^-55 of -ln U.  Only
// integer operations, all unsigned: m = 2^t f with f in [1, 2) as a Q63
// integer F; the top 9 bits of f pick an interval with left end c and
// inv = ceil(2^64/c) >= 1/c, so that r = f inv - 1 is in [0, 2^-9) (one high
// product, truncated by less than 2^-63; interval 0 takes r = f - 1 exactly);
// ln(1 + r) = r - r^2/2 + r^3 h with h = 1/3 - r/4 + r^2/5 - r^3/6, r^2 and
// r^3 by 64-bit high products (Q64) and h by 32-bit ones (Q32, error below
// 1.5 2^-32, times r^3 < 2^-27); the series stops before r^7/7 < 2^-65.
// Then -ln U = (53 - t) ln 2 - ln(inv) - ln(1 + r).  In units of 2^-57:
// ln(1 + r) within 2^-1.2, the table's half unit of 2^-63 and the shift from
// Q63 to Q57 below 1, and (53 - t) ln 2 with ln 2 = (A + phi) 2^-57, A an
// integer taken exactly and phi in Q32 truncated after the product (below
// 1 + 53 2^-33): in all below 2.1 units, 2^-55.9.
constexpr uint32_t kQh3 = 1431655765u;   // round(2^32 / 3)
constexpr uint32_t kQh4 = 1073741824u;   // 2^32 / 4
constexpr uint32_t kQh5 = 858993459u;    // round(2^32 / 5)
constexpr uint32_t kQh6 = 715827883u;    // round(2^32 / 6)
constexpr int64_t kLn2Q57 = 99893036290645747ll;   // floor(ln 2 * 2^57)
constexpr int64_t kLn2Q57Frac32 = 1469302631ll;    // the rest of ln 2 * 2^57, times 2^32, rounded
RS_DEV int64_t qnlog_u57(uint64_t m, const double* __restrict__ tab) {
    const int t = 63 - __clzll((long long)m);
    const uint64_t F = m << (63 - t);
    const int i = (int)((F >> 54) & (kQLogIntervals - 1));
    uint64_t r64;   // r in Q64, below 2^55
    uint64_t lninv = 0;
    if (i == 0) {
        r64 = (F - (1ull << 63)) << 1;
    } else {
        const uint64_t inv = (uint64_t)__double_as_longlong(__ldg(tab + kTabQInv + i));
        r64 = (__umul64hi(F, inv) - (1ull << 63)) << 1;
        lninv = (uint64_t)__double_as_longlong(__ldg(tab + kTabQLn + i));
    }
    const uint64_t r2 = __umul64hi(r64, r64);   // r^2, Q64
    const uint64_t r3 = __umul64hi(r2, r64);    // r^3, Q64
    const uint32_t r32 = (uint32_t)(r64 >> 32);
    uint32_t h = kQh5 - __umulhi(r32, kQh6);
    h = kQh4 - __umulhi(r32, h);
    h = kQh3 - __umulhi(r32, h);
    const uint64_t l1p = r64 - (r2 >> 1) + __umul64hi(r3, (uint64_t)h << 32);   // ln(1 + r), Q64
    const uint64_t lnf = lninv + (l1p >> 1);                                      // ln f, Q63
    const int64_t e = 53 - t;
    return e * kLn2Q57 + ((e * kLn2Q57Frac32) >> 32) - (int64_t)(lnf >> 6);
}

// ln(1+z), z > -1: with u = 1+z rounded, ln(u) * (z / (u-1)) cancels the
// rounding of u to first order (Goldberg 1991).
RS_DEV double dlog1p(double z, const double* __restrict__ tab) {
    const double u = 1.0 + z;
    if (u == 1.0) return z;
    return dlog(u, tab) * (z / (u - 1.0));
}

// 1/x for a positive x in [2^-60, 2^100]: the single-precision quotient of
// x rounded to single precision as the seed (relative error below 2^-23),
// then two Newton steps r <- r + r (1 - x r) with fused multiply-adds;
// within about one ulp of 1/x.  Used where a correctly rounded quotient is
// not needed (Stirling's tail, the argument of ln(1 + z), the ratio-of-
// uniforms abscissa): an FP64 division costs several times as many FP64
// instructions.
RS_DEV double drecip(double x) {
    double r = (double)__fdiv_rn(1.0f, __double2float_rn(x));
    double e = __fma_rn(-x, r, 1.0);
    r = __fma_rn(r, e, r);
    e = __fma_rn(-x, r, 1.0);
    return __fma_rn(r, e, r);
}

// ln(1 + z) for z >= 0 without a division: u = 1 + z rounded, e = (1 + z) - u
// exactly (Knuth's two-sum), ln(1 + z) = ln u + e/u to 2^-106 relative
// (|e/u| <= 2^-53), e/u taken as e times a single-precision 1/u.  The
// logarithm of u is passed in (lnu = dlog(u)) so that callers may evaluate
// it elsewhere.
RS_DEV double log1p_pos_u(double z) { return 1.0 + z; }
RS_DEV double log1p_pos_finish(double z, double lnu) {
    const double u = 1.0 + z;
    const double bb = u - 1.0;
    const double e = (1.0 - (u - bb)) + (z - bb);
    return lnu + e * (double)__fdiv_rn(1.0f, __double2float_rn(u));
}
RS_DEV double dlog1p_pos(double z, const double* __restrict__ tab) {
    return log1p_pos_finish(z, dlog(log1p_pos_u(z), tab));
}

// e^x for x in [-708, 0]: x = k ln2 + r with |r| <= ln2/2, e^r from its
// Taylor polynomial of degree 13, times 2^k assembled from the exponent bits.
RS_DEV double dexp(double x) {
    const int64_t k = (int64_t)floor(x * RS_INV_LN2 + 0.5);
    const double dk = (double)k;
    const double r = (x - dk * RS_LN2_HI) - dk * RS_LN2_LO;
    double p = 1.0 / 6227020800.0;
    p = 1.0 / 479001600.0 + r * p;
    p = 1.0 / 39916800.0 + r * p;
    p = 1.0 / 3628800.0 + r * p;
    p = 1.0 / 362880.0 + r * p;
    p = 1.0 / 40320.0 + r * p;
    p = 1.0 / 5040.0 + r * p;
    p = 1.0 / 720.0 + r * p;
    p = 1.0 / 120.0 + r * p;
    p = 1.0 / 24.0 + r * p;
    p = 1.0 / 6.0 + r * p;
    p = 1.0 / 2.0 + r * p;
    p = 1.0 + r * p;
    p = 1.0 + r * p;
    return p * bits_to_double((uint64_t)(k + 1023) << 52);
}

// Tail of Stirling's series for ln x!: 1/(12x) - 1/(360x^3) + 1/(1260x^5) -
// 1/(1680x^7), from r = 1/x (drecip).
RS_DEV double stirling_tail(double r) {
    const double r2 = r * r;
    return r * (1.0 / 12.0 + r2 * (-1.0 / 360.0 + r2 * (1.0 / 1260.0 + r2 * (-1.0 / 1680.0))));
}

// ln x!; `tab` holds ln i! for i < 256 (built by lf_table_kernel).
RS_DEV double dlf(uint64_t x, const double* __restrict__ tab) {
    if (x < 256) return tab[x];
    const double X = (double)x;
    return (X + 0.5) * dlog(X, tab) - X + RS_HL2PI + stirling_tail(drecip(X));
}

// ln x! - ln y! for x >= y without cancellation of the two large terms:
// (x+1/2) ln(x/y) + (x-y) ln y - (x-y) + tail(x) - tail(y), with
// ln(x/y) = ln(1 + (x-y)/y), for every x - y once y >= 256.
RS_DEV double dlfdiff(uint64_t x, uint64_t y, const double* __restrict__ tab) {
    const uint64_t d = x - y;
    if (d == 0) return 0.0;
    if (x < 256) return tab[x] - tab[y];
    if (y < 256) return dlf(x, tab) - tab[y];
    const double X = (double)x, Y = (double)y, D = (double)d;
    const double rY = drecip(Y);
    const double lp = dlog1p_pos(D * rY, tab);
    return (X + 0.5) * lp + D * dlog(Y, tab) - D + (stirling_tail(drecip(X)) - stirling_tail(rY));
}

// Signed ln x! - ln y!.
RS_DEV double dsd(uint64_t x, uint64_t y, const double* __restrict__ tab) {
    return x >= y ? dlfdiff(x, y, tab) : -dlfdiff(y, x, tab);
}

// ln P! - ln Q! for the ratio-of-uniforms tests, P fixed for the node and
// lnP = dlog(max(P, 1)) computed once: dlfdiff's branches on (max, min),
// with ln of the larger argument = lnP when that is P, and ln of the smaller
// one in the cancellation-free form = lnP when that is P, else ln P -
// ln(P/Q).
RS_DEV double dsd_fixed(uint64_t P, uint64_t Q, double lnP, const double* __restrict__ tab) {
    const bool p_big = P >= Q;
    const uint64_t x = p_big ? P : Q, y = p_big ? Q : P, d = x - y;
    double v;
    if (d == 0) return 0.0;
    if (x < 256) {
        v = tab[x] - tab[y];
    } else {
        const double X = (double)x;
        if (y < 256) {
            const double lx = p_big ? lnP : dlog(X, tab);
            v = ((X + 0.5) * lx - X + RS_HL2PI + stirling_tail(drecip(X))) - tab[y];
        } else {
            const double Y = (double)y, D = (double)d;
            const double rY = drecip(Y);
            const double lp = dlog1p_pos(D * rY, tab);
            const double ly = p_big ? lnP - lp : lnP;
            v = (X + 0.5) * lp + D * ly - D + (stirling_tail(drecip(X)) - stirling_tail(rY));
        }
    }
    return p_big ? v : -v;
}
RS_DEV double log_fixed(uint64_t P, const double* __restrict__ tab) { return dlog((double)(P > 0 ? P : 1), tab); }

// ---------------------------------------------------------------------------
// Single-precision guard of the ratio-of-uniforms test.
//
// The test accepts a trial when 2 ln U <= T, T a signed sum of ln x! - ln y!
// differences evaluated in FP64 as above.  The guard evaluates both sides in
// single precision together with a bound on their error and decides only
// when the two sides are further apart than the bound; otherwise the trial
// is evaluated in FP64 exactly as the definition states.  So the outcome is
// that of the FP64 test bit for bit, and the FP64 pipe (about 1/80 of the
// single-precision rate on GB300) is used only by the trials near the
// boundary.
//
// Error bound (u = 2^-24).  flfdiff returns F and a magnitude m (a sum of
// the absolute values of the terms it combines, each at least as large as
// that term) with |F - (ln x! - ln y!)| <= 12 u m: its inputs are rounded
// once to single precision, each product, reciprocal and sum adds u of its
// result, single-precision logf and log1pf are within 1 ulp (CUDA's
// documented bounds; ln(1 + z) then keeps 6 u relative), the table entries
// are ln i! rounded once, and the Stirling terms past 1/(12x) (below
// 1/(360 x^3) <= 2e-10 for x >= 256) and the rounding of ln(2 pi)/2 are
// covered by the constants added to m.  A sum of four such terms is within
// 15 u of the summed magnitudes; the left side 2 ln U within 4 u (|2 ln U|
// + 1); the FP64 values of the definition within 2^-45 of the same
// magnitudes.  The guard takes kGuardUlps = 24 times u times the summed
// magnitudes (plus |2 ln U| + 2) as its margin.
constexpr float kGuardUlps = 24.0f;
constexpr float kGuardEps = kGuardUlps * 5.9604645e-8f;   // kGuardUlps 2^-24

// ln x! - ln y! for x >= y in single precision; *mag as above.  tf holds
// ln i! (i < 256) rounded to single precision.
RS_DEV float flfdiff(uint64_t x, uint64_t y, const float* __restrict__ tf, float* mag) {
    const uint64_t d = x - y;
    if (d == 0) {
        *mag = 0.0f;
        return 0.0f;
    }
    if (x < 256) {
        const float a = tf[x], b = tf[y];
        *mag = a + b;
        return a - b;
    }
    const float X = __ull2float_rn(x), D = __ull2float_rn(d);
    if (y < 256) {
        // Stirling: (x + 1/2) ln x - x + ln(2 pi)/2 + 1/(12 x), less ln y!
        const float A = (X + 0.5f) * logf(X);
        const float ty = tf[y];
        *mag = A + X + ty + 2.0f;
        return ((A - X) + (0.9189385f + 0.083333336f * __frcp_rn(X))) - ty;
    }
    // (x + 1/2) ln(1 + d/y) + d ln y - d + (1/(12x) - 1/(12y))
    const float Y = __ull2float_rn(y);
    const float rY = __frcp_rn(Y);
    const float A = (X + 0.5f) * log1pf(D * rY);
    const float B = D * logf(Y);
    *mag = A + B + D + 1.0f;
    return ((A + B) - D) + 0.083333336f * (__frcp_rn(X) - rY);
}

// Signed ln P! - ln Q!.
RS_DEV float fsd(uint64_t P, uint64_t Q, const float* __restrict__ tf, float* mag) {
    return P >= Q ? flfdiff(P, Q, tf, mag) : -flfdiff(Q, P, tf, mag);
}

// Single-precision guard of the ratio-of-uniforms abscissa.  The definition
// evaluates X = alpha + h (V - 1/2) / U in FP64; a trial is rejected when X
// lies outside [0, top), else its candidate is k = floor(X).  alpha_f and
// h_f are the node's parameters from the same formulas in single precision:
// each input rounded once (relative u = 2^-24), each product, reciprocal and
// sum once, sqrtf correctly rounded, so alpha_f is within 7 u alpha and h_f
// within 14 u h; with Uf and Vf the uniforms rounded once, |X_f - X| <=
// u (8 alpha + 11 h / U), and the FP64 X is within 2^-50 (alpha + h / U) of
// the same value.  The guard takes 16 u (alpha + h / U + 1) as its margin
// and settles the trial only when no boundary (0, top, an integer) lies
// within it.  Returns 1 (X in [0, top), *k = floor(X)), -1 (outside:
// rejected) or 0 (too close to call).
constexpr float kXGuardEps = 16.0f * 5.9604645e-8f;
RS_DEV int guard_abscissa(float alpha_f, float h_f, float top_f, float Uf, float Vf, uint64_t* k) {
    const float hu = h_f * __frcp_rn(Uf);
    const float X = alpha_f + hu * (Vf - 0.5f);
    const float E = kXGuardEps * ((alpha_f + hu) + 1.0f);
    // top_f is the integer top rounded once to single precision
    const float top_lo = top_f * (1.0f - 2.4e-7f), top_hi = top_f * (1.0f + 2.4e-7f);
    if (X + E < 0.0f || X - E >= top_hi) return -1;
    if (X - E < 0.0f || X + E >= top_lo) return 0;
    const float lo = floorf(X - E);
    if (lo != floorf(X + E)) return 0;
    *k = (uint64_t)lo;
    return 1;
}

// The uniforms of a 64-bit value rounded once to single precision: U in
// (0, 1] and V in [0, 1) of rs_rng.cuh, without FP64 operations.
RS_DEV float u_open_f(uint64_t x) { return __ull2float_rn((x >> 11) + 1) * 1.1102230e-16f; }
RS_DEV float v_closed_f(uint64_t x) { return __ull2float_rn(x >> 11) * 1.1102230e-16f; }

// The guard's decision for 2 ln U against T = tsum (magnitude tmag):
// 1 accept, -1 reject, 0 too close to call.
RS_DEV int guard_decide(float Uf, float tsum, float tmag) {
    const float L = 2.0f * logf(Uf);
    const float margin = kGuardEps * ((tmag + fabsf(L)) + 2.0f);
    if (L + margin < tsum) return 1;
    if (L - margin > tsum) return -1;
    return 0;
}

}  // namespace rs
