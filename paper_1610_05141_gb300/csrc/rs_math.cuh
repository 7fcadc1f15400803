// rs_math.cuh -- the sampler's own FP64 functions on the device.
//
// Built only from IEEE-exact operations (+ - * / sqrt, conversions, bit
// manipulation) and compiled with -fmad=false, so the results are the same
// bits on every IEEE machine that evaluates the same expressions in the same
// order.  The split deviates (Sec. 3: hypergeometric, Sec. 4.6: binomial)
// and the geometric skips of Bernoulli sampling (Sec. 4.7) depend on them.
#pragma once
#include "rs_common.cuh"

namespace rs {

RS_DEV double bits_to_double(uint64_t b) { return __longlong_as_double((long long)b); }
RS_DEV uint64_t double_to_bits(double d) { return (uint64_t)__double_as_longlong(d); }

// ln 2 split for exact range reduction: the high part keeps 32 significant
// bits so k * LN2_HI is exact for |k| < 2^21.
#define RS_RT2 bits_to_double(0x3ff6a09e667f3bcdull)      // nearest double to sqrt(2)
#define RS_LN2_HI bits_to_double(0x3fe62e42fee00000ull)
#define RS_LN2_LO bits_to_double(0x3dea39ef35793c76ull)
#define RS_INV_LN2 bits_to_double(0x3ff71547652b82feull)
#define RS_HL2PI bits_to_double(0x3fed67f1c864beb5ull)    // ln(2 pi) / 2
#define RS_HAT_D1 bits_to_double(0x3ffb72cd3f331398ull)   // 2 sqrt(2/e)
#define RS_HAT_D2 bits_to_double(0x3fecc3ebd3bc711aull)   // 3 - 2 sqrt(3/e)

// ln x for a normal x > 0: x = 2^e m with m in (sqrt2/2, sqrt2], and
// ln m = 2 atanh(s), s = (m-1)/(m+1), from the series sum s^(2i+1)/(2i+1)
// up to i = 12, evaluated by Horner's rule in z = s^2.
RS_DEV double dlog(double x) {
    const uint64_t bits = double_to_bits(x);
    int64_t e = (int64_t)((bits >> 52) & 0x7FF) - 1023;
    double m = bits_to_double((bits & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull);
    if (m > RS_RT2) {
        m = m * 0.5;
        e = e + 1;
    }
    const double f = m - 1.0;
    const double s = f / (2.0 + f);
    const double z = s * s;
    double R = 1.0 / 25.0;
    R = 1.0 / 23.0 + z * R;
    R = 1.0 / 21.0 + z * R;
    R = 1.0 / 19.0 + z * R;
    R = 1.0 / 17.0 + z * R;
    R = 1.0 / 15.0 + z * R;
    R = 1.0 / 13.0 + z * R;
    R = 1.0 / 11.0 + z * R;
    R = 1.0 / 9.0 + z * R;
    R = 1.0 / 7.0 + z * R;
    R = 1.0 / 5.0 + z * R;
    R = 1.0 / 3.0 + z * R;
    R = z * R;
    const double t = s + s * R;
    const double lm = t + t;
    const double de = (double)e;
    return de * RS_LN2_HI + (de * RS_LN2_LO + lm);
}

// ln(1+z), z > -1: with u = 1+z rounded, ln(u) * (z / (u-1)) cancels the
// rounding of u to first order (Goldberg 1991).
RS_DEV double dlog1p(double z) {
    const double u = 1.0 + z;
    if (u == 1.0) return z;
    return dlog(u) * (z / (u - 1.0));
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

// Tail of Stirling's series for ln x!: 1/(12x) - 1/(360x^3) + 1/(1260x^5) - 1/(1680x^7).
RS_DEV double stirling_tail(double x) {
    const double r = 1.0 / x;
    const double r2 = r * r;
    return r * (1.0 / 12.0 + r2 * (-1.0 / 360.0 + r2 * (1.0 / 1260.0 + r2 * (-1.0 / 1680.0))));
}

// ln x!; `tab` holds ln i! for i < 256 (built by lf_table_kernel).
RS_DEV double dlf(uint64_t x, const double* __restrict__ tab) {
    if (x < 256) return tab[x];
    const double X = (double)x;
    return (X + 0.5) * dlog(X) - X + RS_HL2PI + stirling_tail(X);
}

// ln x! - ln y! for x >= y without cancellation of the two large terms:
// (x+1/2) ln(x/y) + (x-y) ln y - (x-y) + tail(x) - tail(y), with
// ln(x/y) = ln1p((x-y)/y).  Short differences are summed directly.
RS_DEV double dlfdiff(uint64_t x, uint64_t y, const double* __restrict__ tab) {
    const uint64_t d = x - y;
    if (d == 0) return 0.0;
    if (x < 256) return tab[x] - tab[y];
    if (d <= 8) {
        double acc = 0.0;
        for (uint64_t i = y + 1; i <= x; ++i) acc = acc + dlog((double)i);
        return acc;
    }
    if (y < 256) return dlf(x, tab) - tab[y];
    const double X = (double)x, Y = (double)y, D = (double)d;
    return (X + 0.5) * dlog1p(D / Y) + D * dlog(Y) - D + (stirling_tail(X) - stirling_tail(Y));
}

// Signed ln x! - ln y!.
RS_DEV double dsd(uint64_t x, uint64_t y, const double* __restrict__ tab) {
    return x >= y ? dlfdiff(x, y, tab) : -dlfdiff(y, x, tab);
}

}  // namespace rs
