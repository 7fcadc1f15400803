// rs_ff.cuh -- a second guard of the split deviates' ratio-of-uniforms
// trials, in float-float arithmetic (a value is an unevaluated sum hi + lo of
// two singles, about 48 significant bits) with fixed-point logarithms.
//
// The definition (Sec. 3.1 and 4.6 as §8(c) reads them) evaluates each trial
// in FP64: the abscissa X = alpha + h (V - 1/2) / U and the test
// 2 ln U <= T, T a signed sum of ln x! - ln y! differences.  The first guard
// (rs_math.cuh) settles most trials in single precision; where it cannot --
// the top of the tree, whose terms reach 10^5 and whose abscissae reach
// 10^9, and the trials near a boundary -- this one tries before FP64.  It
// computes the same quantities to about 2^-44 relative and settles a trial
// only when no boundary lies within a margin that covers its own error and
// the FP64 definition's (2^-45 of the terms' magnitudes for T, 2^-50 of
// alpha + h/U for X, as the first guard's analysis gives); otherwise the
// trial runs the FP64 definition.  So every outcome is the definition's.
//
// Error model.  u = 2^-24.  two_sum and two_prod (with a fused multiply-add)
// are exact; ff_add is within 2^-44 (|x| + |y|), ff_mul within 2^-44 |x y|,
// ff_div within 2^-42 |x / y|, ff_sqrt within 2^-43 |sqrt x|; conversions of
// integers below 2^48 are exact and of larger ones within 2^-47; ln m of an
// integer m is the fixed-point qnlog_u57 (within 2^-55 absolute).  The
// margins below are 2^-36 of the magnitudes involved (plus 2^-26 absolute
// for the Stirling tails, taken in single precision), several hundred times
// the sum of these errors over the few dozen operations of a trial.
#pragma once
#include "rs_math.cuh"

namespace rs {

struct FF {
    float hi, lo;
};

RS_DEV FF ff_fast2(float a, float b) {   // |a| >= |b| or a = 0
    const float s = a + b;
    return FF{s, b - (s - a)};
}
RS_DEV FF ff_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return FF{s, (a - (s - bb)) + (b - bb)};
}
RS_DEV FF ff_add(FF x, FF y) {
    const FF s = ff_two_sum(x.hi, y.hi);
    return ff_fast2(s.hi, s.lo + (x.lo + y.lo));
}
RS_DEV FF ff_neg(FF x) { return FF{-x.hi, -x.lo}; }
RS_DEV FF ff_sub(FF x, FF y) { return ff_add(x, ff_neg(y)); }
RS_DEV FF ff_mul(FF x, FF y) {
    const float p = x.hi * y.hi;
    const float e = __fmaf_rn(x.hi, y.hi, -p) + (x.hi * y.lo + x.lo * y.hi);
    return ff_fast2(p, e);
}
RS_DEV FF ff_mul_f(FF x, float f) {
    const float p = x.hi * f;
    return ff_fast2(p, __fmaf_rn(x.hi, f, -p) + x.lo * f);
}
RS_DEV FF ff_div(FF x, FF y) {
    const float r = __frcp_rn(y.hi);
    const float q1 = x.hi * r;
    const FF rem = ff_sub(x, ff_mul_f(y, q1));   // x - q1 y, small
    return ff_fast2(q1, rem.hi * r);
}
RS_DEV FF ff_sqrt(FF x) {
    const float s = sqrtf(x.hi);
    const float p = s * s;
    const FF d = ff_add(x, FF{-p, -__fmaf_rn(s, s, -p)});   // x - s^2
    return ff_fast2(s, d.hi * (0.5f * __frcp_rn(s)));
}
RS_DEV float ff_val(FF x) { return x.hi + x.lo; }

// Conversions: a 64-bit integer (exact below 2^48), a double (within
// 2^-48), a Q57 fixed-point integer.
RS_DEV FF ff_from_u64(uint64_t x) {
    const float h = __ull2float_rn(x);
    const int64_t rest = (int64_t)(x - __float2ull_rn(h));
    return FF{h, __ll2float_rn(rest)};
}
RS_DEV FF ff_from_double(double d) {
    const float h = __double2float_rn(d);
    return FF{h, __double2float_rn(d - (double)h)};
}
RS_DEV FF ff_from_q57(int64_t L) {
    const float h = __ll2float_rn(L);
    const int64_t rest = L - __float2ll_rn(h);
    return FF{h * 0x1p-57f, __ll2float_rn(rest) * 0x1p-57f};
}

// ln m for an integer m >= 1 in Q57: 53 ln 2 - qnlog_u57(m), within 2^-55
// (qnlog_u57 takes m up to 2^63: above 2^53 its value is negative).
RS_DEV int64_t ln_u64_q57(uint64_t m, const double* __restrict__ tab) {
    return 53 * kLn2Q57 + ((53 * kLn2Q57Frac32) >> 32) - qnlog_u57(m, tab);
}

// The Stirling tail 1/(12x) - 1/(360x^3) of ln x! in single precision, for
// a difference of two tails (each below 3.3e-4 for x >= 256; their
// difference is within 2^-30 of the exact one).
RS_DEV float ff_tail(uint64_t x) {
    const float r = __frcp_rn(__ull2float_rn(x));
    return r * (0.083333333f - 0.0027777778f * r * r);
}

// ln x! - ln y! for x > y; *mag bounds the magnitudes of its parts, so that
// the error is within 2^-40 *mag + 2^-30.  tab is the context's table (ln i!
// for i < 256 in FP64, and the fixed-point logarithm's entries).
RS_DEV FF ff_lfdiff(uint64_t x, uint64_t y, const double* __restrict__ tab, float* mag) {
    if (x < 256) {
        const FF a = ff_from_double(tab[x]), b = ff_from_double(tab[y]);
        *mag = a.hi + b.hi + 1.0f;
        return ff_sub(a, b);
    }
    const FF X = ff_from_u64(x);
    const FF Xh = ff_add(X, FF{0.5f, 0.0f});
    if (y < 256) {
        // (x + 1/2) ln x - x + ln(2 pi)/2 + tail(x) - ln y!
        const FF lx = ff_from_q57(ln_u64_q57(x, tab));
        const FF A = ff_mul(Xh, lx);
        const FF ly = ff_from_double(tab[y]);
        *mag = A.hi + X.hi + ly.hi + 2.0f;
        FF v = ff_sub(A, X);
        v = ff_add(v, FF{9.189385176e-01f, 1.563417662e-08f});   // ln(2 pi)/2 = 0.91893853320467...
        v = ff_add(v, FF{ff_tail(x), 0.0f});
        return ff_sub(v, ly);
    }
    // (x + 1/2) ln(1 + d/y) + d ln y - d + tail(x) - tail(y)
    const uint64_t d = x - y;
    const FF D = ff_from_u64(d);
    const int64_t lyq = ln_u64_q57(y, tab);
    FF l1p;
    if (d < (y >> 5)) {
        // ln(1 + z) = 2 (w + w^3/3 + w^5/5 + w^7/7 + w^9/9), w = d / (2y + d) <= 2^-6
        const FF w = ff_div(D, ff_from_u64(2 * y + d));
        const FF w2 = ff_mul(w, w);
        FF s = ff_add(FF{1.428571492e-01f, -6.386212004e-09f}, ff_mul_f(w2, 1.111111119e-01f));   // 1/7 + w^2/9
        s = ff_add(FF{2.000000030e-01f, -2.980232283e-09f}, ff_mul(w2, s));                       // 1/5 + ...
        s = ff_add(FF{3.333333433e-01f, -9.934107759e-09f}, ff_mul(w2, s));               // 1/3 + ...
        s = ff_add(FF{1.0f, 0.0f}, ff_mul(w2, s));
        l1p = ff_mul_f(ff_mul(w, s), 2.0f);
    } else {
        // ln x - ln y from the fixed-point logarithms (the difference is exact)
        l1p = ff_from_q57(ln_u64_q57(x, tab) - lyq);
    }
    const FF A = ff_mul(Xh, l1p);
    const FF B = ff_mul(D, ff_from_q57(lyq));
    *mag = A.hi + B.hi + D.hi + 1.0f;
    FF v = ff_add(A, B);
    v = ff_sub(v, D);
    return ff_add(v, FF{ff_tail(x) - ff_tail(y), 0.0f});
}

// Signed ln P! - ln Q!.
RS_DEV FF ff_sd(uint64_t P, uint64_t Q, const double* __restrict__ tab, float* mag) {
    if (P == Q) {
        *mag = 0.0f;
        return FF{0.0f, 0.0f};
    }
    return P > Q ? ff_lfdiff(P, Q, tab, mag) : ff_neg(ff_lfdiff(Q, P, tab, mag));
}

// A ratio-of-uniforms node's parameters in float-float: the definition's
// formulas (mean, variance, hat width h, alpha = mean + 1/2, and for the
// binomial ln(p / (1 - p)) as a difference of two fixed-point logarithms)
// with every operation in float-float.
struct FFParams {
    FF mu, alpha, h, logr;
};
RS_DEV FF ff_hat_width(FF var) {
    const FF d1{1.715527773e+00f, -2.982028846e-09f};   // RS_HAT_D1 as two singles
    const FF d2{8.989161849e-01f, -2.284329170e-08f};   // RS_HAT_D2
    return ff_add(ff_mul(d1, ff_sqrt(ff_add(var, FF{0.5f, 0.0f}))), d2);
}
// Hypergeometric: a = min(n, K), b = max(n, K) after the reductions.
RS_DEV FFParams ff_hg_params(uint64_t a, uint64_t b, uint64_t S) {
    FFParams f;
    const FF Sf = ff_from_u64(S);
    f.mu = ff_div(ff_mul(ff_from_u64(a), ff_from_u64(b)), Sf);
    const FF var = ff_mul(ff_mul(f.mu, ff_div(ff_from_u64(S - a), Sf)), ff_div(ff_from_u64(S - b), ff_from_u64(S - 1)));
    f.h = ff_hat_width(var);
    f.alpha = ff_add(f.mu, FF{0.5f, 0.0f});
    f.logr = FF{0.0f, 0.0f};
    return f;
}
// Binomial BIN(c, K / S), K / S <= 1/2.
RS_DEV FFParams ff_bin_params(uint64_t c, uint64_t K, uint64_t S, const double* __restrict__ tab) {
    FFParams f;
    const FF pp = ff_div(ff_from_u64(K), ff_from_u64(S));
    f.mu = ff_mul(ff_from_u64(c), pp);
    f.h = ff_hat_width(ff_mul(f.mu, ff_sub(FF{1.0f, 0.0f}, pp)));
    f.alpha = ff_add(f.mu, FF{0.5f, 0.0f});
    f.logr = (2 * K == S) ? FF{0.0f, 0.0f} : ff_from_q57(ln_u64_q57(K, tab) - ln_u64_q57(S - K, tab));
    return f;
}
// Whether the mean lies below 16 (inversion), from the float-float mean
// where it is clear of 16: 1 yes, 0 no, -1 too close (the FP64 mean decides).
RS_DEV int ff_mean_below_16(FF mu) {
    const float m = ff_val(mu);
    if (m < 15.999f) return 1;
    if (m > 16.001f) return 0;
    return -1;
}

// The second guard's margins (see the error model above).
constexpr float kFFGuardEps = 0x1p-36f;
constexpr float kFFGuardAbs = 0x1p-26f;

// Decision for 2 ln U against T (magnitude tmag): 1 accept, -1 reject, 0
// too close to call.  ux is the trial's 64-bit value of U.
RS_DEV int ff_guard_decide(uint64_t ux, FF T, float tmag, const double* __restrict__ tab) {
    const uint64_t m = (ux >> 11) + 1;   // U = m 2^-53
    const FF L = m == (1ull << 53) ? FF{0.0f, 0.0f} : ff_mul_f(ff_from_q57(-qnlog_u57(m, tab)), 2.0f);
    const FF diff = ff_sub(T, L);   // accept when 2 ln U <= T
    const float margin = kFFGuardEps * ((tmag + fabsf(L.hi)) + 1.0f) + kFFGuardAbs;
    const float dv = ff_val(diff);
    if (dv > margin) return 1;
    if (dv < -margin) return -1;
    return 0;
}

// The abscissa: 1 (X in [0, top), *k = floor(X)), -1 (rejected) or 0 (too
// close to call), from alpha and h in float-float; ux, vx the trial's values
// of U and V; top = a + 1.
RS_DEV int ff_guard_abscissa(FF alpha, FF h, uint64_t top, uint64_t ux, uint64_t vx, uint64_t* k) {
    const FF U = ff_mul_f(ff_from_u64((ux >> 11) + 1), 0x1p-53f);
    const FF Vh = ff_sub(ff_mul_f(ff_from_u64(vx >> 11), 0x1p-53f), FF{0.5f, 0.0f});
    const FF t = ff_div(ff_mul(h, Vh), U);
    const FF X = ff_add(alpha, t);
    const float E = kFFGuardEps * ((alpha.hi + fabsf(h.hi) * __frcp_rn(U.hi)) + 1.0f);
    const float xv = ff_val(X);
    const float topf = __ull2float_rn(top);
    if (xv + E < 0.0f || xv - E >= topf * (1.0f + 1.2e-7f)) return -1;
    if (xv - E < 0.0f || xv + E >= topf * (1.0f - 1.2e-7f)) return 0;
    // floor(X - E) and floor(X + E) from hi and lo separately
    const float fh = floorf(X.hi);
    const float r = (X.hi - fh) + X.lo;   // X - fh; X.hi - fh is exact
    const float klo = floorf(__fadd_rd(r, -E));
    if (klo != floorf(__fadd_ru(r, E))) return 0;
    *k = __float2ull_rn(fh) + (uint64_t)(int64_t)klo;
    return 1;
}

}  // namespace rs
