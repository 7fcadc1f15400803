// rs_deviates.cuh -- the split deviates on the device.
//
// A node holding c samples of [lo, lo+S) sends L of them to its left half of
// floor(S/2) positions.  Without replacement L is hypergeometric (Sec. 3),
// with replacement binomial (Sec. 4.6).  The paper generates these with
// Stadlober's ratio-of-uniforms method; the method here is inversion below a
// mean of 16 and ratio-of-uniforms with the table-mountain hat above, with
// no squeeze.  Uniforms are the 64-bit values of the node's SPLIT stream in
// order: value r for inversion restart r, values 2i and 2i+1 for trial i.
#pragma once
#include "rs_ff.cuh"
#include "rs_math.cuh"
#include "rs_rng.cuh"

namespace rs {

// Warp-cooperative forms (WARP = true): every lane of a full warp calls with
// the same arguments and gets the same result.  Inversion restart r and
// ratio-of-uniforms trial i run on lane r mod 32 (i mod 32) in round r / 32
// (i / 32); the result is that of the first restart or trial in index order
// that succeeds, exactly as in the one-thread form, in about one trial's
// latency instead of the expected number of trials' (GB300 issues an FP64
// warp instruction at the same cost whatever its active lanes).
template <bool WARP>
struct TrialLanes {
    static constexpr uint64_t step = WARP ? 32 : 1;
    RS_DEV static uint64_t lane() { return WARP ? (threadIdx.x & 31u) : 0; }
    // Among the lanes' outcomes (ok, value), the first lane's that succeeded.
    RS_DEV static bool first(bool ok, uint64_t v, uint64_t& out) {
        if constexpr (WARP) {
            const unsigned acc = __ballot_sync(0xffffffffu, ok);
            if (!acc) return false;
            out = __shfl_sync(0xffffffffu, v, __ffs(acc) - 1);
            return true;
        } else {
            if (ok) out = v;
            return ok;
        }
    }
};

// HG(n, K, S): successes among n draws without replacement from S items
// containing K successes.  Returns RS_OK or RS_EITER.  INV: the caller has
// found the mean below 16 (by the same decision), so only inversion is
// compiled in.
template <bool WARP, bool INV = false>
RS_DEV int hypergeometric_t(Key2 key, uint64_t node, uint64_t n, uint64_t K, uint64_t S,
                            const double* __restrict__ tab, uint64_t& out) {
    using TL = TrialLanes<WARP>;
    if (n == 0 || K == 0) { out = 0; return RS_OK; }
    if (K == S) { out = n; return RS_OK; }
    if (n == S) { out = K; return RS_OK; }
    const uint64_t n_in = n;
    // Symmetries: take the smaller of K and S-K, and of n and S-n.
    const bool flipK = K > S - K;
    if (flipK) K = S - K;
    const bool flipN = n > S - n;
    if (flipN) n = S - n;
    const uint64_t a = n < K ? n : K;
    const uint64_t b = n < K ? K : n;
    // the parameters in float-float for the guards (rs_ff.cuh); the FP64
    // ones, as defined, only where a guard leaves a decision open
    const FFParams fp = INV ? FFParams{} : ff_hg_params(a, b, S);
    int below = INV ? 1 : ff_mean_below_16(fp.mu);
    if (below < 0) below = ((double)a * (double)b) * drecip((double)S) < 16.0;
    uint64_t y = 0;
    bool done = false;
    if (below) {
        // Inversion from k = 0 with the pmf recurrence
        // f(k+1) = f(k) (a-k)(b-k) / ((k+1)(S-a-b+k+1)).
        const double f0 = dexp(dsd(S - b, S - a - b, tab) - dsd(S, S - a, tab));
        for (uint64_t r0 = 0; r0 < c_caps.inv_restarts && !done; r0 += TL::step) {
            const uint64_t r = r0 + TL::lane();
            const bool in_cap = r < c_caps.inv_restarts;
            double u = v_closed(stream_value(key, TAG_SPLIT, node, r));
            double f = f0;
            bool ok = false;
            uint64_t yk = 0;
            for (uint64_t k = 0; k <= a && in_cap; ++k) {
                if (u < f) { yk = k; ok = true; break; }
                u = u - f;
                f = (f * ((double)(a - k) * (double)(b - k))) / ((double)(k + 1) * (double)(S - a - b + k + 1));
                // Once f underflows to 0 it stays 0 and u no longer changes, so
                // this pass can only run past a: restart now (same outcome).
                if (f == 0.0) break;
            }
            done = TL::first(ok, yk, y);
        }
    } else {
        const uint64_t M = (uint64_t)(((unsigned __int128)(a + 1) * (b + 1)) / (S + 2));
        const uint64_t m = S - a - b;
        bool have64 = false, haveL = false;
        double alpha = 0.0, h = 0.0, top = 0.0, l0 = 0.0, l1 = 0.0, l2 = 0.0, l3 = 0.0;
        for (uint64_t i0 = 0; i0 < c_caps.rou_trials && !done; i0 += TL::step) {
            const uint64_t i = i0 + TL::lane();
            const uint4 blk = philox_block((uint32_t)i, TAG_SPLIT, node, key);
            const uint64_t ux = ((uint64_t)blk.y << 32) | blk.x, vx = ((uint64_t)blk.w << 32) | blk.z;
            uint64_t k = 0;
            int xd = ff_guard_abscissa(fp.alpha, fp.h, a + 1, ux, vx, &k);
            if (xd == 0) {   // the abscissa in FP64, as defined
                if (!have64) {
                    const double rS = drecip((double)S);
                    const double mu = ((double)a * (double)b) * rS;
                    const double var = mu * ((double)(S - a) * rS) * ((double)(S - b) * drecip((double)(S - 1)));
                    h = RS_HAT_D1 * sqrt(var + 0.5) + RS_HAT_D2;
                    alpha = mu + 0.5;
                    top = (double)a + 1.0;
                    have64 = true;
                }
                const double X = alpha + h * (v_closed(vx) - 0.5) * drecip(u_open(ux));
                xd = (X >= 0.0 && X < top) ? 1 : -1;
                if (xd > 0) k = (uint64_t)X;
            }
            bool ok = false;
            if (xd > 0 && i < c_caps.rou_trials) {
                float mg, mj;
                FF T = ff_sd(M, k, tab, &mg);
                T = ff_add(T, ff_sd(a - M, a - k, tab, &mj));
                mg += mj;
                T = ff_add(T, ff_sd(b - M, b - k, tab, &mj));
                mg += mj;
                T = ff_add(T, ff_sd(m + M, m + k, tab, &mj));
                mg += mj;
                const int dec = ff_guard_decide(ux, T, mg, tab);
                if (dec == 0) {   // the test in FP64, as defined
                    if (!haveL) {
                        l0 = log_fixed(M, tab);
                        l1 = log_fixed(a - M, tab);
                        l2 = log_fixed(b - M, tab);
                        l3 = log_fixed(m + M, tab);
                        haveL = true;
                    }
                    const double T64 = dsd_fixed(M, k, l0, tab) + dsd_fixed(a - M, a - k, l1, tab) +
                                       dsd_fixed(b - M, b - k, l2, tab) + dsd_fixed(m + M, m + k, l3, tab);
                    ok = 2.0 * dlog(u_open(ux), tab) <= T64;
                } else {
                    ok = dec > 0;
                }
            }
            done = TL::first(ok, k, y);
        }
    }
    if (!done) return RS_EITER;
    if (flipN) y = K - y;
    if (flipK) y = n_in - y;
    out = y;
    return RS_OK;
}

// BIN(c, p = K/S) with K/S <= 1/2.  Returns RS_OK or RS_EITER.
template <bool WARP, bool INV = false>
RS_DEV int binomial_t(Key2 key, uint64_t node, uint64_t c, uint64_t K, uint64_t S,
                      const double* __restrict__ tab, uint64_t& out) {
    using TL = TrialLanes<WARP>;
    if (c == 0 || K == 0) { out = 0; return RS_OK; }
    const double p = (double)K / (double)S;
    const FFParams fp = INV ? FFParams{} : ff_bin_params(c, K, S, tab);
    int below = INV ? 1 : ff_mean_below_16(fp.mu);
    if (below < 0) below = (double)c * p < 16.0;
    if (below) {
        const double f0 = dexp((double)c * dlog1p(-p, tab));
        const double r = p / (1.0 - p);
        for (uint64_t q0 = 0; q0 < c_caps.inv_restarts; q0 += TL::step) {
            const uint64_t q = q0 + TL::lane();
            double u = v_closed(stream_value(key, TAG_SPLIT, node, q));
            double f = f0;
            bool ok = false;
            uint64_t yk = 0;
            for (uint64_t k = 0; k <= c && q < c_caps.inv_restarts; ++k) {
                if (u < f) { yk = k; ok = true; break; }
                u = u - f;
                f = (f * ((double)(c - k) * r)) / (double)(k + 1);
                if (f == 0.0) break;
            }
            if (TL::first(ok, yk, out)) return RS_OK;
        }
        return RS_EITER;
    }
    const uint64_t M = (uint64_t)(((unsigned __int128)(c + 1) * K) / S);
    bool have64 = false, haveL = false;
    double alpha = 0.0, h = 0.0, top = 0.0, logr = 0.0, l0 = 0.0, l1 = 0.0;
    for (uint64_t i0 = 0; i0 < c_caps.rou_trials; i0 += TL::step) {
        const uint64_t i = i0 + TL::lane();
        const uint4 blk = philox_block((uint32_t)i, TAG_SPLIT, node, key);
        const uint64_t ux = ((uint64_t)blk.y << 32) | blk.x, vx = ((uint64_t)blk.w << 32) | blk.z;
        uint64_t k = 0;
        int xd = ff_guard_abscissa(fp.alpha, fp.h, c + 1, ux, vx, &k);
        if (xd == 0) {   // the abscissa in FP64, as defined
            if (!have64) {
                const double mu = (double)c * p;
                h = RS_HAT_D1 * sqrt(mu * (1.0 - p) + 0.5) + RS_HAT_D2;
                alpha = mu + 0.5;
                top = (double)c + 1.0;
                have64 = true;
            }
            const double X = alpha + h * (v_closed(vx) - 0.5) * drecip(u_open(ux));
            xd = (X >= 0.0 && X < top) ? 1 : -1;
            if (xd > 0) k = (uint64_t)X;
        }
        bool ok = false;
        if (xd > 0 && i < c_caps.rou_trials) {
            float mg, mj;
            FF T = ff_sd(M, k, tab, &mg);
            T = ff_add(T, ff_sd(c - M, c - k, tab, &mj));
            mg += mj;
            const FF dk = k >= M ? ff_from_u64(k - M) : ff_neg(ff_from_u64(M - k));
            const FF rt = ff_mul(dk, fp.logr);
            T = ff_add(T, rt);
            mg += fabsf(rt.hi) + fabsf(dk.hi);
            const int dec = ff_guard_decide(ux, T, mg, tab);
            if (dec == 0) {   // the test in FP64, as defined
                if (!haveL) {
                    const double r = p / (1.0 - p);
                    logr = (r == 1.0) ? 0.0 : dlog(r, tab);
                    l0 = log_fixed(M, tab);
                    l1 = log_fixed(c - M, tab);
                    haveL = true;
                }
                const double T64 = dsd_fixed(M, k, l0, tab) + dsd_fixed(c - M, c - k, l1, tab) +
                                   (double)((int64_t)k - (int64_t)M) * logr;
                ok = 2.0 * dlog(u_open(ux), tab) <= T64;
            } else {
                ok = dec > 0;
            }
        }
        if (TL::first(ok, k, out)) return RS_OK;
    }
    return RS_EITER;
}

RS_DEV int hypergeometric(Key2 key, uint64_t node, uint64_t n, uint64_t K, uint64_t S,
                          const double* __restrict__ tab, uint64_t& out) {
    return hypergeometric_t<false>(key, node, n, K, S, tab, out);
}
RS_DEV int hypergeometric_warp(Key2 key, uint64_t node, uint64_t n, uint64_t K, uint64_t S,
                               const double* __restrict__ tab, uint64_t& out) {
    return hypergeometric_t<true>(key, node, n, K, S, tab, out);
}
RS_DEV int binomial(Key2 key, uint64_t node, uint64_t c, uint64_t K, uint64_t S,
                    const double* __restrict__ tab, uint64_t& out) {
    return binomial_t<false>(key, node, c, K, S, tab, out);
}
RS_DEV int binomial_warp(Key2 key, uint64_t node, uint64_t c, uint64_t K, uint64_t S,
                         const double* __restrict__ tab, uint64_t& out) {
    return binomial_t<true>(key, node, c, K, S, tab, out);
}
// The inversion paths alone, for callers that have found the mean below 16.
RS_DEV int hypergeometric_inversion(Key2 key, uint64_t node, uint64_t n, uint64_t K, uint64_t S,
                                    const double* __restrict__ tab, uint64_t& out) {
    return hypergeometric_t<false, true>(key, node, n, K, S, tab, out);
}
RS_DEV int binomial_inversion(Key2 key, uint64_t node, uint64_t c, uint64_t K, uint64_t S,
                              const double* __restrict__ tab, uint64_t& out) {
    return binomial_t<false, true>(key, node, c, K, S, tab, out);
}

}  // namespace rs
