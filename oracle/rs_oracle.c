/*
 * rs_oracle.c -- CPU oracle for divide-and-conquer random sampling
 * (Sanders, Lamm, Huebschle-Schneider, Schrade, Dachsbacher, "Efficient
 * Parallel Random Sampling -- Vectorized, Cache-Efficient, and Online").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this file.  The product library
 * shares no code with it: the CUDA path implements the same definitions
 * independently, and the two are compared bit for bit.
 *
 * Plain, slow, sequential C.  Every step follows the written definition of
 * the sampler, in the order the definition gives; nothing is blocked, fused
 * or reordered.  Build with -O2 -ffp-contract=off -fno-fast-math so that
 * every floating-point expression is evaluated exactly as written (IEEE
 * binary64, round to nearest; a fused multiply-add only where fma() is
 * written, single precision only where a (float) conversion is written).
 *
 * Where the paper fixes no detail (the RNG, the deviate algorithm, the
 * leaf draw order), the oracle takes the reading written out next to each
 * function.
 *
 * Parity status: everything here is pinned by the non-GPU tests against
 * known-answer vectors, libm/mpmath, exact rational probabilities, closed-form
 * moments and brute-force enumeration; the bit pattern of a sample is a
 * function of these definitions (no printed worked example survives in the
 * paper), so oracle == GPU is the parity claim for whole samples.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* Error codes (numerically equal to the library's; defined here on their own). */
enum { OR_OK = 0, OR_EINVAL = 1, OR_ECAPACITY = 2, OR_ENOMEM = 3, OR_EITER = 6 };

/* Stream tags (reading: one tag per kind of random decision). */
enum { TAG_SPLIT = 1, TAG_LEAF_H = 2, TAG_LEAF_B = 3, TAG_FIXUP = 4, TAG_BERN = 5, TAG_LEAF_WR = 6 };

/* ------------------------------------------------------------------------ */
/* Randomness.  The paper keys every random decision by the subtree it     */
/* belongs to (Sec. 3.2: the t-th deviate of subproblem j..k is h((j,k,t)), */
/* the local generator of PE i is seeded with h(i)).  Reading: a counter-   */
/* based generator, Philox4x32-10 (Salmon et al., SC'11), keyed by the      */
/* seed, with the counter holding (block t, tag, node id).                  */
/* ------------------------------------------------------------------------ */

/* One Philox4x32-10 block: 10 rounds of the Philox S-box with the Weyl key
 * schedule, as defined in Salmon, Moraes, Dror, Shaw, SC'11, Sec. 4. */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;   /* round multipliers */
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;   /* key increments    */
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * c0;
        uint64_t p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Block t of stream (seed, tag, id): key = (seed mod 2^32, seed >> 32),
 * counter = (t, tag, id mod 2^32, id >> 32).  A stream has 2^32 blocks. */
static void stream_block(uint64_t seed, uint32_t tag, uint64_t id, uint32_t t, uint32_t out[4])
{
    uint32_t ctr[4] = { t, tag, (uint32_t)id, (uint32_t)(id >> 32) };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    or_philox4x32_10(ctr, key, out);
}

/* 32-bit word j of a stream: block floor(j/4), word j mod 4. */
uint32_t or_word(uint64_t seed, uint32_t tag, uint64_t id, uint64_t j)
{
    uint32_t w[4];
    stream_block(seed, tag, id, (uint32_t)(j >> 2), w);
    return w[j & 3];
}

/* 64-bit value j of a stream: (word 2j+1 << 32) | word 2j. */
uint64_t or_value(uint64_t seed, uint32_t tag, uint64_t id, uint64_t j)
{
    uint32_t w[4];
    stream_block(seed, tag, id, (uint32_t)(j >> 1), w);
    uint32_t lo = w[(2 * j) & 3], hi = w[(2 * j + 1) & 3];
    return ((uint64_t)hi << 32) | lo;
}

/* Uniforms from a 64-bit value: U_open in (0,1], V in [0,1); exact. */
static const double TWO_M53 = 1.0 / 9007199254740992.0;   /* 2^-53 */
double or_u_open(uint64_t x) { return (double)((x >> 11) + 1) * TWO_M53; }
double or_v_closed(uint64_t x) { return (double)(x >> 11) * TWO_M53; }

/* Uniform integer in [0, s) by Lemire's multiply-and-reject, one candidate
 * per stream position.  A rejected position is "void": it is skipped but
 * still consumed, so candidate j always comes from the same position.
 * s <= 2^32: candidate j uses word j.  s > 2^32: candidate j uses value j.
 * Returns 1 and sets *v for a valid candidate, 0 for a void one.
 * (The paper only asks for uniform deviates, Sec. 2, Algorithm H.) */
int or_candidate(uint64_t seed, uint32_t tag, uint64_t id, uint64_t s, uint64_t j, uint64_t* v)
{
    if (s <= (1ull << 32)) {
        uint64_t w = or_word(seed, tag, id, j);
        uint64_t prod = w * s;
        uint64_t thr = ((1ull << 32) - s) % s;
        if ((prod & 0xFFFFFFFFull) < thr) return 0;
        *v = prod >> 32;
        return 1;
    } else {
        uint64_t x = or_value(seed, tag, id, j);
        u128 prod = (u128)x * s;
        uint64_t thr = (0 - s) % s;
        if ((uint64_t)prod < thr) return 0;
        *v = (uint64_t)(prod >> 64);
        return 1;
    }
}

/* ------------------------------------------------------------------------ */
/* Project-owned FP64 math, used only through + - * / sqrt, the fused       */
/* multiply-add and integer ops (each IEEE correctly rounded), so that two  */
/* independent implementations agree bit for bit.                          */
/* ------------------------------------------------------------------------ */

static double from_bits(uint64_t b) { double d; memcpy(&d, &b, 8); return d; }
static uint64_t to_bits(double d) { uint64_t b; memcpy(&b, &d, 8); return b; }

#define LN2_HI  from_bits(0x3fe62e42fee00000ull)  /* ln 2 truncated to 32 significant bits */
#define LN2_LO  from_bits(0x3dea39ef35793c76ull)  /* RN(ln 2 - LN2_HI)                 */
#define INV_LN2 from_bits(0x3ff71547652b82feull)  /* RN(1 / ln 2)                      */
#define HL2PI   from_bits(0x3fed67f1c864beb5ull)  /* RN(ln(2 pi) / 2)                  */
#define HAT_D1  from_bits(0x3ffb72cd3f331398ull)  /* RN(2 sqrt(2/e))                   */
#define HAT_D2  from_bits(0x3fecc3ebd3bc711aull)  /* RN(3 - 2 sqrt(3/e))               */

/* Double-double arithmetic for building the logarithm table: error-free
 * sums (Knuth) and products (by fused multiply-add), then renormalization. */
typedef struct { double hi, lo; } dd_t;
static dd_t dd_fast2(double a, double b) { double s = a + b; dd_t r = {s, b - (s - a)}; return r; }
static dd_t dd_two_sum(double a, double b)
{
    double s = a + b;
    double bb = s - a;
    dd_t r = {s, (a - (s - bb)) + (b - bb)};
    return r;
}
static dd_t dd_add(dd_t a, dd_t b)
{
    dd_t s = dd_two_sum(a.hi, b.hi);
    double e = s.lo + (a.lo + b.lo);
    return dd_fast2(s.hi, e);
}
static dd_t dd_mul(dd_t a, dd_t b)
{
    double p = a.hi * b.hi;
    double e = fma(a.hi, b.hi, -p);
    e = e + (a.hi * b.lo + a.lo * b.hi);
    return dd_fast2(p, e);
}
/* a / b to double-double precision: three quotient digits. */
static dd_t dd_div(dd_t a, dd_t b)
{
    double q1 = a.hi / b.hi;
    dd_t t = dd_mul(b, (dd_t){q1, 0.0});
    dd_t r = dd_add(a, (dd_t){-t.hi, -t.lo});
    double q2 = r.hi / b.hi;
    t = dd_mul(b, (dd_t){q2, 0.0});
    r = dd_add(r, (dd_t){-t.hi, -t.lo});
    double q3 = r.hi / b.hi;
    dd_t q = dd_fast2(q1, q2);
    return dd_add(q, (dd_t){q3, 0.0});
}

/* ln v for v in (1/2, 1] in double-double: 2 atanh(s), s = (v-1)/(v+1),
 * sum over k < 36 of s^(2k+1)/(2k+1) (|s| <= 1/3: the first term left
 * out is below 2^-110 relative). */
static dd_t dd_log_unit(double v)
{
    dd_t s = dd_div((dd_t){v - 1.0, 0.0}, dd_two_sum(v, 1.0));
    dd_t s2 = dd_mul(s, s);
    dd_t term = s, sum = s;
    for (int k = 1; k < 36; ++k) {
        term = dd_mul(term, s2);
        sum = dd_add(sum, dd_div(term, (dd_t){(double)(2 * k + 1), 0.0}));
    }
    dd_t r = {2.0 * sum.hi, 2.0 * sum.lo};
    return r;
}

/* Table of the logarithm: mantissa interval i of [1, 2) (i = 1..126, width
 * 2^-7) has centre c = 1 + (2i+1)/256, inv = RN(1/c) and L = -ln(inv) as a
 * double-double; intervals 0 and 127 use c = 1 (see or_log). */
static double log_inv[128], log_hi[128], log_lo[128];

__attribute__((constructor)) static void build_log_table(void)
{
    for (int i = 0; i < 128; ++i) {
        if (i == 0 || i == 127) {
            log_inv[i] = 1.0;
            log_hi[i] = 0.0;
            log_lo[i] = 0.0;
            continue;
        }
        double c = 1.0 + (double)(2 * i + 1) / 256.0;
        double inv = 1.0 / c;
        dd_t l = dd_log_unit(inv);
        log_inv[i] = inv;
        log_hi[i] = -l.hi;
        log_lo[i] = -l.lo;
    }
}

/* Entry i of the logarithm table (for tests): 1/c rounded, and -ln of it
 * as a double-double. */
void or_log_table_entry(int i, double* inv, double* hi, double* lo)
{
    *inv = log_inv[i & 127];
    *hi = log_hi[i & 127];
    *lo = log_lo[i & 127];
}

/* Natural logarithm of a normal x > 0.  x = 2^e m, m in [1, 2); the top 7
 * bits of m pick an interval with centre c and inv = RN(1/c), and
 * ln m = -ln(inv) + ln(1 + r), r = m inv - 1 (one fused multiply-add,
 * |r| <= 2^-8), ln(1 + r) by its Taylor polynomial to r^8/8 (Horner with
 * fused multiply-adds).  The two intervals next to 1 use c = 1 and r = m - 1
 * (or m/2 - 1 with e + 1), exact, so that ln x near 1 keeps its relative
 * accuracy; there |r| <= 2^-7. */
double or_log(double x)
{
    uint64_t bits = to_bits(x);
    int64_t e = (int64_t)((bits >> 52) & 0x7FF) - 1023;
    int i = (int)((bits >> 45) & 0x7F);
    double m = from_bits((bits & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull);
    double r;
    if (i == 127) {
        m = m * 0.5;
        e = e + 1;
        r = m - 1.0;
    } else if (i == 0) {
        r = m - 1.0;
    } else {
        r = fma(m, log_inv[i], -1.0);
    }
    double q = -1.0 / 8.0;
    q = fma(q, r, 1.0 / 7.0);
    q = fma(q, r, -1.0 / 6.0);
    q = fma(q, r, 1.0 / 5.0);
    q = fma(q, r, -1.0 / 4.0);
    q = fma(q, r, 1.0 / 3.0);
    q = fma(q, r, -0.5);
    double p = fma(r * r, q, r);
    double de = (double)e;
    return (de * LN2_HI + log_hi[i]) + ((de * LN2_LO + log_lo[i]) + p);
}

double or_log1p(double z)
{
    double u = 1.0 + z;
    if (u == 1.0) return z;
    return or_log(u) * (z / (u - 1.0));
}

/* 1/x for a positive x in [2^-60, 2^100]: a single-precision quotient of
 * x rounded to single precision as the seed (relative error below 2^-23),
 * then two Newton steps r <- r + r (1 - x r), each with two fused
 * multiply-adds; the result is within about one ulp of 1/x.  It stands for
 * a quotient wherever a correctly rounded one is not needed: Stirling's
 * tail, the argument of ln(1 + z), the ratio-of-uniforms abscissa. */
double or_recip(double x)
{
    double r = (double)(1.0f / (float)x);
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
}

/* ln(1 + z) for z >= 0 without a division: u = 1 + z rounded, e = (1 + z)
 * - u exactly (Knuth's two-sum), ln(1 + z) = ln u + ln(1 + e/u), and since
 * |e/u| <= 2^-53 the last term is e/u to 2^-106 relative; e/u is taken as
 * e times a single-precision 1/u. */
double or_log1p_pos(double z)
{
    double u = 1.0 + z;
    double bb = u - 1.0;
    double e = (1.0 - (u - bb)) + (z - bb);
    return or_log(u) + e * (double)(1.0f / (float)u);
}

/* e^x for x in [-708, 0]: k = round(x / ln 2), r = x - k ln 2 (split in two
 * parts), e^r by its Taylor series to r^13/13!, scaled by 2^k built from bits. */
double or_exp(double x)
{
    int64_t k = (int64_t)floor(x * INV_LN2 + 0.5);
    double dk = (double)k;
    double r = (x - dk * LN2_HI) - dk * LN2_LO;
    double p = 1.0 / 6227020800.0;          /* 1/13! */
    p = 1.0 / 479001600.0 + r * p;          /* 1/12! */
    p = 1.0 / 39916800.0 + r * p;           /* 1/11! */
    p = 1.0 / 3628800.0 + r * p;            /* 1/10! */
    p = 1.0 / 362880.0 + r * p;             /* 1/9!  */
    p = 1.0 / 40320.0 + r * p;              /* 1/8!  */
    p = 1.0 / 5040.0 + r * p;               /* 1/7!  */
    p = 1.0 / 720.0 + r * p;                /* 1/6!  */
    p = 1.0 / 120.0 + r * p;                /* 1/5!  */
    p = 1.0 / 24.0 + r * p;                 /* 1/4!  */
    p = 1.0 / 6.0 + r * p;                  /* 1/3!  */
    p = 1.0 / 2.0 + r * p;                  /* 1/2!  */
    p = 1.0 + r * p;                        /* 1/1!  */
    p = 1.0 + r * p;                        /* 1/0!  */
    return p * from_bits((uint64_t)(k + 1023) << 52);
}

/* ln x! : table below 256 (summed logs), Stirling's series above. */
static double lf_table[256];
static int lf_ready = 0;

static void lf_init(void)
{
    if (lf_ready) return;
    lf_table[0] = 0.0;
    lf_table[1] = 0.0;
    for (int i = 2; i < 256; ++i) lf_table[i] = lf_table[i - 1] + or_log((double)i);
    lf_ready = 1;
}

/* Stirling correction 1/(12x) - 1/(360x^3) + 1/(1260x^5) - 1/(1680x^7),
 * from r = 1/x (or_recip). */
static double stirling_tail(double r)
{
    double r2 = r * r;
    return r * (1.0 / 12.0 + r2 * (-1.0 / 360.0 + r2 * (1.0 / 1260.0 + r2 * (-1.0 / 1680.0))));
}

double or_lf(uint64_t x)
{
    lf_init();
    if (x < 256) return lf_table[x];
    double X = (double)x;
    return (X + 0.5) * or_log(X) - X + HL2PI + stirling_tail(or_recip(X));
}

/* ln x! - ln y! for x >= y, written so that no large term cancels:
 * (x + 1/2) ln(1 + d/y) + d ln y - d + tail(x) - tail(y), d = x - y, for
 * every d once y >= 256 (short differences included: ln(1 + d/y) keeps
 * its relative accuracy for small d/y, and the tails' difference is far
 * below the result's ulp). */
double or_lfdiff(uint64_t x, uint64_t y)
{
    lf_init();
    uint64_t d = x - y;
    if (d == 0) return 0.0;
    if (x < 256) return lf_table[x] - lf_table[y];
    if (y < 256) return or_lf(x) - lf_table[y];
    double X = (double)x, Y = (double)y, Dd = (double)d;
    double rY = or_recip(Y);
    double lp = or_log1p_pos(Dd * rY);
    return (X + 0.5) * lp + Dd * or_log(Y) - Dd + (stirling_tail(or_recip(X)) - stirling_tail(rY));
}

/* Signed difference ln x! - ln y!. */
double or_sd(uint64_t x, uint64_t y)
{
    return x >= y ? or_lfdiff(x, y) : -or_lfdiff(y, x);
}

/* ln P! - ln Q! for the ratio-of-uniforms tests, where P is fixed for the
 * node and lnP = or_log(P) (P >= 1; unused for P = 0) was computed once: the
 * same branches as or_lfdiff on (max, min), except that ln of the larger
 * argument is lnP when that is P, and ln of the smaller one in the
 * cancellation-free form is lnP when that is P, else ln P - ln(P/Q). */
double or_sd_fixed(uint64_t P, uint64_t Q, double lnP)
{
    lf_init();
    int p_big = P >= Q;
    uint64_t x = p_big ? P : Q, y = p_big ? Q : P, d = x - y;
    double v;
    if (d == 0) return 0.0;
    if (x < 256) {
        v = lf_table[x] - lf_table[y];
    } else {
        double X = (double)x;
        if (y < 256) {
            double lx = p_big ? lnP : or_log(X);
            v = ((X + 0.5) * lx - X + HL2PI + stirling_tail(or_recip(X))) - lf_table[y];
        } else {
            double Y = (double)y, Dd = (double)d;
            double rY = or_recip(Y);
            double lp = or_log1p_pos(Dd * rY);
            double ly = p_big ? lnP - lp : lnP;
            v = (X + 0.5) * lp + Dd * ly - Dd + (stirling_tail(or_recip(X)) - stirling_tail(rY));
        }
    }
    return p_big ? v : -v;
}

/* ln P for or_sd_fixed. */
static double log_fixed(uint64_t P)
{
    return or_log((double)(P > 0 ? P : 1));
}

/* ------------------------------------------------------------------------ */
/* Random deviates for the splitting step.                                  */
/* ------------------------------------------------------------------------ */

/* Hypergeometric deviate HG(n, K, S): successes among n draws without
 * replacement from S items of which K are successes.  This is the number L
 * of samples falling left of a split (Sec. 3: L is hypergeometric with
 * parameters n, l, N).  The paper uses Stadlober's ratio-of-uniforms method
 * (Sec. 3.1, Sec. 5); reading: inversion when the mean is below 16, else
 * ratio-of-uniforms with the table-mountain hat and no squeeze.  Uniforms
 * are 64-bit values of the stream (SPLIT, node id), in order. */
int or_hg(uint64_t seed, uint64_t id, uint64_t n, uint64_t K, uint64_t S, uint64_t* out)
{
    if (n == 0 || K == 0) { *out = 0; return OR_OK; }
    if (K == S) { *out = n; return OR_OK; }
    if (n == S) { *out = K; return OR_OK; }
    uint64_t n_orig = n;
    int sK = (2 * (u128)K > S);
    if (sK) K = S - K;
    int sN = (2 * (u128)n > S);
    if (sN) n = S - n;
    uint64_t a = n < K ? n : K;
    uint64_t b = n < K ? K : n;
    double rS = or_recip((double)S);
    double mu = ((double)a * (double)b) * rS;
    uint64_t Y = 0;
    int found = 0;
    if (mu < 16.0) {
        double p0 = or_exp(or_sd(S - b, S - a - b) - or_sd(S, S - a));
        for (uint64_t restart = 0; restart < 64 && !found; ++restart) {
            double u = or_v_closed(or_value(seed, TAG_SPLIT, id, restart));
            double p = p0;
            uint64_t k = 0;
            for (;;) {
                if (u < p) { Y = k; found = 1; break; }
                u = u - p;
                p = (p * ((double)(a - k) * (double)(b - k))) / ((double)(k + 1) * (double)(S - a - b + k + 1));
                k = k + 1;
                if (k > a) break;
                if (p == 0.0) break;   /* p stays 0 and u unchanged: this pass can only run out */
            }
        }
    } else {
        double var = mu * ((double)(S - a) * rS) * ((double)(S - b) * or_recip((double)(S - 1)));
        double c = sqrt(var + 0.5);
        double h = HAT_D1 * c + HAT_D2;
        double alpha = mu + 0.5;
        uint64_t M = (uint64_t)(((u128)(a + 1) * (u128)(b + 1)) / (u128)(S + 2));
        uint64_t m = S - a - b;
        /* the test's four differences have the fixed ends M, a-M, b-M, m+M */
        double l0 = log_fixed(M), l1 = log_fixed(a - M), l2 = log_fixed(b - M), l3 = log_fixed(m + M);
        for (uint64_t i = 0; i < (1ull << 20); ++i) {
            double U = or_u_open(or_value(seed, TAG_SPLIT, id, 2 * i));
            double V = or_v_closed(or_value(seed, TAG_SPLIT, id, 2 * i + 1));
            double X = alpha + h * (V - 0.5) * or_recip(U);
            if (X < 0.0 || X >= (double)a + 1.0) continue;
            uint64_t k = (uint64_t)X;
            double T = or_sd_fixed(M, k, l0) + or_sd_fixed(a - M, a - k, l1) + or_sd_fixed(b - M, b - k, l2)
                     + or_sd_fixed(m + M, m + k, l3);
            if (2.0 * or_log(U) <= T) { Y = k; found = 1; break; }
        }
    }
    if (!found) return OR_EITER;
    if (sN) Y = K - Y;
    if (sK) Y = n_orig - Y;
    *out = Y;
    return OR_OK;
}

/* Binomial deviate BIN(c, K/S), the split for sampling with replacement
 * (Sec. 4.6).  Same method and stream as or_hg; K/S <= 1/2 is assumed. */
int or_bin(uint64_t seed, uint64_t id, uint64_t c, uint64_t K, uint64_t S, uint64_t* out)
{
    if (c == 0 || K == 0) { *out = 0; return OR_OK; }
    double p = (double)K / (double)S;
    double mu = (double)c * p;
    if (mu < 16.0) {
        double p0 = or_exp((double)c * or_log1p(-p));
        double r = p / (1.0 - p);
        for (uint64_t restart = 0; restart < 64; ++restart) {
            double u = or_v_closed(or_value(seed, TAG_SPLIT, id, restart));
            double pk = p0;
            uint64_t k = 0;
            for (;;) {
                if (u < pk) { *out = k; return OR_OK; }
                u = u - pk;
                pk = (pk * ((double)(c - k) * r)) / (double)(k + 1);
                k = k + 1;
                if (k > c) break;
                if (pk == 0.0) break;  /* as above */
            }
        }
        return OR_EITER;
    }
    double var = mu * (1.0 - p);
    double cc = sqrt(var + 0.5);
    double h = HAT_D1 * cc + HAT_D2;
    double alpha = mu + 0.5;
    double r = p / (1.0 - p);
    double logr = (r == 1.0) ? 0.0 : or_log(r);
    uint64_t M = (uint64_t)(((u128)(c + 1) * (u128)K) / (u128)S);
    double l0 = log_fixed(M), l1 = log_fixed(c - M);
    for (uint64_t i = 0; i < (1ull << 20); ++i) {
        double U = or_u_open(or_value(seed, TAG_SPLIT, id, 2 * i));
        double V = or_v_closed(or_value(seed, TAG_SPLIT, id, 2 * i + 1));
        double X = alpha + h * (V - 0.5) * or_recip(U);
        if (X < 0.0 || X >= (double)c + 1.0) continue;
        uint64_t k = (uint64_t)X;
        double T = or_sd_fixed(M, k, l0) + or_sd_fixed(c - M, c - k, l1) + (double)((int64_t)k - (int64_t)M) * logr;
        if (2.0 * or_log(U) <= T) { *out = k; return OR_OK; }
    }
    return OR_EITER;
}

/* ------------------------------------------------------------------------ */
/* Split tree (Sec. 3.1 Algorithm R, Sec. 3.2 Algorithm P, Sec. 4.5).       */
/* Reading: a static depth D instead of the adaptive "n < n0" stop, as in   */
/* Algorithm P's fixed PE tree and the p' >> p fixed jobs of Sec. 4.5.      */
/* ------------------------------------------------------------------------ */

/* Smallest D >= 0 with n <= n0 * 2^D, then lowered until 2^D <= N. */
int or_depth(uint64_t n, uint64_t N, uint32_t n0)
{
    int D = 0;
    while ((u128)n > ((u128)n0 << D)) ++D;
    while (D > 0 && ((u128)1 << D) > (u128)N) --D;
    return D;
}

/* Argument checks shared by every entry point of the oracle. */
static int check_args(uint64_t n, uint64_t N, uint32_t n0, int with_replacement)
{
    if (n0 == 0) return OR_EINVAL;
    if (N > (1ull << 62)) return OR_EINVAL;
    if (n > 0 && N == 0) return OR_EINVAL;
    if (!with_replacement && n > N) return OR_EINVAL;
    return OR_OK;
}

/* Recursive descent in heap order: node v covers [lo, lo+S) and holds c
 * samples.  Its left child 2v gets [lo, lo+floor(S/2)) and L samples, the
 * right child 2v+1 the rest (Algorithm R's split at floor(N/2)).  A node with
 * no samples draws nothing.  Leaf records are (lo, s, n', offset). */
static int tree_rec(uint64_t seed, int kind, uint64_t v, uint64_t lo, uint64_t S, uint64_t c,
                    int level, int D, uint64_t* recs, uint64_t* offset)
{
    if (level == D) {
        uint64_t i = v - (1ull << D);
        recs[4 * i + 0] = lo;
        recs[4 * i + 1] = S;
        recs[4 * i + 2] = c;
        recs[4 * i + 3] = *offset;
        *offset += c;
        return OR_OK;
    }
    uint64_t K = S / 2;
    uint64_t L = 0;
    if (c > 0) {
        int rc = kind == 1 ? or_bin(seed, v, c, K, S, &L) : or_hg(seed, v, c, K, S, &L);
        if (rc) return rc;
    }
    int rc = tree_rec(seed, kind, 2 * v, lo, K, L, level + 1, D, recs, offset);
    if (rc) return rc;
    return tree_rec(seed, kind, 2 * v + 1, lo + K, S - K, c - L, level + 1, D, recs, offset);
}

/* Leaf records of the split tree; kind 0 = hypergeometric splits, 1 =
 * binomial splits.  recs holds 4 * 2^D words. */
int or_tree(uint64_t n, uint64_t N, uint64_t seed, uint32_t n0, int kind, uint64_t* recs,
            uint64_t max_leaves, int* D_out)
{
    int rc = check_args(n, N, n0, kind == 1);
    if (rc) return rc;
    int D = or_depth(n, N, n0);
    *D_out = D;
    if (N == 0) return OR_OK;
    if ((1ull << D) > max_leaves) return OR_ECAPACITY;
    uint64_t offset = 0;
    return tree_rec(seed, kind, 1, 0, N, n, 0, D, recs, &offset);
}

/* ------------------------------------------------------------------------ */
/* Base cases.                                                              */
/* ------------------------------------------------------------------------ */

/* A plain open-addressing set of 64-bit keys (UINT64_MAX marks empty). */
typedef struct { uint64_t* slot; uint64_t mask; } hset;

static int hset_init(hset* h, uint64_t expect)
{
    uint64_t cap = 16;
    while (cap < 2 * expect + 16) cap <<= 1;
    h->slot = (uint64_t*)malloc(cap * sizeof(uint64_t));
    if (!h->slot) return OR_ENOMEM;
    memset(h->slot, 0xFF, cap * sizeof(uint64_t));
    h->mask = cap - 1;
    return OR_OK;
}

/* Inserts v; returns 1 if it was new, 0 if it was already present. */
static int hset_insert(hset* h, uint64_t v)
{
    uint64_t i = (v * 0x9E3779B97F4A7C15ull) >> 20 & h->mask;
    for (;;) {
        if (h->slot[i] == UINT64_MAX) { h->slot[i] = v; return 1; }
        if (h->slot[i] == v) return 0;
        i = (i + 1) & h->mask;
    }
}

static int cmp_u64(const void* a, const void* b)
{
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* The first k distinct valid candidates of stream (tag, id) over [0, s), in
 * candidate order (Algorithm H, Sec. 2: draw, reject what is already in the
 * table).  Writes them unsorted to sel[0..k).  Candidate indices are limited
 * so that the stream's block counter stays below 2^32. */
static int first_distinct(uint64_t seed, uint32_t tag, uint64_t id, uint64_t s, uint64_t k, uint64_t* sel)
{
    if (k == 0) return OR_OK;
    hset h;
    if (hset_init(&h, k)) return OR_ENOMEM;
    uint64_t limit = s <= (1ull << 32) ? (1ull << 34) : (1ull << 33);
    uint64_t got = 0;
    for (uint64_t j = 0; got < k; ++j) {
        if (j >= limit) { free(h.slot); return OR_EITER; }
        uint64_t v;
        if (!or_candidate(seed, tag, id, s, j, &v)) continue;
        if (hset_insert(&h, v)) sel[got++] = v;
    }
    free(h.slot);
    return OR_OK;
}

/* Leaf H: n' distinct values of [0, s) for leaf node id, sorted (Algorithm H
 * with sorted output, Sec. 4.1).  Reading of the n > N/2 rule (Sec. 2) per
 * leaf: when 2n' > s, select k = s - n' values and output the rest.
 * out receives lo + v + 1 (1-based values). */
int or_leaf_h(uint64_t seed, uint64_t id, uint64_t lo, uint64_t s, uint64_t np, uint64_t* out)
{
    if (np == 0) return OR_OK;
    int complement = (2 * (u128)np > s);
    uint64_t k = complement ? s - np : np;
    uint64_t* sel = (uint64_t*)malloc((k + 1) * sizeof(uint64_t));
    if (!sel) return OR_ENOMEM;
    int rc = first_distinct(seed, TAG_LEAF_H, id, s, k, sel);
    if (rc) { free(sel); return rc; }
    qsort(sel, k, sizeof(uint64_t), cmp_u64);
    if (!complement) {
        for (uint64_t j = 0; j < k; ++j) out[j] = lo + sel[j] + 1;
    } else {
        uint64_t j = 0, w = 0;
        for (uint64_t v = 0; v < s; ++v) {
            if (j < k && sel[j] == v) { ++j; continue; }
            out[w++] = lo + v + 1;
        }
    }
    free(sel);
    return OR_OK;
}

/* Leaf WR (sampling with replacement, Sec. 4.6): the first n' valid
 * candidates of stream (LEAF_WR, id), sorted as a multiset. */
int or_leaf_wr(uint64_t seed, uint64_t id, uint64_t lo, uint64_t s, uint64_t np, uint64_t* out)
{
    if (np == 0) return OR_OK;
    uint64_t limit = s <= (1ull << 32) ? (1ull << 34) : (1ull << 33);
    uint64_t got = 0;
    for (uint64_t j = 0; got < np; ++j) {
        if (j >= limit) return OR_EITER;
        uint64_t v;
        if (!or_candidate(seed, TAG_LEAF_WR, id, s, j, &v)) continue;
        out[got++] = v;
    }
    qsort(out, np, sizeof(uint64_t), cmp_u64);
    for (uint64_t j = 0; j < np; ++j) out[j] = lo + out[j] + 1;
    return OR_OK;
}

/* Geometric skips over positions [start, end) with success probability p
 * (0 < p < 1): position pos is chosen when the skip lands on it.  Skip
 * length floor(ln U / ln(1-p)) is Geometric(p) (Sec. 2, Algorithm B).
 * Calls emit(pos) for each chosen position in increasing order and returns
 * the number chosen, or -1 if the stream's block counter would run out. */
typedef void (*emit_fn)(void* ctx, uint64_t pos);

static int64_t geometric_skips(uint64_t seed, uint32_t tag, uint64_t id, double p,
                               uint64_t start, uint64_t end, emit_fn emit, void* ctx)
{
    /* Reading: the quotient ln U / ln(1-p) is taken as ln U times R =
     * RN(1 / ln(1-p)), one division per range (within 2 ulp of the quotient);
     * U = 1 gives skip 0 even where R overflows (p below 2^-1024). */
    double R = 1.0 / or_log1p(-p);
    int64_t pos = (int64_t)start - 1;
    int64_t count = 0;
    for (uint64_t j = 0;; ++j) {
        if (j >= (1ull << 33)) return -1;
        double U = or_u_open(or_value(seed, tag, id, j));
        double q = (U == 1.0) ? 0.0 : or_log(U) * R;
        if (q >= 4611686018427387904.0) break;           /* 2^62 */
        pos = pos + (int64_t)floor(q) + 1;
        if (pos >= (int64_t)end) break;
        emit(ctx, (uint64_t)pos);
        ++count;
    }
    return count;
}

typedef struct { uint64_t* buf; uint64_t n; uint64_t cap; } vec64;

static void vec_push(void* ctx, uint64_t pos)
{
    vec64* v = (vec64*)ctx;
    if (v->n == v->cap) {
        uint64_t nc = v->cap ? 2 * v->cap : 1024;
        uint64_t* nb = (uint64_t*)realloc(v->buf, nc * sizeof(uint64_t));
        if (!nb) { v->cap = 0; return; }   /* caller sees n < count */
        v->buf = nb; v->cap = nc;
    }
    v->buf[v->n++] = pos;
}

/* Leaf B (Algorithm B of Ahrens and Dieter as the base case, Sec. 2 and
 * Sec. 4.7): Bernoulli-sample [0, s) with rho slightly above n'/s, retry if
 * fewer than n' positions came out, then remove c - n' of the c positions,
 * chosen by Algorithm H over their indices [0, c).  Reading: rho =
 * min(1, (n' + 3 sqrt(n') + 10) / s); attempt a uses stream LEAF_B + 256a;
 * the removal uses stream FIXUP. */
int or_leaf_b(uint64_t seed, uint64_t id, uint64_t lo, uint64_t s, uint64_t np, uint64_t* out)
{
    if (np == 0) return OR_OK;
    double dn = (double)np;
    double rho = (dn + 3.0 * sqrt(dn) + 10.0) / (double)s;
    if (rho > 1.0) rho = 1.0;
    vec64 pos = { 0, 0, 0 };
    int attempt;
    for (attempt = 0; attempt < 64; ++attempt) {
        pos.n = 0;
        if (rho == 1.0) {
            for (uint64_t v = 0; v < s; ++v) vec_push(&pos, v);
        } else {
            int64_t cnt = geometric_skips(seed, TAG_LEAF_B + 256u * (uint32_t)attempt, id, rho, 0, s,
                                          vec_push, &pos);
            if (cnt < 0) { free(pos.buf); return OR_EITER; }
            if ((uint64_t)cnt != pos.n) { free(pos.buf); return OR_ENOMEM; }
        }
        if (pos.n >= np) break;
    }
    if (attempt == 64) { free(pos.buf); return OR_EITER; }
    uint64_t c = pos.n, drop = c - np;
    uint64_t* sel = (uint64_t*)malloc((drop + 1) * sizeof(uint64_t));
    if (!sel) { free(pos.buf); return OR_ENOMEM; }
    int rc = first_distinct(seed, TAG_FIXUP, id, c, drop, sel);
    if (rc) { free(sel); free(pos.buf); return rc; }
    qsort(sel, drop, sizeof(uint64_t), cmp_u64);
    uint64_t j = 0, w = 0;
    for (uint64_t i = 0; i < c; ++i) {
        if (j < drop && sel[j] == i) { ++j; continue; }
        out[w++] = lo + pos.buf[i] + 1;
    }
    free(sel);
    free(pos.buf);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Whole samples.                                                           */
/* ------------------------------------------------------------------------ */

/* kind 0: without replacement, leaf H.  kind 1: with replacement (binomial
 * splits, leaf WR).  kind 2: without replacement, leaf B.
 * out receives n values (1-based) in non-decreasing order. */
int or_sample(uint64_t n, uint64_t N, uint64_t seed, uint32_t n0, int kind, uint64_t* out)
{
    int rc = check_args(n, N, n0, kind == 1);
    if (rc) return rc;
    if (n == 0) return OR_OK;
    int D = or_depth(n, N, n0);
    uint64_t L = 1ull << D;
    uint64_t* recs = (uint64_t*)malloc(4 * L * sizeof(uint64_t));
    if (!recs) return OR_ENOMEM;
    int Dd;
    rc = or_tree(n, N, seed, n0, kind == 1 ? 1 : 0, recs, L, &Dd);
    for (uint64_t i = 0; i < L && rc == OR_OK; ++i) {
        uint64_t id = L + i, lo = recs[4 * i], s = recs[4 * i + 1], np = recs[4 * i + 2], off = recs[4 * i + 3];
        if (kind == 0) rc = or_leaf_h(seed, id, lo, s, np, out + off);
        else if (kind == 1) rc = or_leaf_wr(seed, id, lo, s, np, out + off);
        else rc = or_leaf_b(seed, id, lo, s, np, out + off);
    }
    free(recs);
    return rc;
}

/* Output of one leaf by index i (0-based, left to right), for sampled
 * checks of large runs: recs are the leaf records from or_tree. */
int or_leaf(uint64_t seed, int kind, int D, uint64_t i, const uint64_t* rec, uint64_t* out)
{
    uint64_t id = (1ull << D) + i;
    if (kind == 0) return or_leaf_h(seed, id, rec[0], rec[1], rec[2], out);
    if (kind == 1) return or_leaf_wr(seed, id, rec[0], rec[1], rec[2], out);
    return or_leaf_b(seed, id, rec[0], rec[1], rec[2], out);
}

/* Sorted range query: the values of the full sample lying in [a, b)
 * (1-based values), in order; the sample of Sec. 4.1 restricted to a
 * subrange.  Leaves whose value range misses [a, b) contribute nothing. */
int or_range_query(uint64_t n, uint64_t N, uint64_t seed, uint32_t n0, int kind, uint64_t a, uint64_t b,
                   uint64_t* out, uint64_t cap, uint64_t* count)
{
    *count = 0;
    int rc = check_args(n, N, n0, kind == 1);
    if (rc) return rc;
    if (n == 0 || a >= b) return OR_OK;
    int D = or_depth(n, N, n0);
    uint64_t L = 1ull << D;
    uint64_t* recs = (uint64_t*)malloc(4 * L * sizeof(uint64_t));
    if (!recs) return OR_ENOMEM;
    int Dd;
    rc = or_tree(n, N, seed, n0, kind == 1 ? 1 : 0, recs, L, &Dd);
    uint64_t got = 0;
    for (uint64_t i = 0; i < L && rc == OR_OK; ++i) {
        uint64_t lo = recs[4 * i], s = recs[4 * i + 1], np = recs[4 * i + 2];
        if (np == 0 || lo + s + 1 <= a || lo + 1 >= b) continue;   /* values lo+1 .. lo+s */
        uint64_t* tmp = (uint64_t*)malloc(np * sizeof(uint64_t));
        if (!tmp) { rc = OR_ENOMEM; break; }
        rc = or_leaf(seed, kind, D, i, recs + 4 * i, tmp);
        for (uint64_t j = 0; j < np && rc == OR_OK; ++j) {
            if (tmp[j] < a || tmp[j] >= b) continue;
            if (got < cap) out[got] = tmp[j];
            ++got;
        }
        free(tmp);
    }
    free(recs);
    *count = got;
    if (rc == OR_OK && got > cap) rc = OR_ECAPACITY;
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Bernoulli sampling by independent subranges (Sec. 4.7).                 */
/* ------------------------------------------------------------------------ */

/* Chunk size exponent: smallest c >= 0 with 2^c p >= n0, at most 62. */
int or_bern_chunk_log2(double p, uint32_t n0)
{
    int c = 0;
    while (c < 62 && ldexp(1.0, c) * p < (double)n0) ++c;
    return c;
}

typedef struct { uint64_t* out; uint64_t cap; uint64_t got; } bern_sink;

static void bern_emit(void* ctx, uint64_t pos)
{
    bern_sink* b = (bern_sink*)ctx;
    if (b->got < b->cap) b->out[b->got] = pos + 1;
    b->got++;
}

/* Bernoulli(p) sample of positions [0, N), restricted to the window [a, b)
 * whose ends are multiples of the chunk size (or b = N).  Chunk i covers
 * [iC, min((i+1)C, N)) and draws from stream (BERN, i), so chunks are
 * independent (Sec. 4.7).  Writes 1-based positions, sets *count to the
 * number in the window even when it exceeds cap (then ECAPACITY). */
int or_bernoulli(double p, uint64_t N, uint64_t seed, uint32_t n0, uint64_t a, uint64_t b,
                 uint64_t* out, uint64_t cap, uint64_t* count)
{
    *count = 0;
    if (!(p >= 0.0 && p <= 1.0) || n0 == 0 || N > (1ull << 62) || a > b || b > N) return OR_EINVAL;
    int cl = or_bern_chunk_log2(p, n0);
    uint64_t C = 1ull << cl;
    if (a % C != 0 || (b % C != 0 && b != N)) return OR_EINVAL;
    bern_sink sink = { out, cap, 0 };
    if (p == 0.0 || a == b) return OR_OK;
    if (p == 1.0) {
        for (uint64_t x = a; x < b; ++x) bern_emit(&sink, x);
    } else {
        for (uint64_t i = a / C; i * C < b; ++i) {
            uint64_t start = i * C, end = start + C < N ? start + C : N;
            if (geometric_skips(seed, TAG_BERN, i, p, start, end, bern_emit, &sink) < 0) return OR_EITER;
        }
    }
    *count = sink.got;
    return sink.got > cap ? OR_ECAPACITY : OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Bernoulli sampling by its size (Sec. 4.7, relation to Bernoulli          */
/* sampling): the number of chosen positions follows BIN(N, p); drawing it  */
/* first and then that many positions without replacement gives a          */
/* Bernoulli(p) sample with no logarithm per position.                      */
/* ------------------------------------------------------------------------ */

/* The size: BIN(N, p) as the binomial deviate of stream (SPLIT, 0) -- a node
 * id the split tree never uses.  Reading: p is taken as K / 2^62 with
 * K = floor(p 2^62 + 1/2) (p 2^62 is exact in double; the rounding changes p
 * by at most 2^-63); for p > 1/2 the size is N - BIN(N, K'/2^62) with K'
 * from 1 - p (exact for p in [1/2, 1]), as or_bin takes K/S <= 1/2. */
int or_bernoulli_size(double p, uint64_t N, uint64_t seed, uint64_t* count)
{
    *count = 0;
    if (!(p >= 0.0 && p <= 1.0) || N > (1ull << 62)) return OR_EINVAL;
    int flip = p > 0.5;
    double q = flip ? 1.0 - p : p;
    uint64_t K = (uint64_t)floor(q * 0x1p62 + 0.5);
    uint64_t c = 0;
    int rc = or_bin(seed, 0, N, K, 1ull << 62, &c);
    if (rc) return rc;
    *count = flip ? N - c : c;
    return OR_OK;
}

/* The sample: the or_bernoulli_size positions drawn without replacement
 * (or_sample, kind H, the same seed; the tree's nodes use ids from 1), as
 * 1-based positions, restricted to the window [a, b) of 0-based positions
 * (any ends) as a range query of that sample.  *total receives the size. */
int or_bernoulli_by_size(double p, uint64_t N, uint64_t seed, uint32_t n0, uint64_t a, uint64_t b,
                         uint64_t* out, uint64_t cap, uint64_t* count, uint64_t* total)
{
    *count = 0;
    *total = 0;
    if (n0 == 0 || a > b || b > N) return OR_EINVAL;
    uint64_t n = 0;
    int rc = or_bernoulli_size(p, N, seed, &n);
    if (rc) return rc;
    *total = n;
    return or_range_query(n, N, seed, n0, 0, a + 1, b + 1, out, cap, count);
}

/* ------------------------------------------------------------------------ */
/* Sampling from a union of uneven segments (Sec. 4.3, uneven distribution  */
/* of the sampled universe): owner computes.                                */
/* ------------------------------------------------------------------------ */

/* Weyl step for the segments' keys: segment i samples with key
 * seed + (i + 1) * W (mod 2^64), W odd, so the keys differ per segment. */
static const uint64_t UNION_WEYL = 0x9E3779B97F4A7C15ull;

uint64_t or_union_key(uint64_t seed, uint64_t i) { return seed + (i + 1) * UNION_WEYL; }

/* Number of samples per segment.  Reading: the binomial tree of Sec. 4.3 over
 * the p segments is the binary tree of power-of-two aligned ranges, padded to
 * P = 2^ceil(log2 p) segments (the padding holds no elements): node v
 * (heap-numbered, root 1) covers segments [i 2^h, (i+1) 2^h) and its element
 * count is the sum of their sizes, added bottom-up; top-down, a node with c
 * samples gives HG(c, L_left, L_left + L_right) of them to its left child --
 * the hypergeometric deviate of stream (SPLIT, v) with the given seed -- and
 * the rest to its right child.  counts[i] = the samples of segment i. */
int or_union_counts(const uint64_t* L, uint32_t p, uint64_t n, uint64_t seed, uint64_t* counts)
{
    if (p == 0) return n == 0 ? OR_OK : OR_EINVAL;
    uint64_t P = 1;
    while (P < p) P <<= 1;
    uint64_t* sum = (uint64_t*)calloc(2 * P, sizeof(uint64_t));
    uint64_t* cnt = (uint64_t*)calloc(2 * P, sizeof(uint64_t));
    if (!sum || !cnt) { free(sum); free(cnt); return OR_ENOMEM; }
    int rc = OR_OK;
    u128 total = 0;
    for (uint32_t i = 0; i < p; ++i) { sum[P + i] = L[i]; total += L[i]; }
    if (total > ((u128)1 << 62) || n > (uint64_t)total) rc = OR_EINVAL;
    for (uint64_t v = P - 1; v >= 1 && rc == OR_OK; --v) sum[v] = sum[2 * v] + sum[2 * v + 1];
    if (rc == OR_OK) cnt[1] = n;
    for (uint64_t v = 1; v < P && rc == OR_OK; ++v) {
        uint64_t left = 0;
        rc = or_hg(seed, v, cnt[v], sum[2 * v], sum[v], &left);
        cnt[2 * v] = left;
        cnt[2 * v + 1] = cnt[v] - left;
    }
    for (uint32_t i = 0; i < p && rc == OR_OK; ++i) counts[i] = cnt[P + i];
    free(sum);
    free(cnt);
    return rc;
}

/* The union's sample: segment i's counts[i] samples are the sample without
 * replacement of that size from its L_i elements (or_sample, kind H, key
 * or_union_key(seed, i), n0) as 1-based positions within the segment;
 * segments follow each other in order in out[]. */
int or_union_sample(const uint64_t* L, uint32_t p, uint64_t n, uint64_t seed, uint32_t n0, uint64_t* out,
                    uint64_t* counts)
{
    if (n0 == 0) return OR_EINVAL;
    int rc = or_union_counts(L, p, n, seed, counts);
    uint64_t off = 0;
    for (uint32_t i = 0; i < p && rc == OR_OK; ++i) {
        rc = or_sample(counts[i], L[i], or_union_key(seed, i), n0, 0, out + off);
        off += counts[i];
    }
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Online sorted sampling by peeling (Sec. 4.1, last paragraph: split off a */
/* range of about N n0 / n positions at a time).                            */
/* ------------------------------------------------------------------------ */

/* The sample as its batches, in order.  With n_t samples left in the N_t
 * positions after the first lo_t (n_0 = n, N_0 = N, lo_0 = 0), batch t
 * (t = 0, 1, ...) peels the next m_t = ceil(N_t n0 / n_t) positions and
 * takes c_t = HG(n_t, m_t, N_t) of the samples, the deviate of stream
 * (SPLIT, t + 1); once m_t >= N_t the batch is the rest (m_t = N_t,
 * c_t = n_t) and the last.  Batch t's values are leaf H of node t + 1 over
 * [lo_t, lo_t + m_t) with c_t samples; lo_{t+1} = lo_t + m_t, N_{t+1} =
 * N_t - m_t, n_{t+1} = n_t - c_t.  out[] receives the batches one after the
 * other (the sample in increasing order), counts[t] = c_t, *nbatches the
 * number of batches (at most max_batches, else OR_ECAPACITY). */
int or_peel_sample(uint64_t n, uint64_t N, uint64_t seed, uint32_t n0, uint64_t* out, uint64_t* counts,
                   uint64_t max_batches, uint64_t* nbatches)
{
    *nbatches = 0;
    if (n0 == 0 || N > (1ull << 62) || n > N) return OR_EINVAL;
    uint64_t nr = n, Nr = N, lo = 0, off = 0, t = 0;
    while (nr > 0) {
        if (t >= max_batches) return OR_ECAPACITY;
        const u128 m128 = ((u128)Nr * n0 + nr - 1) / nr;
        uint64_t m, c;
        if (m128 >= Nr) {
            m = Nr;
            c = nr;
        } else {
            m = (uint64_t)m128;
            int rc = or_hg(seed, t + 1, nr, m, Nr, &c);
            if (rc) return rc;
        }
        int rc = or_leaf_h(seed, t + 1, lo, m, c, out + off);
        if (rc) return rc;
        counts[t] = c;
        off += c;
        lo += m;
        Nr -= m;
        nr -= c;
        ++t;
    }
    *nbatches = t;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Sampling with replacement from a d-dimensional box by bisection (Sec.    */
/* 4.6, sampling in various spaces: random points in a rectangle).          */
/* ------------------------------------------------------------------------ */

#define OR_POINTS_MAXD 4

typedef struct {
    uint64_t seed;
    uint32_t d;
    int D;
    uint64_t* out;     /* n * d coordinates */
    uint64_t* tmp;     /* room for the largest leaf */
    uint64_t off;      /* points written so far */
} points_ctx;

/* The dimension a box is halved along: the one of largest extent, the
 * lowest such index on ties. */
static uint32_t split_dim(const uint64_t* e, uint32_t d)
{
    uint32_t k = 0;
    for (uint32_t j = 1; j < d; ++j)
        if (e[j] > e[k]) k = j;
    return k;
}

/* Node v is the box [o_k, o_k + e_k) in every dimension k and holds c
 * points.  With ks = split_dim(e), its left child is the box with e_ks
 * replaced by floor(e_ks / 2) and gets BIN(c, floor(e_ks / 2), e_ks) of the
 * points (stream (SPLIT, v); the volumes are in that ratio); the right child
 * is the rest of the box. */
static int points_rec(points_ctx* P, uint64_t v, int level, const uint64_t* o, const uint64_t* e, uint64_t c)
{
    const uint32_t d = P->d;
    if (level == P->D) {
        if (c == 0) return OR_OK;
        /* a leaf draws its points as indices into its box (row-major,
         * dimension 0 most significant): leaf WR of the leaf's node over
         * [0, volume), then each index decoded into coordinates */
        uint64_t vol = 1;
        for (uint32_t k = 0; k < d; ++k) vol *= e[k];
        int rc = or_leaf_wr(P->seed, v, 0, vol, c, P->tmp);
        if (rc) return rc;
        for (uint64_t j = 0; j < c; ++j) {
            uint64_t x = P->tmp[j] - 1;
            uint64_t* pt = P->out + (P->off + j) * d;
            for (uint32_t k = d; k-- > 0;) {
                pt[k] = o[k] + x % e[k];
                x /= e[k];
            }
        }
        P->off += c;
        return OR_OK;
    }
    const uint32_t ks = split_dim(e, d);
    const uint64_t half = e[ks] / 2;
    uint64_t cl = 0;
    if (c > 0) {
        int rc = or_bin(P->seed, v, c, half, e[ks], &cl);
        if (rc) return rc;
    }
    uint64_t oc[OR_POINTS_MAXD], ec[OR_POINTS_MAXD];
    for (uint32_t k = 0; k < d; ++k) { oc[k] = o[k]; ec[k] = e[k]; }
    ec[ks] = half;
    int rc = points_rec(P, 2 * v, level + 1, oc, ec, cl);
    if (rc) return rc;
    oc[ks] = o[ks] + half;
    ec[ks] = e[ks] - half;
    return points_rec(P, 2 * v + 1, level + 1, oc, ec, c - cl);
}

/* n points drawn uniformly and independently from the box [0, E_0) x ... x
 * [0, E_{d-1}) (1 <= d <= 4, every E_k >= 1, volume V <= 2^62): the depth
 * D is that of the one-dimensional tree with N = V (or_depth), the tree
 * halves boxes as points_rec says, and out[] receives the leaves' points in
 * heap order, d coordinates per point (0-based). */
int or_points(uint64_t n, uint32_t d, const uint64_t* E, uint64_t seed, uint32_t n0, uint64_t* out)
{
    if (d == 0 || d > OR_POINTS_MAXD || n0 == 0) return OR_EINVAL;
    u128 V = 1;
    for (uint32_t k = 0; k < d; ++k) {
        if (E[k] == 0) return OR_EINVAL;
        V *= E[k];
        if (V > ((u128)1 << 62)) return OR_EINVAL;
    }
    if (n == 0) return OR_OK;
    points_ctx P;
    P.seed = seed;
    P.d = d;
    P.D = or_depth(n, (uint64_t)V, n0);
    P.out = out;
    P.off = 0;
    P.tmp = (uint64_t*)malloc(n * sizeof(uint64_t));
    if (!P.tmp) return OR_ENOMEM;
    uint64_t o[OR_POINTS_MAXD] = {0, 0, 0, 0};
    int rc = points_rec(&P, 1, 0, o, E, n);
    free(P.tmp);
    return rc;
}

