// rs_tree_warp.cuh -- split-tree nodes processed a warp at a time.
//
// The split deviates (Sec. 3: hypergeometric, Sec. 4.6: binomial) are
// rejection loops whose trial count varies per node, and their log-factorial
// differences take different branches per node.  FP64 instructions cost the
// same however many lanes of a warp are active, so a warp here keeps all
// lanes busy:
//  - lane refill: a warp owns a batch of nodes; a lane whose node is done
//    takes the next one, so trial counts no longer idle lanes;
//  - cooperative logarithms: each ratio-of-uniforms trial first records the
//    arguments of every logarithm it needs (ln U, ln of 1 + D/Y, and in a
//    node's first round those of the differences' fixed ends), the whole
//    warp evaluates them together, and
//    each lane then assembles its acceptance test from the results in
//    exactly the operations and order of the scalar definition
//    (rs_deviates.cuh), so the results are the same bits;
//  - parallel trials: on levels with few nodes a node gets a group of G
//    lanes, lane r of the group evaluating trial t + r.  Trial t of node v
//    uses only Philox block (v, t), so trials are independent; the node
//    takes the lowest accepted trial index, exactly the sequential loop's
//    choice, after about one round instead of the slowest node's many;
//  - parallel terms (tree_terms_warp, the smallest levels): an FP64 warp
//    instruction costs the same whatever the number of active lanes, so a
//    level with few nodes is bound by the length of one trial's instruction
//    stream.  There the four log-factorial differences of a trial go to
//    four lanes, which run one stream of the scalar dsd() side by side, and
//    are summed in the scalar order after shuffles.
#pragma once
#include "rs_deviates.cuh"
#include "rs_ff.cuh"

namespace rs {

constexpr int kLogSlots = 16;   // per lane per trial: up to 9 logarithm arguments, then up to 4 saved reciprocals

// A lane's slots for one trial: logarithm arguments fill them from the
// front (the warp then replaces each by its logarithm); reciprocals that the
// evaluation needs again are saved from the back.
struct LfdArgs {
    double* a;
    int n, ns;
    RS_DEV void push(double v) { a[n++] = v; }
    RS_DEV void save(double v) { a[kLogSlots - 1 - ns++] = v; }
};
struct LfdLogs {
    const double* l;
    int n, ns;
    RS_DEV double next() { return l[n++]; }
    RS_DEV double saved() { return l[kLogSlots - 1 - ns++]; }
};

// The fixed-end difference dsd_fixed(P, Q, lnP) (rs_math.cuh) in two
// halves: sdf_args lists the logarithm arguments it needs, sdf_eval computes
// the value from their logarithms, consumed in the same order.  One call on
// (max, min) with the sign after, so that lanes whose arguments come in
// opposite orders run one copy.
RS_DEV void sdf_args(uint64_t P, uint64_t Q, LfdArgs& A) {
    const bool p_big = P >= Q;
    const uint64_t x = p_big ? P : Q, y = p_big ? Q : P, d = x - y;
    if (d == 0 || x < 256) return;
    if (y < 256) {
        if (!p_big) A.push((double)x);
        return;
    }
    const double rY = drecip((double)y);
    A.push(log1p_pos_u((double)d * rY));
    A.save(rY);
}
RS_DEV double sdf_eval(uint64_t P, uint64_t Q, double lnP, const double* __restrict__ tab, LfdLogs& L) {
    const bool p_big = P >= Q;
    const uint64_t x = p_big ? P : Q, y = p_big ? Q : P, d = x - y;
    double v;
    if (d == 0) return 0.0;
    if (x < 256) {
        v = tab[x] - tab[y];
    } else {
        const double X = (double)x;
        if (y < 256) {
            const double lx = p_big ? lnP : L.next();
            v = ((X + 0.5) * lx - X + RS_HL2PI + stirling_tail(drecip(X))) - tab[y];
        } else {
            const double D = (double)d;
            const double rY = L.saved();
            const double lp = log1p_pos_finish(D * rY, L.next());
            const double ly = p_big ? lnP - lp : lnP;
            v = (X + 0.5) * lp + D * ly - D + (stirling_tail(drecip(X)) - stirling_tail(rY));
        }
    }
    return p_big ? v : -v;
}

// The fixed ends of the test's differences: M and a - M (binomial), or M,
// a - M, b - M and m + M with m = S - a - b (hypergeometric); the moving
// ends replace M by the candidate k.
// Parameters of one node's ratio-of-uniforms loop (rs_deviates.cuh).
struct RouNode {
    uint64_t v;          // node id
    uint64_t lo, S, c, off, K;
    uint64_t a, b, M;    // hypergeometric: reduced draws/successes; binomial: a = c
    uint64_t n_in, Kp;   // un-reduction of the hypergeometric result
    double mu, h, alpha, top, logr;   // FP64 parameters, as defined (set up when a trial first needs them)
    float fa, fh, ftop;  // alpha, h, top in single precision, for the guards
    float logrf;         // binomial: ln(p / (1 - p)) in single precision, for the guard
    FF ffa, ffh, fflogr; // alpha, h, ln(p / (1 - p)) in float-float, for the second guard (rs_ff.cuh)
    double lnP[4];       // ln of the fixed ends (lanes kernel), once per node
    uint32_t trial;
    bool flipN, flipK;
    bool fresh;          // set up, fixed-end logarithms not yet taken
    bool have64;         // h, alpha, top, logr are set
    bool haveff;         // ffa, ffh, fflogr are set
};

// The hat's constants 2 sqrt(2/e) and 3 - 2 sqrt(3/e) in single precision.
constexpr float kHatD1f = 1.71552777f;
constexpr float kHatD2f = 0.898916162f;

// The node's FP64 parameters exactly as the definition computes them
// (rs_deviates.cuh).
template <bool WR>
RS_DEV void setup64(RouNode* q, const double* __restrict__ tab) {
    if (WR) {
        const double p = (double)q->K / (double)q->S;
        const double mu = (double)q->a * p;
        const double var = mu * (1.0 - p);
        q->mu = mu;
        q->h = RS_HAT_D1 * sqrt(var + 0.5) + RS_HAT_D2;
        q->alpha = mu + 0.5;
        const double rr = p / (1.0 - p);
        q->logr = (rr == 1.0) ? 0.0 : dlog(rr, tab);
    } else {
        const uint64_t S = q->S, a = q->a, b = q->b;
        const double rS = drecip((double)S);
        const double mu = ((double)a * (double)b) * rS;
        const double var = mu * ((double)(S - a) * rS) * ((double)(S - b) * drecip((double)(S - 1)));
        q->mu = mu;
        q->h = RS_HAT_D1 * sqrt(var + 0.5) + RS_HAT_D2;
        q->alpha = mu + 0.5;
    }
    q->top = (double)q->a + 1.0;
    q->have64 = true;
}

// The node's alpha, h (and ln(p / (1 - p))) in float-float, for the second
// guard: the definition's formulas (setup64) with every operation in
// float-float (each within 2^-42 of its result), the logarithm of K / (S - K)
// as a difference of two fixed-point logarithms (within 2^-54).
template <bool WR>
RS_DEV void setupff(RouNode* q, const double* __restrict__ tab) {
    const FFParams f = WR ? ff_bin_params(q->a, q->K, q->S, tab) : ff_hg_params(q->a, q->b, q->S);
    q->ffa = f.alpha;
    q->ffh = f.h;
    q->fflogr = f.logr;
    q->haveff = true;
}

template <bool WR>
RS_DEV uint64_t fixed_end(const RouNode& q, int j) {
    if (WR) return j == 0 ? q.M : (j == 1 ? q.a - q.M : 0);
    const uint64_t m = q.S - q.a - q.b;
    return j == 0 ? q.M : (j == 1 ? q.a - q.M : (j == 2 ? q.b - q.M : m + q.M));
}
template <bool WR>
RS_DEV uint64_t moving_end(const RouNode& q, int j, uint64_t k) {
    if (WR) return j == 0 ? k : (j == 1 ? q.a - k : 0);
    const uint64_t m = q.S - q.a - q.b;
    return j == 0 ? k : (j == 1 ? q.a - k : (j == 2 ? q.b - k : m + k));
}

RS_DEV void write_children(NodeRec* __restrict__ rec, uint64_t v, const NodeRec& r, uint64_t K, uint64_t L) {
    rec[2 * v] = NodeRec{r.lo, K, L, r.off};
    rec[2 * v + 1] = NodeRec{r.lo + K, r.S - K, r.c - L, r.off + L};
}

// Prepares node v.  Returns true if the node needs ratio-of-uniforms trials
// (state in *q); otherwise the node is finished here (children written):
// no samples, a fast path, or inversion.  The choice between inversion and
// ratio-of-uniforms (mean below 16) is taken from the single-precision mean
// when that is clear of 16 by its error bound (6 2^-24 relative), else from
// the FP64 mean as defined.  The FP64 parameters are set up here when
// eager64, else by the first trial that needs them.
template <bool WR>
RS_DEV bool node_setup(NodeRec* __restrict__ rec, uint64_t v, Key2 key, const double* __restrict__ tab, int* status,
                       RouNode* q, bool writer = true, bool eager64 = true) {
    // written by the level before, possibly by another SM of the same launch
    // (the fused top levels): read past this SM's L1
    const ulonglong2* pr = reinterpret_cast<const ulonglong2*>(rec + v);
    const ulonglong2 r0 = __ldcg(pr), r1 = __ldcg(pr + 1);
    const NodeRec r{r0.x, r0.y, r1.x, r1.y};
    const uint64_t K = r.S / 2;
    auto finish = [&](uint64_t L) {
        if (writer) write_children(rec, v, r, K, L);
        return false;
    };
    if (r.c == 0) return finish(0);
    float muf;
    if (WR) {
        const uint64_t c = r.c;
        if (K == 0) return finish(0);
        const float pf = __ull2float_rn(K) * __frcp_rn(__ull2float_rn(r.S));
        muf = __ull2float_rn(c) * pf;
        q->fh = kHatD1f * sqrtf(muf * (1.0f - pf) + 0.5f) + kHatD2f;
        q->logrf = (2 * K == r.S) ? 0.0f : logf(pf / (1.0f - pf));
        q->M = (uint64_t)(((unsigned __int128)(c + 1) * K) / r.S);
        q->a = c;
    } else {
        uint64_t n = r.c, Kh = K;
        const uint64_t S = r.S;
        if (Kh == 0) return finish(0);
        if (Kh == S) return finish(n);
        if (n == S) return finish(Kh);
        q->n_in = n;
        q->flipK = Kh > S - Kh;
        if (q->flipK) Kh = S - Kh;
        q->flipN = n > S - n;
        if (q->flipN) n = S - n;
        const uint64_t a = n < Kh ? n : Kh;
        const uint64_t b = n < Kh ? Kh : n;
        const float rSf = __frcp_rn(__ull2float_rn(S));
        muf = (__ull2float_rn(a) * __ull2float_rn(b)) * rSf;
        const float varf = (muf * (__ull2float_rn(S - a) * rSf)) *
                           (__ull2float_rn(S - b) * __frcp_rn(__ull2float_rn(S - 1)));
        q->fh = kHatD1f * sqrtf(varf + 0.5f) + kHatD2f;
        q->M = (uint64_t)(((unsigned __int128)(a + 1) * (b + 1)) / (S + 2));
        q->a = a;
        q->b = b;
        q->Kp = Kh;
    }
    q->v = v;
    q->lo = r.lo;
    q->S = r.S;
    q->c = r.c;
    q->off = r.off;
    q->K = K;
    q->trial = 0;
    q->fresh = true;
    q->have64 = false;
    q->haveff = false;
    q->fa = muf + 0.5f;
    q->ftop = __ull2float_rn(q->a + 1);
    // inversion below a mean of 16 (the FP64 mean decides when the single
    // one is within its error of 16)
    bool inversion = muf < 15.99f;
    if (!inversion && muf <= 16.01f) {
        setup64<WR>(q, tab);
        inversion = q->mu < 16.0;
    }
    if (inversion) {
        uint64_t L = 0;
        const int rc = WR ? binomial_inversion(key, v, r.c, K, r.S, tab, L)
                          : hypergeometric_inversion(key, v, r.c, K, r.S, tab, L);
        if (rc != RS_OK) { set_status(status, rc); L = 0; }
        return finish(L);
    }
    if (eager64 && !q->have64) setup64<WR>(q, tab);
    return true;
}

// Processes nodes v0 .. v0+count-1 (one level) with the calling warp, G
// lanes per node (G a power of two, 1 to 32).  `logs` is this warp's
// scratch of 32 * kLogSlots doubles in shared memory.
template <bool WR>
RS_DEV void tree_batch_warp(NodeRec* __restrict__ rec, uint64_t v0, uint32_t count, Key2 key,
                            const double* __restrict__ tab, int* status, double* logs, uint32_t G = 1,
                            bool guard = true) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t r = lane & (G - 1);         // trial offset inside the group
    const uint32_t gbase = lane - r;           // the group's first lane
    const uint32_t gmask = G == 32 ? 0xFFFFFFFFu : ((1u << G) - 1u) << gbase;
    const float* tf = reinterpret_cast<const float*>(tab + kTabF);
    double* mine = logs + lane * kLogSlots;
    RouNode q;
    bool active = false;                       // the same in all lanes of a group
    uint32_t next = 0;   // batch cursor (warp-uniform)
    for (;;) {
        // refill free groups, in order, until none is free or the batch is used up
        for (;;) {
            const uint32_t freem = __ballot_sync(0xFFFFFFFFu, !active && r == 0);
            if (freem == 0 || next >= count) break;
            const uint32_t take = min((uint32_t)__popc(freem), count - next);
            const uint32_t rank = __popc(freem & ((1u << gbase) - 1u));
            if (!active && rank < take)
                active = node_setup<WR>(rec, v0 + next + rank, key, tab, status, &q, r == 0, !guard);
            next += take;
        }
        if (__ballot_sync(0xFFFFFFFFu, active) == 0) break;
        // one trial per active lane: uniforms, candidate, the guard, and for
        // the trials it leaves open the logarithm arguments
        const uint64_t t = (uint64_t)q.trial + r;   // this lane's trial
        uint64_t k = 0;
        bool inr = false;
        int dec = 0;
        bool fresh_now = false;                    // this round takes the node's fixed-end logarithms
        int nargs = 0;
        constexpr int kTerms = WR ? 2 : 4;
        if (active) {
            const uint4 blk = philox_block((uint32_t)t, TAG_SPLIT, q.v, key);
            const uint64_t ux = ((uint64_t)blk.y << 32) | blk.x;
            const uint64_t vx = ((uint64_t)blk.w << 32) | blk.z;
            const float Uf = u_open_f(ux);
            int xd = guard ? guard_abscissa(q.fa, q.fh, q.ftop, Uf, v_closed_f(vx), &k) : 0;
            if (guard && xd == 0) {   // the second guard
                if (!q.haveff) setupff<WR>(&q, tab);
                xd = ff_guard_abscissa(q.ffa, q.ffh, q.a + 1, ux, vx, &k);
            }
            if (xd == 0) {   // the abscissa in FP64, as defined
                if (!q.have64) setup64<WR>(&q, tab);
                const double U = u_open(ux), V = v_closed(vx);
                const double X = q.alpha + q.h * (V - 0.5) * drecip(U);
                xd = (X < 0.0 || X >= q.top) ? -1 : 1;
                if (xd > 0) k = (uint64_t)X;
            }
            inr = xd > 0 && t < c_caps.rou_trials;
            if (inr) {
                if (guard) {
                    float fm = 0.0f, ft = 0.0f;
#pragma unroll
                    for (int j = 0; j < kTerms; ++j) {
                        float m;
                        ft += fsd(fixed_end<WR>(q, j), moving_end<WR>(q, j, k), tf, &m);
                        fm += m;
                    }
                    if (WR) {
                        const float dk = (float)((int64_t)k - (int64_t)q.M);
                        const float rt = dk * q.logrf;
                        ft += rt;
                        fm += fabsf(rt) + fabsf(dk);
                    }
                    dec = guard_decide(Uf, ft, fm);
                    if (dec == 0) {   // the second guard: the same terms in float-float
                        if (!q.haveff) setupff<WR>(&q, tab);
                        FF t2{0.0f, 0.0f};
                        float m2 = 0.0f;
#pragma unroll
                        for (int j = 0; j < kTerms; ++j) {
                            float m;
                            t2 = ff_add(t2, ff_sd(fixed_end<WR>(q, j), moving_end<WR>(q, j, k), tab, &m));
                            m2 += m;
                        }
                        if (WR) {
                            const FF dk = k >= q.M ? ff_from_u64(k - q.M) : ff_neg(ff_from_u64(q.M - k));
                            const FF rt = ff_mul(dk, q.fflogr);
                            t2 = ff_add(t2, rt);
                            m2 += fabsf(rt.hi) + fabsf(dk.hi);
                        }
                        dec = ff_guard_decide(ux, t2, m2, tab);
                    }
                }
                if (dec == 0) {
                    if (WR && !q.have64) setup64<WR>(&q, tab);   // ln(p / (1 - p)) as defined
                    LfdArgs A{mine, 0, 0};
                    if (q.fresh) {   // the fixed ends' logarithms go with this round's
                        fresh_now = true;
#pragma unroll
                        for (int j = 0; j < kTerms; ++j) {
                            const uint64_t P = fixed_end<WR>(q, j);
                            A.push((double)(P > 0 ? P : 1));
                        }
                    }
                    A.push(u_open(ux));
#pragma unroll
                    for (int j = 0; j < kTerms; ++j) sdf_args(fixed_end<WR>(q, j), moving_end<WR>(q, j, k), A);
                    nargs = A.n;
                }
            }
        }
        __syncwarp();
        // the warp evaluates all logarithms together: item g of the
        // concatenated per-lane lists goes to lane g mod 32; its owner is the
        // first lane whose inclusive prefix exceeds g
        uint32_t incl = (uint32_t)nargs;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= (uint32_t)o) incl += y;
        }
        const uint32_t excl = incl - (uint32_t)nargs;
        const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
        // four items per lane at a time so that their dependent chains overlap
        for (uint32_t base = 0; base < total; base += 128) {
            double* slot[4];
            double x[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t g = base + 32 * j + lane;
                uint32_t pos = 0;
#pragma unroll
                for (uint32_t step = 16; step >= 1; step >>= 1) {
                    const uint32_t v = __shfl_sync(0xFFFFFFFFu, incl, pos + step - 1);
                    if (v <= g) pos += step;
                }
                const uint32_t owner_excl = __shfl_sync(0xFFFFFFFFu, excl, pos);
                slot[j] = (g < total) ? logs + pos * kLogSlots + (g - owner_excl) : nullptr;
                x[j] = slot[j] ? *slot[j] : 1.0;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) x[j] = dlog(x[j], tab);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (slot[j]) *slot[j] = x[j];
        }
        __syncwarp();
        bool acc = dec > 0;
        uint64_t L = 0;
        LfdLogs Lg{mine, 0, 0};
        if (fresh_now) {
#pragma unroll
            for (int j = 0; j < kTerms; ++j) q.lnP[j] = Lg.next();
            q.fresh = false;
        }
        if (active && inr && dec == 0) {
            const double lU = Lg.next();
            double T;
            if (WR) {
                T = sdf_eval(q.M, k, q.lnP[0], tab, Lg) + sdf_eval(q.a - q.M, q.a - k, q.lnP[1], tab, Lg) +
                    (double)((int64_t)k - (int64_t)q.M) * q.logr;
            } else {
                const uint64_t m = q.S - q.a - q.b;
                T = sdf_eval(q.M, k, q.lnP[0], tab, Lg) + sdf_eval(q.a - q.M, q.a - k, q.lnP[1], tab, Lg) +
                    sdf_eval(q.b - q.M, q.b - k, q.lnP[2], tab, Lg) + sdf_eval(m + q.M, m + k, q.lnP[3], tab, Lg);
            }
            acc = 2.0 * lU <= T;
        }
        if (acc) {
            L = k;
            if (!WR) {
                if (q.flipN) L = q.Kp - L;
                if (q.flipK) L = q.n_in - L;
            }
        }
        // the group takes its lowest accepted trial
        const uint32_t accm = __ballot_sync(0xFFFFFFFFu, acc) & gmask;
        const uint64_t Lsel = __shfl_sync(0xFFFFFFFFu, L, accm ? __ffs(accm) - 1 : lane);
        if (active) {
            bool done = false;
            uint64_t Lout = 0;
            if (accm) {
                done = true;
                Lout = Lsel;
            } else {
                q.trial += G;
                if (q.trial >= c_caps.rou_trials) {
                    if (r == 0) set_status(status, RS_EITER);
                    done = true;
                }
            }
            if (done) {
                if (r == 0) write_children(rec, q.v, NodeRec{q.lo, q.S, q.c, q.off}, q.K, Lout);
                active = false;
            }
        }
        __syncwarp();
    }
}

// Nodes v0 .. v0+count-1 with G lanes per node, G a multiple of 4: lane
// 4p + j of a node's group evaluates term j of trial t + p (terms: the four
// differences of ln x! of the hypergeometric test, or the two of the
// binomial one).  All lanes compute ln U; the four lanes of a trial exchange
// their terms and reach the same decision.  The warp's 32 / G groups take the
// nodes in order and a group whose node is done takes the next one, so that
// the trial counts of a few nodes do not idle the rest of the warp.
template <bool WR>
RS_DEV void tree_terms_warp(NodeRec* __restrict__ rec, uint64_t v0, uint32_t count, Key2 key,
                            const double* __restrict__ tab, int* status, uint32_t G, bool guard = true) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t r = lane & (G - 1);
    const uint32_t gbase = lane - r;
    const uint32_t gmask = G == 32 ? 0xFFFFFFFFu : ((1u << G) - 1u) << gbase;
    const uint32_t p = r >> 2, j = r & 3u, tbase = lane & ~3u;
    const float* tf = reinterpret_cast<const float*>(tab + kTabF);
    RouNode q;
    bool active = false;   // the same in all lanes of a group
    uint32_t next = 0;     // batch cursor (warp-uniform)
    uint64_t P = 0;        // this lane's fixed end (term j); its logarithm once the node first needs FP64
    double lnP = 0.0;
    bool haveLnP = false;
    // exact mode: the FP64 set-up and logarithms at once; few nodes per
    // launch (the top of the tree, whose huge terms the first guard cannot
    // settle): the second guard's float-float set-up at once, FP64 only for
    // the trials both guards leave open
    const bool eager = !guard;
    const bool eager_ff = guard && G >= 16;
    for (;;) {
        // free groups take the next nodes, in order
        for (;;) {
            const uint32_t freem = __ballot_sync(0xFFFFFFFFu, !active && r == 0);
            if (freem == 0 || next >= count) break;
            const uint32_t take = min((uint32_t)__popc(freem), count - next);
            const uint32_t rank = __popc(freem & ((1u << gbase) - 1u));
            if (!active && rank < take) {
                active = node_setup<WR>(rec, v0 + next + rank, key, tab, status, &q, r == 0, eager);
                if (active) {
                    P = fixed_end<WR>(q, (int)j);
                    haveLnP = eager;
                    if (eager) lnP = log_fixed(P, tab);
                    if (eager_ff) setupff<WR>(&q, tab);
                }
            }
            next += take;
        }
        if (__ballot_sync(0xFFFFFFFFu, active) == 0) break;
        const uint64_t t = (uint64_t)q.trial + p;
        uint64_t ux = 0, k = 0, Q = P;   // ux: the value of U
        float Uf = 1.0f;
        int xd = 0;   // 1: X in [0, top), k = floor(X); -1: rejected; 0: not settled
        if (active) {
            const uint4 blk = philox_block((uint32_t)t, TAG_SPLIT, q.v, key);
            ux = ((uint64_t)blk.y << 32) | blk.x;
            const uint64_t vx = ((uint64_t)blk.w << 32) | blk.z;
            Uf = u_open_f(ux);
            if (guard) {
                xd = guard_abscissa(q.fa, q.fh, q.ftop, Uf, v_closed_f(vx), &k);
                if (xd == 0) {   // the second guard
                    if (!q.haveff) setupff<WR>(&q, tab);
                    xd = ff_guard_abscissa(q.ffa, q.ffh, q.a + 1, ux, vx, &k);
                }
            }
            if (xd == 0) {   // the abscissa in FP64, as defined
                if (!q.have64) setup64<WR>(&q, tab);
                const double U = u_open(ux), V = v_closed(vx);
                const double X = q.alpha + q.h * (V - 0.5) * drecip(U);
                xd = (X < 0.0 || X >= q.top) ? -1 : 1;
                if (xd > 0) k = (uint64_t)X;
            }
        }
        const bool inr = active && xd > 0 && t < c_caps.rou_trials;
        // this lane's difference ln P! - ln Q! (none: Q = P gives 0)
        if (active) Q = inr ? moving_end<WR>(q, (int)j, k) : P;
        // the guard: the trial's four lanes sum their single-precision terms
        int dec = 0;
        if (guard) {
            float fm;
            float ft = fsd(P, Q, tf, &fm);
            ft += __shfl_xor_sync(0xFFFFFFFFu, ft, 1);
            fm += __shfl_xor_sync(0xFFFFFFFFu, fm, 1);
            ft += __shfl_xor_sync(0xFFFFFFFFu, ft, 2);
            fm += __shfl_xor_sync(0xFFFFFFFFu, fm, 2);
            if (WR && active && inr) {
                const float dk = (float)((int64_t)k - (int64_t)q.M);
                const float rt = dk * q.logrf;
                ft += rt;
                fm += fabsf(rt) + fabsf(dk);
            }
            if (active && inr) dec = guard_decide(Uf, ft, fm);
        }
        // the second guard for the trials the first left open: the same sum
        // of the four lanes' terms in float-float
        if (guard && __any_sync(0xFFFFFFFFu, active && inr && dec == 0)) {
            const bool want = active && inr && dec == 0;   // the same in a trial's four lanes
            if (want && !q.haveff) setupff<WR>(&q, tab);
            float m2;
            FF t2 = ff_sd(P, want ? Q : P, tab, &m2);
#pragma unroll
            for (int o = 1; o <= 2; o <<= 1) {
                const FF y{__shfl_xor_sync(0xFFFFFFFFu, t2.hi, o), __shfl_xor_sync(0xFFFFFFFFu, t2.lo, o)};
                t2 = ff_add(t2, y);
                m2 += __shfl_xor_sync(0xFFFFFFFFu, m2, o);
            }
            if (WR && want) {
                const FF dk = k >= q.M ? ff_from_u64(k - q.M) : ff_neg(ff_from_u64(q.M - k));
                const FF rt = ff_mul(dk, q.fflogr);
                t2 = ff_add(t2, rt);
                m2 += fabsf(rt.hi) + fabsf(dk.hi);
            }
            if (want) dec = ff_guard_decide(ux, t2, m2, tab);
        }
        // FP64, as the definition states, for the trials both guards left open
        const bool need = active && inr && dec == 0;
        bool acc = dec > 0;
        if (__any_sync(0xFFFFFFFFu, need)) {
            if (need && !haveLnP) {
                lnP = log_fixed(P, tab);
                haveLnP = true;
            }
            if (WR && need && !q.have64) setup64<WR>(&q, tab);   // ln(p / (1 - p)) as defined
            // the ends are picked with selects so that all lanes run one copy
            const double term = dsd_fixed(P, need ? Q : P, lnP, tab);
            const double lU = dlog(u_open(ux), tab);
            const double t0 = __shfl_sync(0xFFFFFFFFu, term, tbase);
            const double t1 = __shfl_sync(0xFFFFFFFFu, term, tbase + 1);
            const double t2 = __shfl_sync(0xFFFFFFFFu, term, tbase + 2);
            const double t3 = __shfl_sync(0xFFFFFFFFu, term, tbase + 3);
            if (need) {
                double T;
                if (WR) T = t0 + t1 + (double)((int64_t)k - (int64_t)q.M) * q.logr;
                else T = t0 + t1 + t2 + t3;
                acc = 2.0 * lU <= T;
            }
        }
        uint64_t L = 0;
        if (acc) {
            L = k;
            if (!WR) {
                if (q.flipN) L = q.Kp - L;
                if (q.flipK) L = q.n_in - L;
            }
        }
        // the group takes its lowest accepted trial
        const uint32_t accm = __ballot_sync(0xFFFFFFFFu, acc) & gmask;
        const uint64_t Lsel = __shfl_sync(0xFFFFFFFFu, L, accm ? __ffs(accm) - 1 : lane);
        if (active) {
            bool done = false;
            uint64_t Lout = 0;
            if (accm) {
                done = true;
                Lout = Lsel;
            } else {
                q.trial += G / 4;
                if (q.trial >= c_caps.rou_trials) {
                    if (r == 0) set_status(status, RS_EITER);
                    done = true;
                }
            }
            if (done) {
                if (r == 0) write_children(rec, q.v, NodeRec{q.lo, q.S, q.c, q.off}, q.K, Lout);
                active = false;
            }
        }
        __syncwarp();
    }
}

}  // namespace rs
