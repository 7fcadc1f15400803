// rs_hash_leaf.cuh -- leaf H and leaf WR with MSB-addressed tables.
//
// Algorithm H (Sec. 2) keeps the sample in a hash table addressed by the
// most significant bits of the key; since the keys are random that address
// is a good hash, and since it is monotone in the key the table reads out in
// sorted order once the keys that share an address are put in order
// (Sec. 4.1).  One thread block owns one leaf at a time and keeps the table
// in shared memory.  The leaf's values are the first k distinct valid
// candidates of its stream (k = n', or s - n' for a complement leaf, where
// more than half the leaf is taken: Sec. 2's n > N/2 rule applied per leaf).
//
// Three ways to compute them, all with the same result:
//
//  bucket path (the common case): candidates [0, k) are generated once,
//    kept in shared memory and counted per bucket (about 3/4 of a key per bucket
//    on average, addressed by the top bits; 16-bit counts, no size limit).
//    A scan of the counts gives every bucket its output offset; a second
//    pass scatters the keys into bucket order; each key then finds its rank
//    inside its bucket (four unrolled comparisons, a loop beyond), which is
//    its output position, and is written there.  Equal keys share a rank and
//    so lower the sum of the ranks: a second run then breaks the ties by
//    position.  When the leaf size does not divide 2^32 (2^64)
//    some candidates are void: each leaves a hole among candidates [0, k),
//    and later rounds of exactly as many further candidates as holes
//    remain fill them, so that exactly the first k valid ones are kept.
//    Launches whose leaves are all one power-of-two size compile this out.
//    If
//    a key repeats (without replacement), the distinct values are kept and
//    one warp draws the missing ones from the following candidates, each
//    tested against the set (binary search) and against its batch, so that
//    the set is still the first k distinct valid candidates; the two sorted
//    lists are then merged into the output.
//  bitmap path (complement leaves, and selections dense in a small range):
//    an atomic OR sets bit v and tells whether it was already set; the
//    read-out walks the bits in order.
//  probing path (fallback): linear probing with compare-and-swap in rounds.
//    Round 1 inserts candidates [0, k); each later round inserts exactly as
//    many further candidates as values are still missing, so the set after
//    the last round is the first k distinct valid candidates whatever the
//    order of concurrent inserts.  The read-out ranks each key inside its
//    cluster of occupied slots (a key's home slot lies inside its cluster and
//    homes are monotone in the key, so clusters come out in key order).
//
// For sampling with replacement (Sec. 4.6) duplicates are kept: the bucket
// path only needs valid candidates, and the probing path orders equal keys
// by slot.
#pragma once
#include <type_traits>

#include "rs_block.cuh"
#include "rs_internal.h"
#include "rs_rng.cuh"

namespace rs {

// The paths other than the bucket path's first run are compiled as calls of
// their own, so that their registers do not weigh on the common case.
#define RS_COLD __device__ __noinline__

constexpr uint32_t kHashCap = kLeafFastCap;         // largest selection of the shared-memory paths
constexpr uint32_t kHashSlack = 64;                 // probing: slots past the end instead of wrap-around

template <typename KeyT>
struct HashEmpty;
template <>
struct HashEmpty<uint32_t> { static constexpr uint32_t v = 0xFFFFFFFFu; };
template <>
struct HashEmpty<uint64_t> { static constexpr uint64_t v = ~0ull; };

// Shared memory of one leaf group: CAP is the largest selection of the
// shared-memory paths (the table holds 2 CAP + slack keys).
template <typename KeyT, int NW, uint32_t CAP = kHashCap>
struct HashShared {
    static constexpr uint32_t kCap = CAP;
    static constexpr uint32_t kSlots = 2 * CAP + kHashSlack;
    static constexpr uint32_t kBits = 32 * kSlots;        // largest leaf range of the bitmap path
    static constexpr uint32_t kBuckets = CAP + 64;        // bucket path: at most this many buckets
    KeyT tab[kSlots];              // bucket path: keys (first k + 3), then keys in bucket order;
                                   // probing table; bitmap; tallies
    alignas(16) uint32_t cnt[kBuckets / 2 + 5];   // bucket path: word 3 is zero; from word 4 on, 16-bit
                                                  // counts, two per word, then offsets
    uint32_t scan_tmp[NW + 1];
    uint32_t warp_cnt[NW];
    uint32_t newcount[3];          // rounds: values added in round r go to newcount[r % 3]
    uint32_t topcount;             // probing, 32-bit keys: copies of 2^32-1 (it equals the empty mark)
    uint32_t overflow;             // probing ran past the slack
    uint64_t jnext;                // bucket path: index of the candidate after the k-th valid one
    uint32_t nadded;               // bucket path: values drawn after a repeat
    uint32_t fill;                 // bucket path, leaves with void candidates: holes left by round 1
    uint32_t fill2;                //   and holes filled by the later rounds
    uint32_t repair_fail;
    uint32_t ranksum;              // bucket path: sum of the keys' ranks (k (k - 1) / 2 without ties)
    uint64_t thr;                  // Lemire rejection threshold of the leaf
    uint64_t mult;                 // address multiplier of the current table
};

// Lemire rejection threshold for a leaf of size s: (2^32 - s) mod s for
// 32-bit candidates (a 32-bit remainder), (2^64 - s) mod s for 64-bit ones.
RS_DEV uint64_t lemire_threshold(uint64_t s) {
    if (s == (1ull << 32)) return 0;
    if (s < (1ull << 32)) {
        const uint32_t s32 = (uint32_t)s;
        return (0u - s32) % s32;
    }
    return (0ull - s) % s;
}

// Barrier over the NT threads of a leaf group (named barrier `ID`).
template <int ID, int NT>
RS_DEV void group_sync() {
    if (ID == 0) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"n"(ID), "n"(NT) : "memory");
}

template <int ID, int NT>
RS_DEV bool group_sync_or(bool p) {
    if (ID == 0) return __syncthreads_or(p) != 0;
    uint32_t r;
    asm volatile("{ .reg .pred a, b; setp.ne.u32 a, %1, 0; bar.red.or.pred b, %2, %3, a; selp.u32 %0, 1, 0, b; }"
                 : "=r"(r) : "r"((uint32_t)p), "n"(ID), "n"(NT) : "memory");
    return r != 0;
}

RS_DEV uint32_t hash_slot(uint32_t v, uint64_t mult) { return __umulhi(v, (uint32_t)mult); }
RS_DEV uint32_t hash_slot(uint64_t v, uint64_t mult) { return (uint32_t)__umul64hi(v, mult); }

// Multiplier of the monotone address map v -> floor(v * mult / 2^width),
// which sends [0, s) into [0, T).
template <typename KeyT>
RS_DEV uint64_t slot_mult(uint64_t s, uint32_t T) {
    if (sizeof(KeyT) == 4) {
        const uint64_t m = ((uint64_t)T << 32) / s;
        return m > 0xFFFFFFFFull ? 0xFFFFFFFFull : m;
    }
    return (uint64_t)T >= s ? ~0ull : (uint64_t)(((unsigned __int128)T << 64) / s);
}

// A multiplier of the same kind computed in single precision, each step
// rounded down, so that mult <= T 2^width / s and every slot stays below T.  Any such multiplier keeps the order of the
// values, which is all the bucket path relies on.
template <typename KeyT>
RS_DEV uint64_t slot_mult_fast(uint64_t s, uint32_t T) {
    const float q = __fdiv_rd((float)T, __ull2float_ru(s));   // <= T / s
    if (sizeof(KeyT) == 4) {
        const float m = __fmul_rd(q, 4294967296.0f);
        return m >= 4294967295.0f ? 0xFFFFFFFFull : (uint64_t)__float2uint_rd(m);
    }
    const float m = __fmul_rd(q, 18446744073709551616.0f);
    return m >= 18446744073709551615.0f ? ~0ull : __float2ull_rd(m);
}

RS_DEV uint32_t cas_key(uint32_t* p, uint32_t cmp, uint32_t val) { return atomicCAS(p, cmp, val); }
RS_DEV uint64_t cas_key(uint64_t* p, uint64_t cmp, uint64_t val) {
    return (uint64_t)atomicCAS((unsigned long long*)p, (unsigned long long)cmp, (unsigned long long)val);
}

struct LeafRec {
    uint64_t lo, s, np, off, id;
};

// Walks the candidates [J, J+m) of the leaf's stream; calls f(rel, v) for
// each valid one (rel = its index - J) and sets *void_seen if one was void.
// 32-bit words when s <= 2^32, 64-bit values otherwise.
template <int NT, typename F>
RS_DEV void for_candidates(const LeafRec& r, uint64_t thr64, Key2 key, uint32_t tag, uint64_t J, uint32_t m,
                           uint32_t tid, bool* void_seen, F&& f) {
    // Block and candidate indices stay below 2^32 and 2^34 (callers stop a
    // round earlier), so the block index is 32-bit; offsets are relative to J.
    if (r.s <= (1ull << 32)) {
        const uint32_t thr = (uint32_t)thr64;
        const uint32_t s32 = (uint32_t)(r.s - 1);   // s - 1 fits 32 bits; s = (s - 1) + 1
        const uint32_t b0 = (uint32_t)(J >> 2);
        const uint32_t nblk = (uint32_t)(((J + m - 1) >> 2) - (J >> 2) + 1);
        const uint32_t skip = (uint32_t)(J & 3);   // candidates of the first block before J
        auto use = [&](uint32_t w, uint32_t rel) {
            if (rel >= m) return;
            // w * s = w * (s - 1) + w, exact in 64 bits
            const uint64_t prod = (uint64_t)w * s32 + w;
            if ((uint32_t)prod < thr) {
                *void_seen = true;
                return;
            }
            f(rel, (uint64_t)(prod >> 32));
        };
        for (uint32_t i = tid; i < nblk; i += 2 * NT) {
            const uint32_t i2 = i + NT;
            const uint4 w = philox_block(b0 + i, tag, r.id, key);
            uint4 w2 = make_uint4(0, 0, 0, 0);
            if (i2 < nblk) w2 = philox_block(b0 + i2, tag, r.id, key);
            const uint32_t base = 4 * i - skip, base2 = 4 * i2 - skip;   // relative index of word 0 (mod 2^32)
            if (i > 0 || skip == 0) use(w.x, base);
            if (i > 0 || skip <= 1) use(w.y, base + 1);
            if (i > 0 || skip <= 2) use(w.z, base + 2);
            use(w.w, base + 3);
            if (i2 < nblk) {
                use(w2.x, base2);
                use(w2.y, base2 + 1);
                use(w2.z, base2 + 2);
                use(w2.w, base2 + 3);
            }
        }
    } else {
        const uint64_t thr = thr64;
        const uint32_t b0 = (uint32_t)(J >> 1);
        const uint32_t nblk = (uint32_t)(((J + m - 1) >> 1) - (J >> 1) + 1);
        const uint32_t skip = (uint32_t)(J & 1);
        for (uint32_t i = tid; i < nblk; i += NT) {
            const uint4 w = philox_block(b0 + i, tag, r.id, key);
            const uint64_t xs[2] = {((uint64_t)w.y << 32) | w.x, ((uint64_t)w.w << 32) | w.z};
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                if (i == 0 && (uint32_t)c < skip) continue;
                const uint32_t rel = 2 * i + c - skip;
                if (rel >= m) continue;
                if (xs[c] * r.s < thr) {
                    *void_seen = true;
                    continue;
                }
                f(rel, __umul64hi(xs[c], r.s));
            }
        }
    }
}

// Exclusive prefix sums, in place, of the nb 16-bit counts packed two per
// word in w[0 .. nb/2), nb a multiple of 64 and at most 24 NT, w 16-byte
// aligned.  Thread t owns Q consecutive 16-byte groups (8 counts each), Q = 1
// or 3 (odd, so that the 16-byte accesses of a quarter warp fall in distinct
// banks), kept in registers between the two halves.  Two barriers: warp
// totals go to tmp[], then each warp adds up those of the warps before it.
template <int NT>
RS_DEV void scan_counts16(uint32_t* w, uint32_t nb, uint32_t* tmp, uint32_t tid) {
    uint4* g = reinterpret_cast<uint4*>(w);
    const uint32_t groups = nb >> 3;
    const uint32_t Q = groups > NT ? 3u : 1u;
    const uint32_t g0 = tid * Q;
    auto sum2 = [](uint32_t x) { return (x & 0xFFFFu) + (x >> 16); };
    uint4 x[3];
    uint32_t local = 0;
#pragma unroll
    for (uint32_t q = 0; q < 3; ++q) {
        x[q] = make_uint4(0, 0, 0, 0);
        if (q < Q && g0 + q < groups) x[q] = g[g0 + q];
        local += (sum2(x[q].x) + sum2(x[q].y)) + (sum2(x[q].z) + sum2(x[q].w));
    }
    const uint32_t lane = tid & 31, warp = tid >> 5;
    uint32_t incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= (uint32_t)o) incl += y;
    }
    if (lane == 31) tmp[warp] = incl;
    __syncthreads();
    uint32_t run = incl - local + __reduce_add_sync(0xFFFFFFFFu, lane < warp ? tmp[lane] : 0u);
    auto put = [&](uint32_t v) {   // the two counts of a word -> their first positions
        const uint32_t lo = run, hi = run + (v & 0xFFFFu);
        run = hi + (v >> 16);
        return lo | (hi << 16);
    };
#pragma unroll
    for (uint32_t q = 0; q < 3; ++q) {
        if (q < Q && g0 + q < groups) {
            uint4 y;
            y.x = put(x[q].x);
            y.y = put(x[q].y);
            y.z = put(x[q].z);
            y.w = put(x[q].w);
            g[g0 + q] = y;
        }
    }
    __syncthreads();
}

// Candidate j of the leaf's stream (the same definition as for_candidates):
// false if it is void.
RS_DEV bool candidate_at(const LeafRec& r, uint64_t thr, Key2 key, uint32_t tag, uint64_t j, uint64_t* v) {
    if (r.s <= (1ull << 32)) {
        const uint4 w = philox_block((uint32_t)(j >> 2), tag, r.id, key);
        const uint32_t c = (uint32_t)(j & 3);
        const uint32_t x = c == 0 ? w.x : (c == 1 ? w.y : (c == 2 ? w.z : w.w));
        const uint64_t prod = (uint64_t)x * (uint32_t)(r.s - 1) + x;
        if ((uint32_t)prod < (uint32_t)thr) return false;
        *v = prod >> 32;
        return true;
    }
    const uint4 w = philox_block((uint32_t)(j >> 1), tag, r.id, key);
    const uint64_t x = (j & 1) ? (((uint64_t)w.w << 32) | w.z) : (((uint64_t)w.y << 32) | w.x);
    if (x * r.s < thr) return false;
    *v = __umul64hi(x, r.s);
    return true;
}

// Bucket path, leaves whose first k valid candidates repeat a value: A[0..k)
// holds them sorted.  Keeps the d distinct values (B), draws the k - d
// missing ones from candidates jnext, jnext+1, ... (a candidate counts if it
// is valid and new), and writes the merged sorted leaf.  False if the stream
// runs out (the probing path then reports it).
template <typename KeyT, int NT, int BAR, uint32_t CAP>
RS_COLD bool bucket_repair(HashShared<KeyT, NT / 32, CAP>& sm, const LeafRec& r, Key2 key, uint32_t k, uint64_t thr,
                          KeyT* A, KeyT* B, uint64_t* __restrict__ dst, uint32_t tid) {
    // distinct values of the sorted A, in order, into B
    const uint32_t Q = (k + NT - 1) / NT;
    const uint32_t i0 = min(tid * Q, k), i1 = min(i0 + Q, k);
    uint32_t local = 0;
    for (uint32_t i = i0; i < i1; ++i) local += (i == 0 || A[i] != A[i - 1]) ? 1u : 0u;
    uint32_t d;
    uint32_t pos = block_exclusive_scan<NT>(local, sm.scan_tmp, &d);
    for (uint32_t i = i0; i < i1; ++i)
        if (i == 0 || A[i] != A[i - 1]) B[pos++] = A[i];
    if (tid == 0) sm.repair_fail = 0;
    group_sync<BAR, NT>();
    // one warp draws the missing values, 32 candidates at a time, in index order
    KeyT* NV = A;   // the new values (at most k - d)
    const uint32_t need = k - d;
    if (tid < 32) {
        const uint32_t lane = tid;
        const uint64_t jlimit = (r.s > (1ull << 32) ? 2 : 4) * c_caps.stream_blocks;
        uint64_t J = sm.jnext;
        uint32_t added = 0;
        while (added < need) {
            if (J + 32 > jlimit) {
                if (lane == 0) sm.repair_fail = 1;
                break;
            }
            uint64_t v64 = 0;
            bool fresh = candidate_at(r, thr, key, TAG_LEAF_H, J + lane, &v64);
            const KeyT v = (KeyT)v64;
            if (fresh) {   // already in the set?
                uint32_t lo = 0, hi = d;
                while (lo < hi) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (B[mid] < v) lo = mid + 1; else hi = mid;
                }
                if (lo < d && B[lo] == v) fresh = false;
                for (uint32_t t = 0; t < added && fresh; ++t)
                    if (NV[t] == v) fresh = false;
            }
            // an earlier lane of this batch drew the same value
            const uint32_t same = __match_any_sync(0xFFFFFFFFu, (unsigned long long)v64) &
                                  __ballot_sync(0xFFFFFFFFu, fresh);
            if (fresh && (uint32_t)(__ffs(same) - 1) != lane) fresh = false;
            const uint32_t keepm = __ballot_sync(0xFFFFFFFFu, fresh);
            const uint32_t take = min((uint32_t)__popc(keepm), need - added);
            const uint32_t rank = __popc(keepm & ((1u << lane) - 1u));
            if (fresh && rank < take) NV[added + rank] = v;
            added += take;
            J += 32;
            __syncwarp();
        }
    }
    group_sync<BAR, NT>();
    if (sm.repair_fail) return false;
    // sort the new values (distinct) by counting, into the free end of B
    KeyT* NS = B + d;
    for (uint32_t t = tid; t < need; t += NT) {
        const KeyT v = NV[t];
        uint32_t rank = 0;
        for (uint32_t u = 0; u < need; ++u) rank += NV[u] < v ? 1u : 0u;
        NS[rank] = v;
    }
    group_sync<BAR, NT>();
    // merge: each value's place is its index plus the number of values of the
    // other list below it
    const uint64_t base = r.lo + 1;
    for (uint32_t i = tid; i < d; i += NT) {
        const KeyT v = B[i];
        uint32_t lo = 0, hi = need;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (NS[mid] < v) lo = mid + 1; else hi = mid;
        }
        dst[i + lo] = base + v;
    }
    for (uint32_t t = tid; t < need; t += NT) {
        const KeyT v = NS[t];
        uint32_t lo = 0, hi = d;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (B[mid] < v) lo = mid + 1; else hi = mid;
        }
        dst[t + lo] = base + v;
    }
    group_sync<BAR, NT>();
    return true;
}

// Pass 3 of the bucket path over B (keys in bucket order, B[k .. k+3) the
// largest key value) with bucket ends ch[] (ch[-1] = 0): each key's rank
// among its bucket's keys is its place in the sorted leaf.  Without TIES the
// rank counts the smaller keys only, and the key goes to dst[rank]; with
// TIES equal keys are ordered by position in B, and the key goes to
// dst[rank] (with replacement) or A[rank] (without, for the repair).
// Returns the thread's sum of ranks.
template <typename KeyT, int NT, bool TIES, bool WR>
RS_DEV uint32_t rank_keys(const KeyT* B, KeyT* A, const uint16_t* ch, uint32_t k, uint64_t mult, uint64_t base,
                          uint64_t* __restrict__ dst, uint32_t tid) {
    constexpr uint32_t U = 4;   // keys per thread at a time, so that their load chains overlap
    uint32_t rsum = 0;
    // (key, position) order; 32-bit keys compare as one 64-bit value
    auto before = [](KeyT y, uint32_t j, KeyT x, uint32_t i) {
        if (sizeof(KeyT) == 4) return (((uint64_t)y << 32) | j) < (((uint64_t)x << 32) | i);
        return (y < x) || (y == x && j < i);
    };
    // `full` tiles need no bounds tests
    auto tile = [&](uint32_t i0, auto full_tag) {
        constexpr bool full = decltype(full_tag)::value;
        KeyT x[U];
        uint32_t s0[U], s1[U], rank[U];
#pragma unroll
        for (uint32_t q = 0; q < U; ++q) {
            const uint32_t i = i0 + q * NT;
            const bool ok = full || i < k;
            x[q] = ok ? B[i] : KeyT(0);
            const uint32_t b = hash_slot(x[q], mult);
            s0[q] = ch[(int)b - 1];
            s1[q] = ok ? ch[b] : 0u;
            rank[q] = s0[q];
        }
        // a window of four from the bucket start, unrolled and without
        // branches: reads past the bucket meet only larger keys (buckets
        // are monotone in the key) or the padding
#pragma unroll
        for (uint32_t u = 0; u < 4; ++u) {
#pragma unroll
            for (uint32_t q = 0; q < U; ++q) {
                const uint32_t j = s0[q] + u;
                const KeyT y = B[j];
                if (!TIES) rank[q] += y < x[q] ? 1u : 0u;
                else rank[q] += before(y, j, x[q], i0 + q * NT) ? 1u : 0u;
            }
        }
        // buckets of more than four keys: one loop for the U keys, reads
        // past the leaf clamped to the padding
        uint32_t extra = 0;
#pragma unroll
        for (uint32_t q = 0; q < U; ++q) extra = max(extra, s1[q] - min(s1[q], s0[q] + 4));
        for (uint32_t e = 0; e < extra; ++e) {
#pragma unroll
            for (uint32_t q = 0; q < U; ++q) {
                const uint32_t j = min(s0[q] + 4 + e, k + 2);
                const KeyT y = B[j];
                if (!TIES) rank[q] += y < x[q] ? 1u : 0u;
                else rank[q] += before(y, j, x[q], i0 + q * NT) ? 1u : 0u;
            }
        }
#pragma unroll
        for (uint32_t q = 0; q < U; ++q)
            if (full || i0 + q * NT < k) {
                rsum += rank[q];
                if (!TIES || WR) dst[rank[q]] = base + x[q];
                else A[rank[q]] = x[q];
            }
    };
    uint32_t i0 = tid;
    for (; i0 + (U - 1) * NT < k; i0 += U * NT) tile(i0, std::true_type{});
    if (i0 < k) tile(i0, std::false_type{});
    return rsum;
}

// The bucket path's leaves with equal keys (after the first rank run): the
// tie-broken run rewrites the leaf (with replacement) or sorts the keys into
// A for the repair of repeats (without).
template <typename KeyT, int NT, int BAR, bool WR, uint32_t CAP>
RS_COLD bool bucket_ties(HashShared<KeyT, NT / 32, CAP>& sm, const LeafRec& r, Key2 key, uint32_t k, uint64_t thr,
                         uint64_t mult, uint64_t* __restrict__ dst, uint32_t tid) {
    KeyT* A = sm.tab;
    KeyT* B = sm.tab + ((k + 3) & ~3u);
    const uint16_t* ch = reinterpret_cast<const uint16_t*>(sm.cnt + 4);
    rank_keys<KeyT, NT, true, WR>(B, A, ch, k, mult, r.lo + 1, dst, tid);
    group_sync<BAR, NT>();
    if (WR) return true;
    return bucket_repair<KeyT, NT, BAR, CAP>(sm, r, key, k, thr, A, B, dst, tid);   // rewrites the whole leaf
}

// The later rounds of the void-candidate pass 1: fill the nh holes listed in
// B's room from candidates k, k + 1, ... (see void_leaf_pass1).
template <typename KeyT, int NT, int BAR, uint32_t CAP, typename K2>
__device__ __forceinline__ bool fill_holes(HashShared<KeyT, NT / 32, CAP>& sm, const LeafRec& r, const K2& key,
                                           uint32_t tag, uint32_t k, uint32_t nh, uint64_t thr, uint64_t mult, KeyT* A,
                                           KeyT* B, uint32_t* cw, uint32_t tid) {
    const bool w32 = r.s <= (1ull << 32);
    const uint32_t lg = w32 ? 2u : 1u;
    const uint64_t jcap = min((uint64_t)c_caps.stream_blocks, (uint64_t)1 << 32) << lg;
    const uint32_t* H = reinterpret_cast<const uint32_t*>(B);
    auto count = [&](KeyT v) {
        const uint32_t b = hash_slot(v, mult);
        atomicAdd(&cw[b >> 1], 1u << ((b & 1u) << 4));
    };
    // later rounds: fill the holes from candidates k, k + 1, ...
    const uint32_t lane = tid & 31;
    const uint32_t lt = (1u << lane) - 1u;
    uint64_t J = k;   // next candidate index
    uint32_t got = 0;
    while (got < nh) {   // the same in all threads
        if (J >= jcap) return false;
        const uint64_t jend = min(J + (uint64_t)(nh - got), jcap);
        const uint64_t bfirst = J >> lg;
        const uint32_t nbr = (uint32_t)(((jend - 1) >> lg) - bfirst + 1);
        for (uint32_t i0 = tid - lane; i0 < nbr; i0 += NT) {   // warp-uniform trips
            const uint32_t i = i0 + lane;
            const uint64_t blk = bfirst + i;
            KeyT v[4] = {0, 0, 0, 0};
            uint32_t ok = 0;   // bit c: candidate (blk << lg) + c is valid and in [J, jend)
            if (i < nbr) {
                const uint4 w = philox_block((uint32_t)blk, tag, r.id, key);
                if (w32) {
                    const uint32_t s32 = (uint32_t)(r.s - 1), thr32 = (uint32_t)thr;
                    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const uint64_t prod = (uint64_t)ws[c] * s32 + ws[c];
                        const uint64_t j = (blk << 2) + c;
                        v[c] = (KeyT)(prod >> 32);
                        ok |= ((uint32_t)prod >= thr32 && j >= J && j < jend ? 1u : 0u) << c;
                    }
                } else {
                    const uint64_t xs[2] = {((uint64_t)w.y << 32) | w.x, ((uint64_t)w.w << 32) | w.z};
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const uint64_t j = (blk << 1) + c;
                        v[c] = (KeyT)__umul64hi(xs[c], r.s);
                        ok |= (xs[c] * r.s >= thr && j >= J && j < jend ? 1u : 0u) << c;
                    }
                }
            }
            const uint32_t q0 = __ballot_sync(0xFFFFFFFFu, ok & 1u), q1 = __ballot_sync(0xFFFFFFFFu, ok & 2u);
            const uint32_t q2 = __ballot_sync(0xFFFFFFFFu, ok & 4u), q3 = __ballot_sync(0xFFFFFFFFu, ok & 8u);
            const uint32_t tot = __popc(q0) + __popc(q1) + __popc(q2) + __popc(q3);
            uint32_t base = 0;
            if (lane == 0 && tot) base = atomicAdd(&sm.fill2, tot);
            uint32_t pos = __shfl_sync(0xFFFFFFFFu, base, 0) + __popc(q0 & lt) + __popc(q1 & lt) +
                           __popc(q2 & lt) + __popc(q3 & lt);
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if ((ok >> c) & 1u) {
                    A[H[pos++]] = v[c];
                    count(v[c]);
                }
        }
        group_sync<BAR, NT>();
        const uint32_t now = sm.fill2;
        // every candidate of the last round was valid: the k-th is jend - 1
        if (now == nh && tid == 0) sm.jnext = jend;
        got = now;
        J = jend;
        if (got < nh) group_sync<BAR, NT>();   // every thread has read the count before the next round adds
    }
    return true;
}

template <typename KeyT, int NT, int BAR, uint32_t CAP, typename K2>
RS_COLD bool void_fill_holes(HashShared<KeyT, NT / 32, CAP>& sm, const LeafRec& r, const K2& key, uint32_t tag,
                             uint32_t k, uint32_t nh, uint64_t thr, uint64_t mult, KeyT* A, KeyT* B, uint32_t* cw,
                             uint32_t tid) {
    return fill_holes<KeyT, NT, BAR, CAP>(sm, r, key, tag, k, nh, thr, mult, A, B, cw, tid);
}

// Pass 1 of the bucket path for leaves with void candidates (sizes that are
// not powers of two): the first k valid candidates to A[0..k) (in no
// particular order: later passes only need the set), counted per bucket,
// sm.jnext set to the index after the k-th.  Round 1 runs as on the
// power-of-two path: candidate j of [0, k) goes to A[j] (16-byte stores),
// by Lemire's map (w s) >> width; a void one leaves a hole, listed in B's
// room (not yet in use).  Void candidates are rare unless the leaf size is
// just above a power of two (up to half of them), so most leaves end here.
// Later rounds fill the h holes: round r takes the next m_r candidates of
// the stream, m_r the holes still open, and puts every valid one into a
// hole; a round can never take more values than are missing, so after the
// last one A holds exactly the first k valid candidates, with no ordering
// or scan.  False if the stream runs out.
template <typename KeyT, int NT, int BAR, uint32_t CAP, typename K2>
RS_COLD bool void_leaf_pass1(HashShared<KeyT, NT / 32, CAP>& sm, const LeafRec& r, const K2& key, uint32_t tag,
                             uint32_t k, uint64_t thr, uint64_t mult, KeyT* A, KeyT* B, uint32_t* cw, uint32_t tid) {
    const bool w32 = r.s <= (1ull << 32);
    const uint32_t lg = w32 ? 2u : 1u;   // candidates per Philox block: 2^lg
    // candidates come from blocks below the stream's limit (and 2^32)
    const uint64_t jcap = min((uint64_t)c_caps.stream_blocks, (uint64_t)1 << 32) << lg;
    if (k > jcap) return false;   // the stream ran out: the probing path reports it
    uint32_t* H = reinterpret_cast<uint32_t*>(B);   // the holes (B holds k + 3 keys)
    auto count = [&](KeyT v) {
        const uint32_t b = hash_slot(v, mult);
        atomicAdd(&cw[b >> 1], 1u << ((b & 1u) << 4));
    };
    auto put = [&](uint32_t j, KeyT v, bool ok) {   // candidate j already in A[j]
        if (ok) count(v);
        else H[atomicAdd(&sm.fill, 1u)] = j;
    };
    // round 1: candidates [0, k)
    if (w32) {
        const uint32_t s32 = (uint32_t)(r.s - 1), thr32 = (uint32_t)thr;
        const uint32_t full = k >> 2;   // Philox blocks whose four words are all used
        for (uint32_t i = tid; i < full; i += NT) {
            const uint4 w = philox_block(i, tag, r.id, key);
            // w * s = w * (s - 1) + w, exact in 64 bits; valid when its low word >= thr
            const uint64_t p0 = (uint64_t)w.x * s32 + w.x, p1 = (uint64_t)w.y * s32 + w.y;
            const uint64_t p2 = (uint64_t)w.z * s32 + w.z, p3 = (uint64_t)w.w * s32 + w.w;
            const uint4 v = make_uint4((uint32_t)(p0 >> 32), (uint32_t)(p1 >> 32), (uint32_t)(p2 >> 32),
                                       (uint32_t)(p3 >> 32));
            if (sizeof(KeyT) == 4) {
                reinterpret_cast<uint4*>(A)[i] = v;   // one 16-byte store (A is 16-byte aligned)
            } else {
                A[4 * i] = v.x;
                A[4 * i + 1] = v.y;
                A[4 * i + 2] = v.z;
                A[4 * i + 3] = v.w;
            }
            put(4 * i, (KeyT)v.x, (uint32_t)p0 >= thr32);
            put(4 * i + 1, (KeyT)v.y, (uint32_t)p1 >= thr32);
            put(4 * i + 2, (KeyT)v.z, (uint32_t)p2 >= thr32);
            put(4 * i + 3, (KeyT)v.w, (uint32_t)p3 >= thr32);
        }
        if (tid == 0 && (k & 3u)) {
            const uint4 w = philox_block(full, tag, r.id, key);
            const uint32_t ws[3] = {w.x, w.y, w.z};
            for (uint32_t c = 0; c < (k & 3u); ++c) {
                const uint64_t p = (uint64_t)ws[c] * s32 + ws[c];
                A[4 * full + c] = (KeyT)(p >> 32);
                put(4 * full + c, (KeyT)(p >> 32), (uint32_t)p >= thr32);
            }
        }
    } else {
        const uint32_t full = k >> 1;
        for (uint32_t i = tid; i < full; i += NT) {
            const uint4 w = philox_block(i, tag, r.id, key);
            const uint64_t x0 = ((uint64_t)w.y << 32) | w.x, x1 = ((uint64_t)w.w << 32) | w.z;
            const KeyT v0 = (KeyT)__umul64hi(x0, r.s), v1 = (KeyT)__umul64hi(x1, r.s);
            A[2 * i] = v0;
            A[2 * i + 1] = v1;
            put(2 * i, v0, x0 * r.s >= thr);
            put(2 * i + 1, v1, x1 * r.s >= thr);
        }
        if (tid == 0 && (k & 1u)) {
            const uint4 w = philox_block(full, tag, r.id, key);
            const uint64_t x0 = ((uint64_t)w.y << 32) | w.x;
            const KeyT v0 = (KeyT)__umul64hi(x0, r.s);
            A[2 * full] = v0;
            put(2 * full, v0, x0 * r.s >= thr);
        }
    }
    group_sync<BAR, NT>();
    const uint32_t nh = sm.fill;   // the same in all threads
    if (nh == 0) {
        if (tid == 0) sm.jnext = k;
        return true;
    }
    return fill_holes<KeyT, NT, BAR, CAP>(sm, r, key, tag, k, nh, thr, mult, A, B, cw, tid);
}

// Bucket path.  Returns true on success (leaf written), false if the leaf
// must take the probing path (whatever was written is overwritten later).
// K2 is Key2 or RoundKeys (the same generator, round keys precomputed).
// POW2: the caller knows every leaf size to be a power of two, so the code
// for void candidates is left out (a leaf of another size then returns
// false and takes the probing path).  INL: with 32-bit words the first
// round of the void pass runs inline (faster for the single-call kernel;
// the batch's kernels are faster with the whole pass as one call).
template <typename KeyT, int NT, int BAR, bool WR, uint32_t CAP = kHashCap, typename K2 = Key2, bool POW2 = false,
          bool INL = false>
RS_DEV bool bucket_leaf(HashShared<KeyT, NT / 32, CAP>& sm, const LeafRec& r, const K2& key, uint32_t k,
                        uint64_t* __restrict__ dst, uint32_t tid) {
    static_assert(HashShared<KeyT, NT / 32, CAP>::kBuckets <= 24 * NT, "scan_counts16 takes at most 24 NT counts");
    const uint32_t tag = WR ? TAG_LEAF_WR : TAG_LEAF_H;
    // buckets: about 3/4 of a key each (measured best on GB300 among 7/8 to
    // 2 keys per bucket), a multiple of 64, at most kBuckets
    const uint32_t nb = min(HashShared<KeyT, NT / 32, CAP>::kBuckets, max(64u, (k * 4 / 3 + 63) & ~63u));
    KeyT* A = sm.tab;                     // candidate j at A[j]; later the sorted leaf
    KeyT* B = sm.tab + ((k + 3) & ~3u);   // keys in bucket order
    uint32_t* cw = sm.cnt + 4;            // count of bucket b: 16-bit half b & 1 of word b >> 1
    const uint16_t* ch = reinterpret_cast<const uint16_t*>(cw);   // ch[-1] = 0, the high half of cnt[3]
    for (uint32_t i = tid; i < nb / 8; i += NT) reinterpret_cast<uint4*>(cw)[i] = make_uint4(0, 0, 0, 0);
    if (tid == 0) sm.cnt[3] = 0;
    if (tid == 0) {   // once per leaf; the last reads of these fields came before the last barrier
        if ((r.s & (r.s - 1)) == 0) {
            // a power of two 2^t: the map v -> v nb 2^-t by a shift (no
            // division or conversion on the path to the barrier), no void
            // candidates
            const uint32_t t = 63u - (uint32_t)__clzll((long long)r.s);
            const uint32_t w = sizeof(KeyT) == 4 ? 32u : 64u;
            const uint64_t m = (uint64_t)nb << (w - t);
            sm.mult = (sizeof(KeyT) == 4 && m > 0xFFFFFFFFull) ? 0xFFFFFFFFull : m;
            sm.thr = 0;
        } else {
            sm.mult = slot_mult_fast<KeyT>(r.s, nb);
            sm.thr = lemire_threshold(r.s);
            sm.fill = 0;
            sm.fill2 = 0;
        }
    }
    group_sync<BAR, NT>();
    const uint64_t mult = sm.mult;
    const uint64_t thr = sm.thr;
    if (tid == 0) sm.ranksum = 0;   // every read of the last leaf's sum came before this barrier
    // pass 1: generate, keep, count per bucket
    auto keep = [&](uint32_t j, uint64_t v) {
        A[j] = (KeyT)v;
        const uint32_t b = hash_slot((KeyT)v, mult);
        atomicAdd(&cw[b >> 1], 1u << ((b & 1u) << 4));
    };
    if (POW2 && thr != 0) return false;   // not a power of two after all
    if (POW2 || thr == 0) {
        // No candidate can be void (the leaf size is a power of two 2^t, the
        // only sizes that divide 2^32 or 2^64): candidates [0, k) are the
        // first k valid ones and Lemire's map (w s) >> width is w >> (width - t).
        const uint32_t t = 63u - (uint32_t)__clzll(r.s);
        if (r.s <= (1ull << 32)) {
            const uint32_t sh = 32u - t;   // 0 when s = 2^32
            const uint32_t full = k >> 2;  // Philox blocks whose four words are all used
            auto count = [&](uint32_t v) {
                const uint32_t b = hash_slot((KeyT)v, mult);
                atomicAdd(&cw[b >> 1], 1u << ((b & 1u) << 4));
            };
            for (uint32_t i = tid; i < full; i += NT) {
                const uint4 w = philox_block(i, tag, r.id, key);
                const uint4 v = sh < 32 ? make_uint4(w.x >> sh, w.y >> sh, w.z >> sh, w.w >> sh) : make_uint4(0, 0, 0, 0);
                if (sizeof(KeyT) == 4) {
                    reinterpret_cast<uint4*>(A)[i] = v;   // one 16-byte store (A is 16-byte aligned)
                } else {
                    A[4 * i] = v.x;
                    A[4 * i + 1] = v.y;
                    A[4 * i + 2] = v.z;
                    A[4 * i + 3] = v.w;
                }
                count(v.x);
                count(v.y);
                count(v.z);
                count(v.w);
            }
            if (tid == 0 && (k & 3u)) {
                const uint4 w = philox_block(full, tag, r.id, key);
                const uint32_t ws[3] = {w.x, w.y, w.z};
                for (uint32_t c = 0; c < (k & 3u); ++c) keep(4 * full + c, sh < 32 ? (ws[c] >> sh) : 0u);
            }
        } else {
            const uint32_t sh = 64u - t;   // s > 2^32: 1 <= sh < 32
            const uint32_t full = k >> 1;
            for (uint32_t i = tid; i < full; i += NT) {
                const uint4 w = philox_block(i, tag, r.id, key);
                keep(2 * i, ((((uint64_t)w.y) << 32) | w.x) >> sh);
                keep(2 * i + 1, ((((uint64_t)w.w) << 32) | w.z) >> sh);
            }
            if (tid == 0 && (k & 1u)) {
                const uint4 w = philox_block(full, tag, r.id, key);
                keep(2 * full, ((((uint64_t)w.y) << 32) | w.x) >> sh);
            }
        }
        if (tid == 0) sm.jnext = k;
        group_sync<BAR, NT>();
    } else if (INL && r.s <= (1ull << 32)) {
        // round 1 of void_leaf_pass1, inline; the hole rounds are a call
        if (k > (min((uint64_t)c_caps.stream_blocks, (uint64_t)1 << 32) << 2)) return false;
        const uint32_t s32 = (uint32_t)(r.s - 1), thr32 = (uint32_t)thr;
        const uint32_t full = k >> 2;
        uint32_t* H = reinterpret_cast<uint32_t*>(B);
        auto put = [&](uint32_t j, uint32_t v, bool ok) {
            if (ok) {
                const uint32_t b = hash_slot((KeyT)v, mult);
                atomicAdd(&cw[b >> 1], 1u << ((b & 1u) << 4));
            } else {
                H[atomicAdd(&sm.fill, 1u)] = j;
            }
        };
        for (uint32_t i = tid; i < full; i += NT) {
            const uint4 w = philox_block(i, tag, r.id, key);
            const uint64_t p0 = (uint64_t)w.x * s32 + w.x, p1 = (uint64_t)w.y * s32 + w.y;
            const uint64_t p2 = (uint64_t)w.z * s32 + w.z, p3 = (uint64_t)w.w * s32 + w.w;
            const uint4 v = make_uint4((uint32_t)(p0 >> 32), (uint32_t)(p1 >> 32), (uint32_t)(p2 >> 32),
                                       (uint32_t)(p3 >> 32));
            if (sizeof(KeyT) == 4) {
                reinterpret_cast<uint4*>(A)[i] = v;
            } else {
                A[4 * i] = v.x;
                A[4 * i + 1] = v.y;
                A[4 * i + 2] = v.z;
                A[4 * i + 3] = v.w;
            }
            put(4 * i, v.x, (uint32_t)p0 >= thr32);
            put(4 * i + 1, v.y, (uint32_t)p1 >= thr32);
            put(4 * i + 2, v.z, (uint32_t)p2 >= thr32);
            put(4 * i + 3, v.w, (uint32_t)p3 >= thr32);
        }
        if (tid == 0 && (k & 3u)) {
            const uint4 w = philox_block(full, tag, r.id, key);
            const uint32_t ws[3] = {w.x, w.y, w.z};
            for (uint32_t c = 0; c < (k & 3u); ++c) {
                const uint64_t p = (uint64_t)ws[c] * s32 + ws[c];
                A[4 * full + c] = (KeyT)(p >> 32);
                put(4 * full + c, (uint32_t)(p >> 32), (uint32_t)p >= thr32);
            }
        }
        group_sync<BAR, NT>();
        const uint32_t nh = sm.fill;
        if (nh == 0) {
            if (tid == 0) sm.jnext = k;
        } else if (!void_fill_holes<KeyT, NT, BAR, CAP>(sm, r, key, tag, k, nh, thr, mult, A, B, cw, tid)) {
            return false;
        }
        group_sync<BAR, NT>();
    } else {
        // leaves with void candidates: a call of its own (its registers stay
        // out of the power-of-two path)
        if (!void_leaf_pass1<KeyT, NT, BAR, CAP>(sm, r, key, tag, k, thr, mult, A, B, cw, tid)) return false;
        group_sync<BAR, NT>();
    }
    // B[k .. k+3) hold the largest key value (after pass 1, which may stage
    // candidates there): the rank pass's window of four may run past the end
    // of the leaf, and reads past a key's bucket meet only larger keys
    // (buckets are monotone in the key) or these
    if (tid < 3) B[k + tid] = ~KeyT(0);
    scan_counts16<NT>(cw, nb, sm.scan_tmp, tid);   // half b = first position of bucket b
    // Passes 2 and 3 take four independent keys per thread at a time so
    // that their load -> address -> load chains overlap.
    constexpr uint32_t U = 4;
    // pass 2: scatter into bucket order; afterwards half b = end of bucket b
    auto scatter = [&](KeyT x) {
        const uint32_t b = hash_slot(x, mult);
        const uint32_t sh = (b & 1u) << 4;
        B[(atomicAdd(&cw[b >> 1], 1u << sh) >> sh) & 0xFFFFu] = x;
    };
    if (sizeof(KeyT) == 4) {   // four keys per 16-byte load (the order within a bucket is free)
        const uint32_t k4 = k >> 2;
        for (uint32_t g = tid; g < k4; g += NT) {
            const uint4 v = reinterpret_cast<const uint4*>(A)[g];
            scatter((KeyT)v.x);
            scatter((KeyT)v.y);
            scatter((KeyT)v.z);
            scatter((KeyT)v.w);
        }
        for (uint32_t j = 4 * k4 + tid; j < k; j += NT) scatter(A[j]);
    } else {
        for (uint32_t j0 = tid; j0 < k; j0 += U * NT) {
            KeyT x[U];
#pragma unroll
            for (uint32_t q = 0; q < U; ++q) x[q] = j0 + q * NT < k ? A[j0 + q * NT] : KeyT(0);
#pragma unroll
            for (uint32_t q = 0; q < U; ++q)
                if (j0 + q * NT < k) scatter(x[q]);
        }
    }
    group_sync<BAR, NT>();
    // pass 3: the rank of B[i] among its bucket's keys, ordered by (key,
    // position in B), is its place in the sorted leaf; it lies in the
    // bucket's range, a few places from i, so the stores straight to the
    // output stay nearly coalesced.  The first run counts only the smaller
    // keys: equal keys then share a rank, which shows as a sum of ranks below
    // k (k - 1) / 2, and a second run breaks the ties.
    // With replacement, a leaf of size s likely has equal keys once k^2 is
    // about s (P(none) ~ exp(-k^2 / 2s)): it takes the tie-broken run at once.
    if (WR && (uint64_t)k * k >= r.s / 2) return bucket_ties<KeyT, NT, BAR, WR, CAP>(sm, r, key, k, thr, mult, dst, tid);
    const uint32_t rsum =
        __reduce_add_sync(0xFFFFFFFFu, rank_keys<KeyT, NT, false, WR>(B, A, ch, k, mult, r.lo + 1, dst, tid));
    if ((tid & 31) == 0) atomicAdd(&sm.ranksum, rsum);
    group_sync<BAR, NT>();
    // (a barrier either way: the next leaf clears the counts this pass reads)
    if (sm.ranksum == (uint32_t)((uint64_t)k * (k - 1) / 2)) return true;
    return bucket_ties<KeyT, NT, BAR, WR, CAP>(sm, r, key, k, thr, mult, dst, tid);
}

// Rounds of distinct insertion shared by the bitmap and probing paths:
// insert(v) returns 1 if v was new.  Returns false if the candidate stream
// ran out (status set).
template <int NT, int BAR, typename Insert, typename Abort>
RS_DEV bool distinct_rounds(uint32_t* newcount, const LeafRec& r, uint64_t thr, Key2 key, uint32_t tag, uint32_t k,
                            int* status, uint32_t tid, Insert&& insert, Abort&& aborted) {
    uint32_t d = 0, round = 0;
    uint64_t J = 0;
    const uint64_t jlimit = (r.s > (1ull << 32) ? 2 : 4) * c_caps.stream_blocks;
    while (d < k) {
        const uint32_t m = k - d;
        if (J + m > jlimit) {
            if (tid == 0) set_status(status, RS_EITER);
            group_sync<BAR, NT>();
            return false;
        }
        uint32_t added = 0;
        bool vs = false;
        for_candidates<NT>(r, thr, key, tag, J, m, tid, &vs, [&](uint32_t, uint64_t v) { added += insert(v); });
        if (added) atomicAdd(&newcount[round % 3], added);
        // Counter (round+1) % 3 was last read before the previous round's
        // barrier, which this thread has passed, and is next written after
        // this round's barrier: clearing it here races with nothing.
        if (tid == 0) newcount[(round + 1) % 3] = 0;
        group_sync<BAR, NT>();
        d += newcount[round % 3];
        J += m;
        ++round;
        if (aborted()) return true;
    }
    return true;
}

// Count path for dense leaves with replacement (s below the table size): the first
// n' valid candidates are tallied per value; an exclusive scan of the tallies
// gives each value's run of output positions.
template <typename KeyT, int NT, int BAR, uint32_t CAP>
RS_COLD void count_leaf(HashShared<KeyT, NT / 32, CAP>& sm, const LeafRec& r, Key2 key, uint32_t k,
                       uint64_t* __restrict__ dst, int* status, uint32_t tid) {
    uint32_t* h = reinterpret_cast<uint32_t*>(sm.tab);
    const uint32_t s = (uint32_t)r.s;
    for (uint32_t i = tid; i <= s; i += NT) h[i] = 0;
    if (tid < 3) sm.newcount[tid] = 0;
    if (tid == 0) sm.thr = lemire_threshold(r.s);
    group_sync<BAR, NT>();
    const bool ok = distinct_rounds<NT, BAR>(
        sm.newcount, r, sm.thr, key, TAG_LEAF_WR, k, status, tid,
        [&](uint64_t v) -> uint32_t {
            atomicAdd(&h[v], 1u);
            return 1u;
        },
        [] { return false; });
    if (!ok) return;
    block_scan_counts<NT>(h, s, sm.scan_tmp);   // h[v] = first position of value v, h[s] = k
    for (uint32_t o = tid; o < k; o += NT) {
        uint32_t lo = 0, hi = s;   // the value whose run holds o: last v with h[v] <= o
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (h[mid] <= o) lo = mid; else hi = mid;
        }
        dst[o] = r.lo + 1 + lo;
    }
    group_sync<BAR, NT>();
}

// Bitmap path for leaves without replacement with s at most the table bits.
template <typename KeyT, int NT, int BAR, uint32_t CAP>
RS_COLD void bitmap_leaf(HashShared<KeyT, NT / 32, CAP>& sm, const LeafRec& r, Key2 key, uint32_t k, bool comp,
                        uint64_t* __restrict__ dst, int* status, uint32_t tid) {
    constexpr int NW = NT / 32;
    const uint32_t lane = tid & 31, warp = tid >> 5;
    uint32_t* bm = reinterpret_cast<uint32_t*>(sm.tab);
    const uint32_t words = (uint32_t)((r.s + 31) >> 5);
    for (uint32_t i = tid; i < words; i += NT) bm[i] = 0;
    if (tid < 3) sm.newcount[tid] = 0;
    if (tid == 0) sm.thr = lemire_threshold(r.s);
    group_sync<BAR, NT>();
    const bool ok = distinct_rounds<NT, BAR>(
        sm.newcount, r, sm.thr, key, TAG_LEAF_H, k, status, tid,
        [&](uint64_t v) -> uint32_t {
            const uint32_t bit = 1u << (v & 31);
            return (atomicOr(&bm[v >> 5], bit) & bit) ? 0u : 1u;
        },
        [] { return false; });
    if (!ok) return;
    // each warp takes a contiguous run of words; a lane takes one bit of the
    // current word so that the writes are coalesced
    const uint32_t per = (words + NW - 1) / NW;
    const uint32_t w0 = min(warp * per, words), w1 = min(w0 + per, words);
    auto bits_of = [&](uint32_t w) {
        uint32_t bits = bm[w];
        if (comp) {
            bits = ~bits;
            if ((uint64_t)w * 32 + 32 > r.s) bits &= (1u << (uint32_t)(r.s & 31)) - 1u;   // beyond the leaf
        }
        return bits;
    };
    uint32_t cnt = 0;
    for (uint32_t w = w0 + lane; w < w1; w += 32) cnt += __popc(bits_of(w));
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
    if (lane == 0) sm.warp_cnt[warp] = cnt;
    group_sync<BAR, NT>();
    uint32_t base = 0;
    for (uint32_t i = 0; i < warp; ++i) base += sm.warp_cnt[i];
    const uint32_t nout = comp ? (uint32_t)(r.s - k) : k;
    if ((uint64_t)nout * 8 >= (uint64_t)words * 32) {
        // dense: a word at a time, one bit per lane (coalesced stores)
        for (uint32_t w = w0; w < w1; ++w) {
            const uint32_t bits = bits_of(w);
            if ((bits >> lane) & 1u)
                dst[base + __popc(bits & ((1u << lane) - 1u))] = r.lo + 1 + (uint64_t)w * 32 + lane;
            base += __popc(bits);
        }
    } else {
        // sparse: 32 words at a time, one per lane; a warp scan of their bit
        // counts places each lane's run of outputs
        for (uint32_t wc = w0; wc < w1; wc += 32) {
            const uint32_t w = wc + lane;
            uint32_t bits = w < w1 ? bits_of(w) : 0u;
            const uint32_t c = __popc(bits);
            uint32_t incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= (uint32_t)o) incl += y;
            }
            uint32_t p = base + incl - c;
            while (bits) {
                const uint32_t t = (uint32_t)__ffs(bits) - 1u;
                dst[p++] = r.lo + 1 + (uint64_t)w * 32 + t;
                bits &= bits - 1u;
            }
            base += __shfl_sync(0xFFFFFFFFu, incl, 31);
        }
    }
    group_sync<BAR, NT>();
}

// Probing path.  Returns false if a probe ran past the slack (general path).
template <typename KeyT, int NT, int BAR, bool WR, uint32_t CAP>
RS_COLD bool probe_leaf(HashShared<KeyT, NT / 32, CAP>& sm, const LeafRec& r, Key2 key, uint32_t k,
                       uint64_t* __restrict__ dst, int* status, uint32_t tid) {
    constexpr int NW = NT / 32;
    constexpr KeyT E = HashEmpty<KeyT>::v;
    const uint32_t tag = WR ? TAG_LEAF_WR : TAG_LEAF_H;
    const uint32_t lane = tid & 31, warp = tid >> 5;
    const uint32_t T = ((2 * k + 127) / 128) * 128;
    {
        uint32_t* w32 = reinterpret_cast<uint32_t*>(sm.tab);
        const uint32_t n32 = (T + kHashSlack) * (uint32_t)(sizeof(KeyT) / 4);
        uint4* w128 = reinterpret_cast<uint4*>(w32);
        for (uint32_t i = tid; i < n32 / 4; i += NT) w128[i] = make_uint4(~0u, ~0u, ~0u, ~0u);
        if (tid == 0) {
            sm.newcount[0] = 0;
            sm.newcount[1] = 0;
            sm.newcount[2] = 0;
            sm.topcount = 0;
            sm.overflow = 0;
            sm.mult = slot_mult<KeyT>(r.s, T);
            sm.thr = lemire_threshold(r.s);
        }
    }
    group_sync<BAR, NT>();
    const uint64_t mult = sm.mult;
    const bool ok = distinct_rounds<NT, BAR>(
        sm.newcount, r, sm.thr, key, tag, k, status, tid,
        [&](uint64_t v64) -> uint32_t {
            const KeyT v = (KeyT)v64;
            if (sizeof(KeyT) == 4 && v == E) {
                const uint32_t old = atomicAdd(&sm.topcount, 1u);
                return WR ? 1u : (old == 0);
            }
            uint32_t i = hash_slot(v, mult);
            const uint32_t end = T + kHashSlack;
            while (i < end) {
                const KeyT old = cas_key(&sm.tab[i], E, v);
                if (old == E) return 1u;
                if (!WR && old == v) return 0u;
                ++i;
            }
            sm.overflow = 1;
            return 0u;
        },
        [&] { return sm.overflow != 0; });
    if (!ok) return true;
    if (sm.overflow != 0) {
        group_sync<BAR, NT>();
        return false;
    }
    // read-out: count occupied slots per warp chunk, then rank inside clusters
    const uint32_t chunk = ((T / NW) + 31) & ~31u;
    const uint32_t c0 = min(warp * chunk, T), c1 = min(c0 + chunk, T);
    const uint32_t c1x = (warp == NW - 1) ? T + kHashSlack : c1;   // the last warp owns the slack
    uint32_t cnt = 0;
    for (uint32_t i = c0 + lane; i < c1x; i += 32) cnt += sm.tab[i] != E;
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
    if (lane == 0) sm.warp_cnt[warp] = cnt;
    group_sync<BAR, NT>();
    uint32_t base = 0;
    for (uint32_t i = 0; i < warp; ++i) base += sm.warp_cnt[i];
    for (uint32_t i0 = c0; i0 < c1x; i0 += 32) {
        const uint32_t i = i0 + lane;
        const KeyT v = i < c1x ? sm.tab[i] : E;
        const bool occ = v != E;
        const uint32_t mask = __ballot_sync(0xFFFFFFFFu, occ);
        if (occ) {
            const uint32_t before = base + __popc(mask & ((1u << lane) - 1u));
            const bool left = lane > 0 ? ((mask >> (lane - 1)) & 1u) : (i > 0 && sm.tab[i - 1] != E);
            const bool right = lane < 31 ? ((mask >> (lane + 1)) & 1u) : (i + 1 < T + kHashSlack && sm.tab[i + 1] != E);
            uint32_t pos = before;
            if (left || right) {
                uint32_t cs = i, ce = i + 1;
                while (cs > 0 && sm.tab[cs - 1] != E) --cs;
                while (ce < T + kHashSlack && sm.tab[ce] != E) ++ce;
                uint32_t rank = 0;
                for (uint32_t t = cs; t < ce; ++t) {
                    const KeyT y = sm.tab[t];
                    rank += (y < v) || (WR && y == v && t < i);
                }
                pos = before - (i - cs) + rank;
            }
            dst[pos] = r.lo + 1 + (uint64_t)v;
        }
        base += __popc(mask);
    }
    if (sizeof(KeyT) == 4) {
        const uint32_t top = WR ? sm.topcount : (sm.topcount ? 1u : 0u);   // copies of 2^32-1 go last
        for (uint32_t t = tid; t < top; t += NT) dst[k - top + t] = r.lo + 1 + 0xFFFFFFFFull;
    }
    group_sync<BAR, NT>();
    return true;
}

// Selects the leaf's values and writes them sorted to out[off ..].  Returns
// false if the leaf must go to the general (global-memory) path, having
// written nothing of use.  All NT threads of the group call it; tid is the
// thread's index in the group.
template <typename KeyT, int NT, int BAR, bool WR, uint32_t CAP = kHashCap, typename K2 = Key2, bool POW2 = false,
          bool INL = false>
RS_DEV bool hash_leaf(HashShared<KeyT, NT / 32, CAP>& sm, const LeafRec& r, const K2& key, uint64_t* __restrict__ out,
                      int* status, uint32_t tid, uint32_t cap) {
    const bool comp = !WR && (r.np > r.s - r.np);
    const uint64_t k64 = comp ? r.s - r.np : r.np;
    if (k64 > cap) return false;
    const uint32_t k = (uint32_t)k64;
    uint64_t* dst = out + r.off;
    const bool use_bitmap = !WR && r.s <= HashShared<KeyT, NT / 32, CAP>::kBits && (comp || r.s <= 64ull * k);
    if (comp && !use_bitmap) return false;
    if (k == 0 && !comp) return true;
    if (WR && r.s < HashShared<KeyT, NT / 32, CAP>::kSlots && r.s <= 64ull * k) {
        count_leaf<KeyT, NT, BAR, CAP>(sm, r, key, k, dst, status, tid);
        return true;
    }
    if (use_bitmap) {
        bitmap_leaf<KeyT, NT, BAR, CAP>(sm, r, key, k, comp, dst, status, tid);
        return true;
    }
    if (bucket_leaf<KeyT, NT, BAR, WR, CAP, K2, POW2, INL>(sm, r, key, k, dst, tid)) return true;
    return probe_leaf<KeyT, NT, BAR, WR, CAP>(sm, r, key, k, dst, status, tid);
}

}  // namespace rs
