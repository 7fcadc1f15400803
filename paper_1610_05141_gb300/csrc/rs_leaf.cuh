// rs_leaf.cuh -- shared-memory selection machinery of the leaf kernels.
//
// select_leaf computes, sorted, the first k distinct (or, for sampling with
// replacement, simply the first k) valid candidates of a leaf's stream over
// [0, s) -- Algorithm H (Sec. 2) with sorted output (Sec. 4.1).  The sorted
// hash table of the paper, addressed by the most significant bits of the
// key, becomes a counting sort over a monotone bucket map
// b(v) = floor(v T / s) followed by ordering each (expected O(1)-sized)
// bucket by rank.  The result depends only on the candidate sequence.
//
// The selection is computed in rounds.  Round 1 takes candidates [0, k);
// every later round takes exactly as many candidates as values are still
// missing, starting where the previous round stopped, so a round can never
// overshoot the k-th distinct value.  Duplicates and values already selected
// are dropped and the survivors merged into the sorted selection.
#pragma once
#include "rs_block.cuh"
#include "rs_internal.h"
#include "rs_rng.cuh"

namespace rs {

constexpr int kLeafThreads = 512;
constexpr uint32_t kInvalid = 0xFFFFFFFFu;

template <typename KeyT>
struct LeafShared {
    KeyT keys[kLeafCap];
    uint32_t cnt[kLeafCap + 1];
    uint32_t tmp[kLeafThreads / 32 + 1];
};

// Candidate draws of one Philox block: CPB = 4 candidates of 32-bit words
// (s <= 2^32) or CPB = 2 candidates of 64-bit values (s > 2^32).
template <int CPB>
struct Draw;

template <>
struct Draw<4> {
    Bounded32 b;
    template <typename KeyT>
    RS_DEV bool operator()(const uint4& w, int c, KeyT& out) const {
        const uint32_t x = c == 0 ? w.x : c == 1 ? w.y : c == 2 ? w.z : w.w;
        uint32_t v;
        const bool ok = b.draw(x, v);
        out = (KeyT)v;
        return ok;
    }
};

template <>
struct Draw<2> {
    Bounded64 b;
    template <typename KeyT>
    RS_DEV bool operator()(const uint4& w, int c, KeyT& out) const {
        const uint64_t x = c == 0 ? (((uint64_t)w.y << 32) | w.x) : (((uint64_t)w.w << 32) | w.z);
        uint64_t v;
        const bool ok = b.draw(x, v);
        out = (KeyT)v;
        return ok;
    }
};

// Monotone bucket map into [0, T): floor(v * mult / 2^width), with
// mult <= T 2^width / s so that v < s gives a bucket < T.
RS_DEV uint32_t bucket_of(uint32_t v, uint64_t mult) { return __umulhi(v, (uint32_t)mult); }
RS_DEV uint32_t bucket_of(uint64_t v, uint64_t mult) { return (uint32_t)__umul64hi(v, mult); }

template <typename KeyT>
RS_DEV uint64_t bucket_mult(uint64_t s, uint32_t T) {
    if (sizeof(KeyT) == 4) {
        const uint64_t m = ((uint64_t)T << 32) / s;
        return m > 0xFFFFFFFFull ? 0xFFFFFFFFull : m;
    }
    if ((uint64_t)T >= s) return ~0ull;
    return (uint64_t)(((unsigned __int128)T << 64) / s);
}

// Round register budget: BPT Philox blocks per thread cover a batch of up to
// kLeafCap candidates plus a partial block at each end.
template <int CPB>
struct RoundShape {
    static constexpr int BPT = (int)((kLeafCap / CPB + 2 + kLeafThreads - 1) / kLeafThreads);
    static constexpr int E = BPT * CPB;
};
constexpr int kMaxE = RoundShape<4>::E > RoundShape<2>::E ? RoundShape<4>::E : RoundShape<2>::E;
constexpr int kPer = (int)(kLeafCap / kLeafThreads);   // elements per thread in merge steps

// Draws the batch of candidates [J, J+m) into registers and counts them per
// bucket (shared-memory atomics give each value its arrival slot).
template <int CPB, typename KeyT>
RS_DEV void draw_batch(const Draw<CPB>& draw, Key2 key, uint32_t tag, uint64_t id, uint64_t J, uint32_t m,
                       uint64_t mult, uint32_t* cnt, KeyT (&v)[kMaxE], uint32_t (&ba)[kMaxE]) {
    using Shape = RoundShape<CPB>;
    const uint64_t blk_lo = J / CPB, blk_hi = (J + m - 1) / CPB;
#pragma unroll
    for (int t = 0; t < Shape::BPT; ++t) {
        const uint64_t blk = blk_lo + threadIdx.x + (uint64_t)t * kLeafThreads;
        if (blk <= blk_hi) {
            const uint4 w = philox_block((uint32_t)blk, tag, id, key);
#pragma unroll
            for (int c = 0; c < CPB; ++c) {
                const int slot = t * CPB + c;
                const uint64_t j = blk * CPB + c;
                ba[slot] = kInvalid;
                if (j >= J && j < J + m) {
                    KeyT x;
                    if (draw(w, c, x)) {
                        const uint32_t b = bucket_of(x, mult);
                        const uint32_t a = atomicAdd(&cnt[b], 1u);
                        v[slot] = x;
                        ba[slot] = (b << 16) | a;
                    }
                }
            }
        } else {
#pragma unroll
            for (int c = 0; c < CPB; ++c) ba[t * CPB + c] = kInvalid;
        }
    }
#pragma unroll
    for (int slot = Shape::E; slot < kMaxE; ++slot) ba[slot] = kInvalid;
}

// Counting sort of the registered batch into keys[base .. base+mv): scan the
// bucket counts, scatter by arrival, then order each bucket by rank (ties by
// slot, which keeps equal values adjacent).  Returns mv; *dup tells whether
// two equal values met.
template <typename KeyT>
RS_DEV uint32_t sort_batch(LeafShared<KeyT>& sm, uint32_t T, uint32_t base, const KeyT (&v)[kMaxE],
                           uint32_t (&ba)[kMaxE], bool* dup_out) {
    block_scan_counts<kLeafThreads>(sm.cnt, T, sm.tmp);
    const uint32_t mv = sm.cnt[T];
#pragma unroll
    for (int slot = 0; slot < kMaxE; ++slot) {
        if (ba[slot] != kInvalid) sm.keys[base + sm.cnt[ba[slot] >> 16] + (ba[slot] & 0xFFFFu)] = v[slot];
    }
    __syncthreads();
    bool dup = false;
#pragma unroll
    for (int slot = 0; slot < kMaxE; ++slot) {
        if (ba[slot] == kInvalid) continue;
        const uint32_t b = ba[slot] >> 16, a = ba[slot] & 0xFFFFu;
        const uint32_t bs = sm.cnt[b], be = sm.cnt[b + 1];
        uint32_t fin = bs;
        if (be - bs > 1) {
            const uint32_t pos = bs + a;
            const KeyT x = v[slot];
            uint32_t r = 0;
            for (uint32_t i = bs; i < be; ++i) {
                const KeyT y = sm.keys[base + i];
                r += (y < x) || (y == x && i < pos);
                dup |= (y == x) && (i != pos);
            }
            fin = bs + r;
        }
        ba[slot] = fin;
    }
    __syncthreads();
#pragma unroll
    for (int slot = 0; slot < kMaxE; ++slot) {
        if (ba[slot] != kInvalid) sm.keys[base + ba[slot]] = v[slot];
    }
    *dup_out = __syncthreads_or(dup) != 0;
    return mv;
}

// Keeps, in order, the values of keys[d .. d+mv) that differ from their
// predecessor and are not in keys[0..d); moves them to keys[d .. d+x).
template <typename KeyT>
RS_DEV uint32_t compact_new(LeafShared<KeyT>& sm, uint32_t d, uint32_t mv) {
    const uint32_t per = (mv + kLeafThreads - 1) / kLeafThreads;
    const uint32_t i0 = threadIdx.x * per;
    KeyT vals[kPer];
    uint32_t keep = 0, count = 0;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const uint32_t i = i0 + q;
        if ((uint32_t)q < per && i < mv) {
            const KeyT e = sm.keys[d + i];
            bool k = (i == 0) || (sm.keys[d + i - 1] != e);
            if (k && d > 0) {
                const uint32_t p = lower_bound(sm.keys, d, e);
                k = !(p < d && sm.keys[p] == e);
            }
            vals[q] = e;
            keep |= (uint32_t)k << q;
            count += k;
        }
    }
    uint32_t x;
    uint32_t w = block_exclusive_scan<kLeafThreads>(count, sm.tmp, &x);
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        if (keep >> q & 1) sm.keys[d + w++] = vals[q];
    }
    __syncthreads();
    return x;
}

// Merges the sorted runs keys[0..d) and keys[d..d+x) in place.  Elements of
// the first run go before equal elements of the second.
template <typename KeyT>
RS_DEV void merge_runs(LeafShared<KeyT>& sm, uint32_t d, uint32_t x) {
    const uint32_t n = d + x;
    const uint32_t per = (n + kLeafThreads - 1) / kLeafThreads;
    const uint32_t i0 = threadIdx.x * per;
    KeyT vals[kPer];
    uint32_t pos[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const uint32_t i = i0 + q;
        pos[q] = kInvalid;
        if ((uint32_t)q < per && i < n) {
            const KeyT e = sm.keys[i];
            vals[q] = e;
            pos[q] = i < d ? i + lower_bound(sm.keys + d, x, e) : (i - d) + upper_bound(sm.keys, d, e);
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        if (pos[q] != kInvalid) sm.keys[pos[q]] = vals[q];
    }
    __syncthreads();
}

// The leaf's selection, sorted, in keys[0..k).  Returns false after setting
// the status word if the candidate stream would run out.
template <typename KeyT, int CPB, bool DISTINCT>
RS_DEV bool select_leaf(LeafShared<KeyT>& sm, const Draw<CPB>& draw, Key2 key, uint32_t tag, uint64_t id,
                        uint64_t s, uint32_t k, int* status) {
    const uint64_t jlimit = CPB == 4 ? (1ull << 34) : (1ull << 33);
    KeyT v[kMaxE];
    uint32_t ba[kMaxE];
    uint32_t d = 0;
    uint64_t J = 0;
    while (d < k) {
        const uint32_t m = k - d;
        if (J + m > jlimit) {
            if (threadIdx.x == 0) set_status(status, RS_EITER);
            return false;
        }
        const uint32_t T = next_pow2_at_least(m, 32);
        const uint64_t mult = bucket_mult<KeyT>(s, T);
        for (uint32_t i = threadIdx.x; i <= T; i += kLeafThreads) sm.cnt[i] = 0;
        __syncthreads();
        draw_batch<CPB, KeyT>(draw, key, tag, id, J, m, mult, sm.cnt, v, ba);
        __syncthreads();
        bool dup;
        const uint32_t mv = sort_batch<KeyT>(sm, T, d, v, ba, &dup);
        J += m;
        if (!DISTINCT) {
            if (d > 0) merge_runs<KeyT>(sm, d, mv);
            d += mv;
            continue;
        }
        if (d == 0 && !dup) {
            d = mv;
            continue;
        }
        const uint32_t x = compact_new<KeyT>(sm, d, mv);
        if (d > 0) merge_runs<KeyT>(sm, d, x);
        d += x;
    }
    return true;
}

// out[i] = lo + keys[i] + 1 for i < k, with 16-byte stores where aligned.
template <typename KeyT>
RS_DEV void write_sorted(const KeyT* keys, uint32_t k, uint64_t lo, uint64_t* __restrict__ dst) {
    const uint32_t head = (((uintptr_t)dst) & 15) ? 1u : 0u;
    const uint64_t base = lo + 1;
    if (head && k > 0 && threadIdx.x == 0) dst[0] = base + keys[0];
    const uint32_t rest = k > head ? k - head : 0;
    const uint32_t pairs = rest >> 1;
    for (uint32_t p = threadIdx.x; p < pairs; p += kLeafThreads) {
        const uint32_t i = head + 2 * p;
        const uint64_t a = base + keys[i], b = base + keys[i + 1];
        asm volatile("st.global.v2.u64 [%0], {%1, %2};" ::"l"(dst + i), "l"(a), "l"(b) : "memory");
    }
    if ((rest & 1) && threadIdx.x == 0) dst[k - 1] = base + keys[k - 1];
}

// Writes the complement of the sorted selection keys[0..k) within [0, s):
// output o is v = o + c with c = #{i : keys[i] - i <= o}.  Each warp walks a
// contiguous range, lane-interleaved, carrying c forward.
template <typename KeyT>
RS_DEV void write_complement(const KeyT* keys, uint32_t k, uint64_t s, uint64_t lo,
                             uint64_t* __restrict__ dst) {
    const uint64_t nout = s - k;
    constexpr uint32_t NW = kLeafThreads / 32;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t chunk = ((nout + NW - 1) / NW + 31) & ~31ull;
    const uint64_t o0 = (uint64_t)warp * chunk, o1 = min(o0 + chunk, nout);
    uint64_t o = o0 + lane;
    if (o >= o1) return;
    uint32_t lo_i = 0, hi_i = k;
    while (lo_i < hi_i) {
        const uint32_t mid = (lo_i + hi_i) >> 1;
        if ((uint64_t)keys[mid] - mid <= o) lo_i = mid + 1; else hi_i = mid;
    }
    uint32_t c = lo_i;
    for (; o < o1; o += 32) {
        while (c < k && (uint64_t)keys[c] - c <= o) ++c;
        dst[o] = lo + 1 + o + c;
    }
}

}  // namespace rs
