// rs_big_leaf.cuh -- the general (global-memory) leaf path.
//
// Leaves whose selection exceeds the shared-memory capacity run the same
// rounds as the shared-memory paths (first k distinct valid candidates,
// Sec. 2 Algorithm H; sorted, Sec. 4.1) over global scratch: candidates are
// bucketed by their top bits with a counting sort, buckets ordered by rank,
// duplicates and already-selected values dropped, survivors merged.
#pragma once
#include "rs_leaf.cuh"

namespace rs {

constexpr int kBigThreads = 1024;

struct BigScratch {
    uint64_t* keys;   // kmax
    uint64_t* cand;   // kmax
    uint64_t* tmp;    // kmax
    uint32_t* bkt;    // kmax
    uint32_t* arr;    // kmax
    uint32_t* cnt;    // tmax + 1
    uint64_t kmax;
};

// The scratch arrays carved from one pool of big_pool_bytes(kmax) bytes.
inline BigScratch carve_big_scratch(void* pool, uint64_t kmax) {
    BigScratch sc;
    unsigned char* p = static_cast<unsigned char*>(pool);
    sc.keys = reinterpret_cast<uint64_t*>(p); p += kmax * 8;
    sc.cand = reinterpret_cast<uint64_t*>(p); p += kmax * 8;
    sc.tmp = reinterpret_cast<uint64_t*>(p); p += kmax * 8;
    sc.bkt = reinterpret_cast<uint32_t*>(p); p += kmax * 4;
    sc.arr = reinterpret_cast<uint32_t*>(p); p += kmax * 4;
    sc.cnt = reinterpret_cast<uint32_t*>(p);
    sc.kmax = kmax;
    return sc;
}

template <int CPB>
RS_DEV void big_round(const Draw<CPB>& draw, Key2 key, uint32_t tag, uint64_t id, uint64_t s, uint64_t J,
                      uint64_t m, uint32_t T, uint64_t d, const BigScratch& sc, uint32_t* tmp, uint64_t* mv_out,
                      bool* dup_out) {
    const uint64_t mult = bucket_mult<uint64_t>(s, T);
    for (uint64_t i = threadIdx.x; i <= T; i += kBigThreads) sc.cnt[i] = 0;
    __syncthreads();
    const uint64_t blk_lo = J / CPB, blk_hi = (J + m - 1) / CPB;
    for (uint64_t blk = blk_lo + threadIdx.x; blk <= blk_hi; blk += kBigThreads) {
        const uint4 w = philox_block((uint32_t)blk, tag, id, key);
        for (int c = 0; c < CPB; ++c) {
            const uint64_t j = blk * CPB + c;
            if (j < J || j >= J + m) continue;
            const uint64_t slot = j - J;
            uint64_t x;
            sc.bkt[slot] = kInvalid;
            if (draw(w, c, x)) {
                const uint32_t b = bucket_of(x, mult);
                sc.cand[slot] = x;
                sc.bkt[slot] = b;
                sc.arr[slot] = atomicAdd(&sc.cnt[b], 1u);
            }
        }
    }
    __syncthreads();
    // exclusive scan of the counts
    {
        const uint64_t per = (T + kBigThreads - 1) / kBigThreads;
        const uint64_t b0 = threadIdx.x * per, b1 = min(b0 + per, (uint64_t)T);
        uint32_t local = 0;
        for (uint64_t b = b0; b < b1; ++b) local += sc.cnt[b];
        uint32_t total;
        uint32_t run = block_exclusive_scan<kBigThreads>(local, tmp, &total);
        for (uint64_t b = b0; b < b1; ++b) {
            const uint32_t c = sc.cnt[b];
            sc.cnt[b] = run;
            run += c;
        }
        if (threadIdx.x == 0) sc.cnt[T] = total;
        __syncthreads();
    }
    for (uint64_t slot = threadIdx.x; slot < m; slot += kBigThreads) {
        if (sc.bkt[slot] != kInvalid) sc.keys[d + sc.cnt[sc.bkt[slot]] + sc.arr[slot]] = sc.cand[slot];
    }
    __syncthreads();
    bool dup = false;
    for (uint64_t slot = threadIdx.x; slot < m; slot += kBigThreads) {
        if (sc.bkt[slot] == kInvalid) continue;
        const uint32_t b = sc.bkt[slot];
        const uint64_t bs = sc.cnt[b], be = sc.cnt[b + 1];
        const uint64_t pos = bs + sc.arr[slot];
        const uint64_t x = sc.cand[slot];
        uint64_t r = 0;
        for (uint64_t i = bs; i < be; ++i) {
            const uint64_t y = sc.keys[d + i];
            r += (y < x) || (y == x && i < pos);
            dup |= (y == x) && (i != pos);
        }
        sc.arr[slot] = (uint32_t)r;
    }
    __syncthreads();
    for (uint64_t slot = threadIdx.x; slot < m; slot += kBigThreads) {
        if (sc.bkt[slot] != kInvalid) sc.keys[d + sc.cnt[sc.bkt[slot]] + sc.arr[slot]] = sc.cand[slot];
    }
    *dup_out = __syncthreads_or(dup) != 0;
    *mv_out = sc.cnt[T];
}

template <bool WR>
RS_DEV bool big_select(const NodeRec& r, uint64_t id, Key2 key, uint64_t k, const BigScratch& sc, uint32_t* tmp,
                       int* status) {
    const uint32_t tag = WR ? TAG_LEAF_WR : TAG_LEAF_H;
    const bool wide = r.S > (1ull << 32);
    const uint64_t jlimit = (wide ? 2 : 4) * c_caps.stream_blocks;
    uint64_t d = 0, J = 0;
    while (d < k) {
        const uint64_t m = k - d;
        if (J + m > jlimit) {
            if (threadIdx.x == 0) set_status(status, RS_EITER);
            return false;
        }
        uint32_t T = 32;
        while (T < m) T <<= 1;
        uint64_t mv;
        bool dup;
        if (wide) {
            Draw<2> dr{Bounded64{r.S, (0ull - r.S) % r.S}};
            big_round<2>(dr, key, tag, id, r.S, J, m, T, d, sc, tmp, &mv, &dup);
        } else {
            Draw<4> dr{Bounded32{r.S, (uint32_t)(((1ull << 32) - r.S) % r.S)}};
            big_round<4>(dr, key, tag, id, r.S, J, m, T, d, sc, tmp, &mv, &dup);
        }
        J += m;
        uint64_t x = mv;
        if (!WR && (d > 0 || dup)) {
            // keep first-of-run values that are not yet selected, in order
            const uint64_t per = (mv + kBigThreads - 1) / kBigThreads;
            const uint64_t i0 = threadIdx.x * per, i1 = min(i0 + per, mv);
            uint32_t count = 0;
            for (uint64_t i = i0; i < i1; ++i) {
                const uint64_t e = sc.keys[d + i];
                bool keep = (i == 0) || sc.keys[d + i - 1] != e;
                if (keep && d > 0) {
                    uint64_t lo = 0, hi = d;
                    while (lo < hi) {
                        const uint64_t mid = (lo + hi) >> 1;
                        if (sc.keys[mid] < e) lo = mid + 1; else hi = mid;
                    }
                    keep = !(lo < d && sc.keys[lo] == e);
                }
                count += keep;
            }
            uint32_t total;
            uint32_t w = block_exclusive_scan<kBigThreads>(count, tmp, &total);
            for (uint64_t i = i0; i < i1; ++i) {
                const uint64_t e = sc.keys[d + i];
                bool keep = (i == 0) || sc.keys[d + i - 1] != e;
                if (keep && d > 0) {
                    uint64_t lo = 0, hi = d;
                    while (lo < hi) {
                        const uint64_t mid = (lo + hi) >> 1;
                        if (sc.keys[mid] < e) lo = mid + 1; else hi = mid;
                    }
                    keep = !(lo < d && sc.keys[lo] == e);
                }
                if (keep) sc.tmp[w++] = e;
            }
            __syncthreads();
            x = total;
            for (uint64_t i = threadIdx.x; i < x; i += kBigThreads) sc.keys[d + i] = sc.tmp[i];
            __syncthreads();
        }
        if (d > 0) {
            const uint64_t n = d + x;
            for (uint64_t i = threadIdx.x; i < n; i += kBigThreads) {
                const uint64_t e = sc.keys[i];
                uint64_t lo = 0, hi, base;
                const uint64_t* a;
                if (i < d) { a = sc.keys + d; hi = x; base = i; }
                else { a = sc.keys; hi = d; base = i - d; }
                while (lo < hi) {
                    const uint64_t mid = (lo + hi) >> 1;
                    const bool go = i < d ? (a[mid] < e) : (a[mid] <= e);
                    if (go) lo = mid + 1; else hi = mid;
                }
                sc.tmp[base + lo] = e;
            }
            __syncthreads();
            for (uint64_t i = threadIdx.x; i < n; i += kBigThreads) sc.keys[i] = sc.tmp[i];
            __syncthreads();
        }
        d += x;
    }
    return true;
}


// Writes the selection (or its complement) of a leaf processed by big_select.
RS_DEV void big_write(const NodeRec& r, uint64_t k, bool comp, const BigScratch& sc, uint64_t* dst) {
    if (!comp) {
        for (uint64_t i = threadIdx.x; i < k; i += kBigThreads) dst[i] = r.lo + 1 + sc.keys[i];
    } else {
        const uint64_t nout = r.S - k;
        for (uint64_t o = threadIdx.x; o < nout; o += kBigThreads) {
            uint64_t lo = 0, hi = k;
            while (lo < hi) {
                const uint64_t mid = (lo + hi) >> 1;
                if (sc.keys[mid] - mid <= o) lo = mid + 1; else hi = mid;
            }
            dst[o] = r.lo + 1 + o + lo;
        }
    }
}

}  // namespace rs
