// rs_block.cuh -- block-wide scans and reductions used by the leaf kernels.
#pragma once
#include "rs_common.cuh"

namespace rs {

// Exclusive scan of one value per thread across a block of NT threads.
// `tmp` needs NT/32 + 1 words of shared memory.  Returns the exclusive
// prefix; *total receives the block sum.  Contains three __syncthreads(),
// the last one after `tmp` has been read, so calls may follow each other.
template <int NT>
RS_DEV uint32_t block_exclusive_scan(uint32_t x, uint32_t* tmp, uint32_t* total) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) tmp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < NW ? tmp[lane] : 0;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < NW) tmp[lane] = wi - w;
        if (lane == NW - 1) tmp[NW] = wi;
    }
    __syncthreads();
    const uint32_t r = tmp[warp] + incl - x;
    *total = tmp[NW];
    __syncthreads();
    return r;
}

// In-place exclusive scan of cnt[0..T); afterwards cnt[T] = sum.  Each
// thread scans a contiguous run of ceil(T/NT) counters.  Ends synchronized.
template <int NT>
RS_DEV void block_scan_counts(uint32_t* cnt, uint32_t T, uint32_t* tmp) {
    const uint32_t per = (T + NT - 1) / NT;
    const uint32_t b0 = threadIdx.x * per;
    const uint32_t b1 = min(b0 + per, T);
    uint32_t local = 0;
    for (uint32_t b = b0; b < b1; ++b) local += cnt[b];
    uint32_t total;
    uint32_t run = block_exclusive_scan<NT>(local, tmp, &total);
    for (uint32_t b = b0; b < b1; ++b) {
        const uint32_t c = cnt[b];
        cnt[b] = run;
        run += c;
    }
    if (threadIdx.x == 0) cnt[T] = total;
    __syncthreads();
}

// Number of elements < key (strict) or <= key in the sorted range a[0..n).
template <typename KeyT>
RS_DEV uint32_t lower_bound(const KeyT* a, uint32_t n, KeyT key) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}
template <typename KeyT>
RS_DEV uint32_t upper_bound(const KeyT* a, uint32_t n, KeyT key) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (a[mid] <= key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

RS_DEV uint32_t next_pow2_at_least(uint32_t x, uint32_t floor_value) {
    uint32_t t = floor_value;
    while (t < x) t <<= 1;
    return t;
}

}  // namespace rs
