// rs_leaf.cu -- base-case kernels: leaf H (without replacement) and leaf WR
// (with replacement), plus the sorted write-out.
//
// Leaf H is Algorithm H (Sec. 2) with sorted output (Sec. 4.1): the leaf's
// selection is the first k distinct valid candidates of its LEAF_H stream,
// k = n' (or s - n' when more than half the leaf is taken, whose complement
// is then written: Sec. 2's n > N/2 rule applied per leaf).
//
// Leaf WR (Sec. 4.6) is the same machinery without the distinctness rule:
// the first n' valid candidates of its LEAF_WR stream, sorted as a multiset.
#include "rs_hash_leaf.cuh"
#include "rs_leaf.cuh"

namespace rs {

struct LeafJob {
    const NodeRec* leaves;   // leaf records, leaf i at leaves[i]
    uint64_t nleaves;
    uint64_t first_id;       // heap id of leaf 0 (= 2^D)
    uint64_t seed;
    uint64_t* out;
    int* status;
    uint32_t* ovf_list;      // leaves left to the general path
    uint32_t* ovf_count;
    uint32_t cap;            // largest selection handled here
};

constexpr int kHashThreads = 256;

// One block per leaf at a time, persistent over the leaves; leaves the
// shared-memory table cannot take go to the general path's list.
template <typename KeyT, bool WR>
__global__ void __launch_bounds__(kHashThreads) leaf_kernel(LeafJob job) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto& sm = *reinterpret_cast<HashShared<KeyT, kHashThreads / 32>*>(smem_raw);
    const Key2 key = make_key(job.seed);
    for (uint64_t leaf = blockIdx.x; leaf < job.nleaves; leaf += gridDim.x) {
        const NodeRec r = job.leaves[leaf];
        if (r.c == 0) continue;
        const LeafRec lr{r.lo, r.S, r.c, r.off, job.first_id + leaf};
        if (!hash_leaf<KeyT, kHashThreads, 0, WR>(sm, lr, key, job.out, job.status, threadIdx.x, job.cap)) {
            if (threadIdx.x == 0) job.ovf_list[atomicAdd(job.ovf_count, 1u)] = (uint32_t)leaf;
        }
    }
}

// ---------------------------------------------------------------------------
// General path: the same rounds over global scratch memory, one block per
// leaf, for selections larger than the shared-memory capacity.
// ---------------------------------------------------------------------------

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
    const uint64_t jlimit = wide ? (1ull << 33) : (1ull << 34);
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

template <bool WR>
__global__ void __launch_bounds__(kBigThreads) big_leaf_kernel(LeafJob job, BigScratch sc) {
    __shared__ uint32_t tmp[kBigThreads / 32 + 1];
    const Key2 key = make_key(job.seed);
    const uint32_t count = *job.ovf_count;
    for (uint32_t t = 0; t < count; ++t) {
        const uint64_t leaf = job.ovf_list[t];
        const NodeRec r = job.leaves[leaf];
        const bool comp = !WR && (r.c > r.S - r.c);
        const uint64_t k = comp ? r.S - r.c : r.c;
        if (k > sc.kmax) {
            if (threadIdx.x == 0) set_status(job.status, RS_ECAPACITY);
            continue;
        }
        if (!big_select<WR>(r, job.first_id + leaf, key, k, sc, tmp, job.status)) continue;
        uint64_t* dst = job.out + r.off;
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
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------

template <typename KeyT, bool WR>
static cudaError_t launch_fast(const LeafJob& job, int sms, cudaStream_t st) {
    const size_t smem = sizeof(HashShared<KeyT, kHashThreads / 32>);
    auto kern = leaf_kernel<KeyT, WR>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kHashThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const uint64_t grid = std::min<uint64_t>(job.nleaves, (uint64_t)sms * per_sm);
    kern<<<(unsigned)grid, kHashThreads, smem, st>>>(job);
    return cudaGetLastError();
}

cudaError_t launch_leaves(const LeafLaunch& L, cudaStream_t st) {
    LeafJob job{L.leaves, L.nleaves, L.first_id, L.seed, L.out, L.status, L.ovf_list, L.ovf_count,
                L.cap ? std::min<uint32_t>(L.cap, kHashCap) : kHashCap};
    cudaError_t e = cudaMemsetAsync(L.ovf_count, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    const bool narrow = L.smax <= (1ull << 32);
    if (L.with_replacement)
        e = narrow ? launch_fast<uint32_t, true>(job, L.sms, st) : launch_fast<uint64_t, true>(job, L.sms, st);
    else
        e = narrow ? launch_fast<uint32_t, false>(job, L.sms, st) : launch_fast<uint64_t, false>(job, L.sms, st);
    if (e != cudaSuccess) return e;
    if (L.big_kmax == 0) return cudaSuccess;   // no leaf can exceed the capacity
    BigScratch sc;
    uint64_t kmax = L.big_kmax;
    uint64_t tmax = 32;
    while (tmax < kmax) tmax <<= 1;
    unsigned char* p = static_cast<unsigned char*>(L.big_pool);
    sc.keys = reinterpret_cast<uint64_t*>(p); p += kmax * 8;
    sc.cand = reinterpret_cast<uint64_t*>(p); p += kmax * 8;
    sc.tmp = reinterpret_cast<uint64_t*>(p); p += kmax * 8;
    sc.bkt = reinterpret_cast<uint32_t*>(p); p += kmax * 4;
    sc.arr = reinterpret_cast<uint32_t*>(p); p += kmax * 4;
    sc.cnt = reinterpret_cast<uint32_t*>(p);
    sc.kmax = kmax;
    if (L.with_replacement) big_leaf_kernel<true><<<1, kBigThreads, 0, st>>>(job, sc);
    else big_leaf_kernel<false><<<1, kBigThreads, 0, st>>>(job, sc);
    return cudaGetLastError();
}

uint64_t big_pool_bytes(uint64_t kmax) {
    uint64_t tmax = 32;
    while (tmax < kmax) tmax <<= 1;
    return kmax * (8 + 8 + 8 + 4 + 4) + (tmax + 1) * 4;
}

}  // namespace rs
