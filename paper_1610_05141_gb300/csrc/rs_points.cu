// rs_points.cu -- sampling with replacement from a d-dimensional box by
// bisection (Sec. 4.6: uniform samples from any space that can be halved,
// e.g. random points in a rectangle).
//
// The split tree of the one-dimensional sampler with replacement, over
// boxes: a node halves its largest extent and sends a binomial share of its
// points to the lower half (the volumes' ratio is that of the halved
// extent).  A leaf draws its points as indices into its own box with the
// library's leaf WR (sorted), and a decode pass turns each index into
// coordinates.
#include <algorithm>

#include "rs_deviates.cuh"
#include "rs_points.h"

namespace rs {

constexpr int kPointsThreads = 128;
// Levels of at most this many nodes take one warp per node.
constexpr uint64_t kPointsWarpNodes = 1024;

__global__ void box_root_kernel(BoxRec* rec, uint32_t d, BoxExtents E, uint64_t n) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    BoxRec r{};
    for (uint32_t k = 0; k < d; ++k) r.e[k] = E.e[k];
    r.c = n;
    r.off = 0;
    rec[1] = r;
}

__global__ void __launch_bounds__(kPointsThreads) box_level_kernel(BoxRec* rec, uint64_t w, uint32_t d, Key2 key,
                                                                   const double* __restrict__ tab, int* status) {
    for (uint64_t v = w + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < 2 * w;
         v += (uint64_t)gridDim.x * blockDim.x) {
        const BoxRec r = rec[v];
        uint32_t ks = 0;
        for (uint32_t k = 1; k < d; ++k)
            if (r.e[k] > r.e[ks]) ks = k;
        const uint64_t half = r.e[ks] / 2;
        uint64_t cl = 0;
        if (r.c > 0) {
            const int rc = binomial(key, v, r.c, half, r.e[ks], tab, cl);
            if (rc != RS_OK) {
                set_status(status, rc);
                cl = 0;
            }
        }
        BoxRec L = r, R = r;
        L.e[ks] = half;
        L.c = cl;
        R.o[ks] = r.o[ks] + half;
        R.e[ks] = r.e[ks] - half;
        R.c = r.c - cl;
        R.off = r.off + cl;
        rec[2 * v] = L;
        rec[2 * v + 1] = R;
    }
}

// The same for narrow levels: one warp per node, the deviate's trials spread
// over the warp's lanes.
__global__ void __launch_bounds__(kPointsThreads) box_level_warp_kernel(BoxRec* rec, uint64_t w, uint32_t d,
                                                                        Key2 key, const double* __restrict__ tab,
                                                                        int* status) {
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
    for (uint64_t v = w + (uint64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; v < 2 * w; v += warps) {
        const BoxRec r = rec[v];
        uint32_t ks = 0;
        for (uint32_t k = 1; k < d; ++k)
            if (r.e[k] > r.e[ks]) ks = k;
        const uint64_t half = r.e[ks] / 2;
        uint64_t cl = 0;
        int rc = RS_OK;
        if (r.c > 0) rc = binomial_warp(key, v, r.c, half, r.e[ks], tab, cl);
        if ((threadIdx.x & 31) == 0) {
            if (rc != RS_OK) {
                set_status(status, rc);
                cl = 0;
            }
            BoxRec L = r, R = r;
            L.e[ks] = half;
            L.c = cl;
            R.o[ks] = r.o[ks] + half;
            R.e[ks] = r.e[ks] - half;
            R.c = r.c - cl;
            R.off = r.off + cl;
            rec[2 * v] = L;
            rec[2 * v + 1] = R;
        }
    }
}

__global__ void box_leaf_recs_kernel(const BoxRec* __restrict__ leaves, uint64_t nleaves, uint32_t d,
                                     NodeRec* __restrict__ nr, unsigned long long* stats) {
    unsigned long long mv = 0, mc = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nleaves;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const BoxRec r = leaves[i];
        uint64_t vol = 1;
        for (uint32_t k = 0; k < d; ++k) vol *= r.e[k];
        nr[i] = NodeRec{0, vol, r.c, r.off};
        if (r.c > 0 && vol > mv) mv = vol;
        if (r.c > mc) mc = r.c;
    }
    for (int s = 16; s > 0; s >>= 1) {
        const unsigned long long a = __shfl_xor_sync(0xffffffffu, mv, s), b = __shfl_xor_sync(0xffffffffu, mc, s);
        mv = a > mv ? a : mv;
        mc = b > mc ? b : mc;
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&stats[0], mv);
        atomicMax(&stats[1], mc);
    }
}

// Division by an extent e that stays fixed over a leaf, for dividends below
// 2^62 (Granlund and Montgomery, "Division by invariant integers using
// multiplication", 1994, Thm. 4.2 with N = 62): with l = ceil(log2 e) and
// m = ceil(2^(62+l) / e) < 2^64, floor(x / e) = floor(x m / 2^(62+l)) =
// umulhi(x, m) >> (l - 2); powers of two by a shift.
struct InvariantDiv {
    uint64_t e, m;
    uint32_t shift;
    bool pow2;
    RS_DEV void init(uint64_t ext) {
        e = ext;
        pow2 = (ext & (ext - 1)) == 0;
        if (pow2) {
            shift = 63 - __clzll(ext);
            m = 0;
        } else {
            const uint32_t l = 64 - __clzll(ext - 1);
            m = (uint64_t)((((unsigned __int128)1 << (62 + l)) - 1) / ext) + 1;
            shift = l - 2;
        }
    }
    RS_DEV uint64_t quot(uint64_t x) const { return pow2 ? x >> shift : __umul64hi(x, m) >> shift; }
};

constexpr int kDecodeThreads = 256;
constexpr int kDecodeUnroll = 4;   // indices loaded per thread before any is decoded

// One block per leaf at a time: the leaf's points decoded by its threads,
// kDecodeUnroll loads in flight per thread; two-dimensional points as one
// 16-byte store where the output allows.
__global__ void __launch_bounds__(kDecodeThreads) box_decode_kernel(const BoxRec* __restrict__ leaves,
                                                                    uint64_t nleaves, uint32_t d,
                                                                    const uint64_t* __restrict__ idx,
                                                                    uint64_t* __restrict__ out) {
    __shared__ InvariantDiv div[kPointsMaxDim];
    const bool pair = d == 2 && ((uintptr_t)out & 15) == 0;
    for (uint64_t i = blockIdx.x; i < nleaves; i += gridDim.x) {
        const BoxRec r = leaves[i];
        if (r.c == 0) continue;
        if (threadIdx.x < d) div[threadIdx.x].init(r.e[threadIdx.x]);
        __syncthreads();
        const uint64_t c = r.c, off = r.off, o0 = r.o[0], o1 = r.o[1], e1 = r.e[1];
        for (uint64_t j0 = threadIdx.x; j0 < c; j0 += (uint64_t)kDecodeThreads * kDecodeUnroll) {
            uint64_t xs[kDecodeUnroll];
#pragma unroll
            for (int u = 0; u < kDecodeUnroll; ++u) {
                const uint64_t j = j0 + (uint64_t)u * kDecodeThreads;
                xs[u] = j < c ? idx[off + j] - 1 : 0;
            }
            if (pair) {
                const InvariantDiv dv = div[1];
#pragma unroll
                for (int u = 0; u < kDecodeUnroll; ++u) {
                    const uint64_t j = j0 + (uint64_t)u * kDecodeThreads;
                    if (j >= c) break;
                    const uint64_t q = dv.quot(xs[u]);
                    *reinterpret_cast<ulonglong2*>(out + (off + j) * 2) =
                        make_ulonglong2(o0 + q, o1 + (xs[u] - q * e1));
                }
                continue;
            }
#pragma unroll
            for (int u = 0; u < kDecodeUnroll; ++u) {
                const uint64_t j = j0 + (uint64_t)u * kDecodeThreads;
                if (j >= c) break;
                uint64_t x = xs[u];
                uint64_t* pt = out + (off + j) * d;
                for (uint32_t k = d - 1; k > 0; --k) {
                    const uint64_t q = div[k].quot(x);
                    pt[k] = r.o[k] + (x - q * r.e[k]);
                    x = q;
                }
                pt[0] = r.o[0] + x;
            }
        }
        __syncthreads();
    }
}

static unsigned grid_of(uint64_t items) {
    const uint64_t g = (items + kPointsThreads - 1) / kPointsThreads;
    return (unsigned)(g < 65535 ? (g ? g : 1) : 65535);
}

cudaError_t launch_points_tree(BoxRec* rec, uint32_t d, const BoxExtents& E, uint64_t n, uint64_t seed, int D,
                               const double* tab, int* status, cudaStream_t st) {
    box_root_kernel<<<1, 32, 0, st>>>(rec, d, E, n);
    const Key2 key = make_key(seed);
    for (int l = 0; l < D; ++l) {
        const uint64_t w = 1ull << l;
        if (w <= kPointsWarpNodes)
            box_level_warp_kernel<<<grid_of(32 * w), kPointsThreads, 0, st>>>(rec, w, d, key, tab, status);
        else
            box_level_kernel<<<grid_of(w), kPointsThreads, 0, st>>>(rec, w, d, key, tab, status);
    }
    return cudaGetLastError();
}

cudaError_t launch_points_leaf_recs(const BoxRec* leaves, uint64_t nleaves, uint32_t d, NodeRec* nr,
                                    unsigned long long* stats, cudaStream_t st) {
    box_leaf_recs_kernel<<<grid_of(nleaves), kPointsThreads, 0, st>>>(leaves, nleaves, d, nr, stats);
    return cudaGetLastError();
}

cudaError_t launch_points_decode(const BoxRec* leaves, uint64_t nleaves, uint32_t d, const uint64_t* idx,
                                 uint64_t* out, int sms, cudaStream_t st) {
    const uint64_t grid = std::min<uint64_t>(nleaves, (uint64_t)sms * 8);
    box_decode_kernel<<<(unsigned)(grid ? grid : 1), kDecodeThreads, 0, st>>>(leaves, nleaves, d, idx, out);
    return cudaGetLastError();
}

}  // namespace rs
