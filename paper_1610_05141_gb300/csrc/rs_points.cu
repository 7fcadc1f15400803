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

// One block per leaf at a time: the leaf's points decoded by its threads.
__global__ void __launch_bounds__(256) box_decode_kernel(const BoxRec* __restrict__ leaves, uint64_t nleaves,
                                                         uint32_t d, const uint64_t* __restrict__ idx,
                                                         uint64_t* __restrict__ out) {
    for (uint64_t i = blockIdx.x; i < nleaves; i += gridDim.x) {
        const BoxRec r = leaves[i];
        for (uint64_t j = threadIdx.x; j < r.c; j += blockDim.x) {
            uint64_t x = idx[r.off + j] - 1;
            uint64_t* pt = out + (r.off + j) * d;
            for (uint32_t k = d - 1; k > 0; --k) {
                const uint64_t q = x / r.e[k];
                pt[k] = r.o[k] + (x - q * r.e[k]);
                x = q;
            }
            pt[0] = r.o[0] + x;
        }
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
    for (int l = 0; l < D; ++l)
        box_level_kernel<<<grid_of(1ull << l), kPointsThreads, 0, st>>>(rec, 1ull << l, d, key, tab, status);
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
    box_decode_kernel<<<(unsigned)(grid ? grid : 1), 256, 0, st>>>(leaves, nleaves, d, idx, out);
    return cudaGetLastError();
}

}  // namespace rs
