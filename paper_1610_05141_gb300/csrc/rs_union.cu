// rs_union.cu -- sample counts of the segments of a union (Sec. 4.3, uneven
// distribution of the universe over its owners).
//
// The paper's owners learn their share of the sample from a tree of
// hypergeometric splits over the owners, then sample their own elements
// alone.  Here the owners are segments of one universe; the tree is the
// binary tree of power-of-two aligned groups of segments, one launch per
// level, one warp per node on narrow levels and one thread per node on wide
// ones.  The per-segment samples are the batch
// engine's (rs_batch.cu), each segment a request with its own key.
#include "rs_deviates.cuh"
#include "rs_union.h"

namespace rs {

constexpr int kUnionThreads = 128;
// Levels of at most this many nodes take one warp per node.
constexpr uint64_t kUnionWarpNodes = 1024;

__global__ void union_init_kernel(const uint64_t* __restrict__ L, uint32_t p, uint64_t P, uint64_t n,
                                  uint64_t* __restrict__ sum, uint64_t* __restrict__ cnt) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (uint64_t)gridDim.x * blockDim.x)
        sum[P + i] = i < p ? L[i] : 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) cnt[1] = n;
}

// Nodes [w, 2w): sum of the two children.
__global__ void union_sum_level_kernel(uint64_t* sum, uint64_t w) {
    for (uint64_t v = w + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < 2 * w;
         v += (uint64_t)gridDim.x * blockDim.x)
        sum[v] = sum[2 * v] + sum[2 * v + 1];
}

// Nodes [w, 2w): the left child's share of the node's samples.
__global__ void __launch_bounds__(kUnionThreads) union_split_level_kernel(const uint64_t* __restrict__ sum,
                                                                          uint64_t* cnt, uint64_t w, Key2 key,
                                                                          const double* __restrict__ tab,
                                                                          int* status) {
    for (uint64_t v = w + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < 2 * w;
         v += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t c = cnt[v];
        uint64_t left = 0;
        const int rc = hypergeometric(key, v, c, sum[2 * v], sum[v], tab, left);
        if (rc != RS_OK) {
            set_status(status, rc);
            left = 0;
        }
        cnt[2 * v] = left;
        cnt[2 * v + 1] = c - left;
    }
}

// The same for narrow levels: one warp per node, the deviate's trials spread
// over the warp's lanes (lower latency when the level has few nodes).
__global__ void __launch_bounds__(kUnionThreads) union_split_warp_kernel(const uint64_t* __restrict__ sum,
                                                                         uint64_t* cnt, uint64_t w, Key2 key,
                                                                         const double* __restrict__ tab,
                                                                         int* status) {
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
    for (uint64_t v = w + (uint64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; v < 2 * w; v += warps) {
        const uint64_t c = cnt[v];
        uint64_t left = 0;
        const int rc = hypergeometric_warp(key, v, c, sum[2 * v], sum[v], tab, left);
        if ((threadIdx.x & 31) == 0) {
            if (rc != RS_OK) {
                set_status(status, rc);
                left = 0;
            }
            cnt[2 * v] = left;
            cnt[2 * v + 1] = c - left;
        }
    }
}

static unsigned grid_for(uint64_t items) {
    const uint64_t g = (items + kUnionThreads - 1) / kUnionThreads;
    return (unsigned)(g < 65535 ? (g ? g : 1) : 65535);
}

cudaError_t launch_union_counts(const uint64_t* L, uint32_t p, int log2P, uint64_t n, uint64_t seed, uint64_t* sum,
                                uint64_t* cnt, const double* tab, int* status, cudaStream_t st) {
    const uint64_t P = 1ull << log2P;
    union_init_kernel<<<grid_for(P), kUnionThreads, 0, st>>>(L, p, P, n, sum, cnt);
    for (int l = log2P - 1; l >= 0; --l)
        union_sum_level_kernel<<<grid_for(1ull << l), kUnionThreads, 0, st>>>(sum, 1ull << l);
    const Key2 key = make_key(seed);
    for (int l = 0; l < log2P; ++l) {
        const uint64_t w = 1ull << l;
        if (w <= kUnionWarpNodes)
            union_split_warp_kernel<<<grid_for(32 * w), kUnionThreads, 0, st>>>(sum, cnt, w, key, tab, status);
        else
            union_split_level_kernel<<<grid_for(w), kUnionThreads, 0, st>>>(sum, cnt, w, key, tab, status);
    }
    return cudaGetLastError();
}

}  // namespace rs
