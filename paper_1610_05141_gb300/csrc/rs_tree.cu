// rs_tree.cu -- the split tree (Sec. 3.1 Algorithm R, Sec. 3.2 Algorithm P).
//
// Node v covers the positions [lo, lo+S) and holds c samples.  Its left child
// 2v receives the first floor(S/2) positions and L samples, L drawn from the
// node's own SPLIT stream (hypergeometric, or binomial with replacement);
// the right child 2v+1 receives the rest.  Children also inherit the output
// offset (left: the parent's, right: parent's + L), so the leaves come out
// with their final write positions and no prefix sum is needed.  A node with
// no samples draws nothing.  Depth D is fixed in advance (as in Algorithm P's
// tree over PEs and the p' >> p jobs of Sec. 4.5), so the tree, and with it
// the sample, does not depend on how the work is scheduled.
#include "rs_deviates.cuh"
#include "rs_internal.h"

namespace rs {

__global__ void lf_table_kernel(double* tab) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    tab[0] = 0.0;
    tab[1] = 0.0;
    for (int i = 2; i < 256; ++i) tab[i] = tab[i - 1] + dlog((double)i);
}

cudaError_t launch_lf_table(double* tab, cudaStream_t st) {
    lf_table_kernel<<<1, 1, 0, st>>>(tab);
    return cudaGetLastError();
}

__global__ void tree_root_kernel(NodeRec* rec, uint64_t n, uint64_t N) {
    if (threadIdx.x == 0 && blockIdx.x == 0) rec[1] = NodeRec{0, N, n, 0};
}

template <bool WR>
__global__ void tree_level_kernel(NodeRec* __restrict__ rec, int level, uint64_t seed,
                                  const double* __restrict__ tab, int* status) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (1ull << level)) return;
    const uint64_t v = (1ull << level) + i;
    const NodeRec r = rec[v];
    const uint64_t K = r.S / 2;
    uint64_t L = 0;
    if (r.c > 0) {
        const Key2 key = make_key(seed);
        const int rc = WR ? binomial(key, v, r.c, K, r.S, tab, L) : hypergeometric(key, v, r.c, K, r.S, tab, L);
        if (rc != RS_OK) {
            set_status(status, rc);
            L = 0;
        }
    }
    rec[2 * v] = NodeRec{r.lo, K, L, r.off};
    rec[2 * v + 1] = NodeRec{r.lo + K, r.S - K, r.c - L, r.off + L};
}

cudaError_t launch_tree(NodeRec* rec, uint64_t n, uint64_t N, uint64_t seed, int D, bool with_replacement,
                        const double* tab, int* status, cudaStream_t st) {
    tree_root_kernel<<<1, 32, 0, st>>>(rec, n, N);
    for (int level = 0; level < D; ++level) {
        const uint64_t nodes = 1ull << level;
        const unsigned threads = nodes < 128 ? 32 : 128;
        const unsigned blocks = (unsigned)((nodes + threads - 1) / threads);
        if (with_replacement) tree_level_kernel<true><<<blocks, threads, 0, st>>>(rec, level, seed, tab, status);
        else tree_level_kernel<false><<<blocks, threads, 0, st>>>(rec, level, seed, tab, status);
    }
    return cudaGetLastError();
}

__global__ void export_leaves_kernel(const NodeRec* __restrict__ leaves, uint64_t nleaves, uint64_t* __restrict__ out) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nleaves; i += (uint64_t)gridDim.x * blockDim.x) {
        const NodeRec r = leaves[i];
        out[4 * i + 0] = r.lo;
        out[4 * i + 1] = r.S;
        out[4 * i + 2] = r.c;
        out[4 * i + 3] = r.off;
    }
}

cudaError_t launch_export_leaves(const NodeRec* leaves, uint64_t nleaves, uint64_t* recs_out, cudaStream_t st) {
    const unsigned blocks = (unsigned)std::min<uint64_t>((nleaves + 255) / 256, 4096);
    export_leaves_kernel<<<blocks, 256, 0, st>>>(leaves, nleaves, recs_out);
    return cudaGetLastError();
}

}  // namespace rs
