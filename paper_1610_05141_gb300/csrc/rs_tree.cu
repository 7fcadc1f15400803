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
#include <cooperative_groups.h>

#include "rs_internal.h"
#include "rs_tree_warp.cuh"

namespace rs {

// The context's table: first the logarithm's 128 entries and the 512 of
// the fixed-point logarithm (one thread each), then, in a second launch
// (the logarithm reads its entries through the read-only cache), ln i! for
// i < 256.
__global__ void log_table_kernel(double* tab) {
    if (blockIdx.x == 0 && threadIdx.x < 128) build_log_entry((int)threadIdx.x, tab);
    if (blockIdx.x == 0 && threadIdx.x < kQLogIntervals) build_qlog_entry((int)threadIdx.x, tab);
}

__global__ void lf_table_kernel(double* tab) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    tab[kTabLf + 0] = 0.0;
    tab[kTabLf + 1] = 0.0;
    for (int i = 2; i < 256; ++i) tab[kTabLf + i] = tab[kTabLf + i - 1] + dlog((double)i, tab);
    float* tf = reinterpret_cast<float*>(tab + kTabF);
    for (int i = 0; i < 256; ++i) tf[i] = __double2float_rn(tab[kTabLf + i]);
}

cudaError_t launch_lf_table(double* tab, cudaStream_t st) {
    log_table_kernel<<<1, kQLogIntervals, 0, st>>>(tab);
    lf_table_kernel<<<1, 1, 0, st>>>(tab);
    return cudaGetLastError();
}

__global__ void tree_root_kernel(NodeRec* rec, uint64_t n, uint64_t N) {
    if (threadIdx.x == 0 && blockIdx.x == 0) rec[1] = NodeRec{0, N, n, 0};
}

constexpr int kTreeWarps = 4;            // warps per block of the level kernel
constexpr uint32_t kTreeBatch = 128;     // nodes per warp (lanes refill from it)

// Nodes first .. first+nodes-1 of one level: each warp takes a batch of
// consecutive nodes, G lanes per node.
template <bool WR>
__global__ void __launch_bounds__(kTreeWarps * 32) tree_level_kernel(NodeRec* __restrict__ rec, uint64_t first,
                                                                    uint64_t nodes, uint32_t batch, uint32_t G,
                                                                    uint64_t seed, const double* __restrict__ tab,
                                                                    int* status, bool guard) {
    extern __shared__ double tree_logs[];
    const uint32_t warp = threadIdx.x >> 5;
    const uint64_t start = ((uint64_t)blockIdx.x * kTreeWarps + warp) * batch;
    if (start >= nodes) return;
    const uint64_t left = nodes - start;
    const uint32_t count = left < batch ? (uint32_t)left : batch;
    tree_batch_warp<WR>(rec, first + start, count, make_key(seed), tab, status,
                        tree_logs + warp * 32 * kLogSlots, G, guard);
}

// Nodes of a small launch: G >= 4 lanes per node, parallel terms and trials;
// a warp takes `batch` nodes (a multiple of 32 / G), its groups refilling.
template <bool WR>
__global__ void __launch_bounds__(kTreeWarps * 32) tree_terms_kernel(NodeRec* __restrict__ rec, uint64_t first,
                                                                    uint64_t nodes, uint32_t batch, uint32_t G,
                                                                    uint64_t seed, const double* __restrict__ tab,
                                                                    int* status, bool guard) {
    const uint32_t warp = threadIdx.x >> 5;
    const uint64_t start = ((uint64_t)blockIdx.x * kTreeWarps + warp) * batch;
    if (start >= nodes) return;
    const uint64_t left = nodes - start;
    const uint32_t count = left < batch ? (uint32_t)left : batch;
    tree_terms_warp<WR>(rec, first + start, count, make_key(seed), tab, status, G, guard);
}

// The root and the top `levels` levels in one cooperative launch (one block
// of kTreeWarps warps per SM, all resident): level l's 2^l nodes are spread
// over the grid's warps, a group of G lanes per node running trials in
// parallel, and the grid synchronizes between levels.  These levels hold few
// nodes each, so their time is the latency of one node's chain of FP64
// operations; one launch instead of one per level saves the launches and
// the cold start of each.
constexpr int kTopFused = 12;   // levels of the fused launch, at most

template <bool WR>
__global__ void __launch_bounds__(kTreeWarps * 32) tree_top_kernel(NodeRec* __restrict__ rec, uint64_t n, uint64_t N,
                                                                  int levels, uint64_t seed,
                                                                  const double* __restrict__ tab, int* status,
                                                                  bool guard) {
    namespace cg = cooperative_groups;
    cg::grid_group grid = cg::this_grid();
    if (blockIdx.x == 0 && threadIdx.x == 0) rec[1] = NodeRec{0, N, n, 0};
    grid.sync();
    const uint64_t W = (uint64_t)gridDim.x * kTreeWarps;
    const uint64_t w = (uint64_t)blockIdx.x * kTreeWarps + (threadIdx.x >> 5);
    for (int level = 0; level < levels; ++level) {
        const uint64_t nodes = 1ull << level;
        uint32_t G = 32;
        while (G > 4 && nodes * G > W * 32) G >>= 1;
        const uint64_t groups = 32 / G;   // nodes a warp holds at once
        const uint64_t per = groups * ((nodes + W * groups - 1) / (W * groups));
        const uint64_t start = w * per;
        if (start < nodes)
            tree_terms_warp<WR>(rec, nodes + start, (uint32_t)min(per, nodes - start), make_key(seed), tab, status, G,
                                guard);
        grid.sync();
    }
}

// The last `levels` levels below level L0 in one launch: warp t takes the
// subtree under node 2^L0 + t and splits its nodes level by level (its
// level-j nodes (2^L0 + t) 2^j .. + 2^j - 1 read the records its own
// earlier level wrote; __syncwarp orders them).  A level of 32 nodes or
// more runs a node per lane, a smaller one four lanes per node (one trial
// at a time, its four terms side by side).  No launch or grid-wide wait
// between these levels: each subtree runs at the latency of its own chain,
// and the other subtrees keep the SMs busy meanwhile.  Measured on GB300 at
// depth 18 (tree ms): 0.413 with a launch per level; subtrees of 4, 5 and
// 6 levels 0.456, 0.396 and 0.494; at most 128 registers (four blocks per
// SM) 0.366 for 5 levels, and with four lanes per node on the small levels
// (instead of 32 / nodes) 0.343.
constexpr int kSubtreeLevels = 5;   // levels of the subtree launch, at most

template <bool WR>
__global__ void __launch_bounds__(kTreeWarps * 32, 4) tree_subtree_kernel(NodeRec* __restrict__ rec, int L0, int levels,
                                                                      uint64_t seed, const double* __restrict__ tab,
                                                                      int* status, bool guard) {
    extern __shared__ double tree_logs[];
    const uint32_t warp = threadIdx.x >> 5;
    const uint64_t t = (uint64_t)blockIdx.x * kTreeWarps + warp;
    if (t >= (1ull << L0)) return;
    const uint64_t u = (1ull << L0) + t;
    const Key2 key = make_key(seed);
    for (int j = 0; j < levels; ++j) {
        const uint32_t count = 1u << j;
        if (count >= 32)
            tree_batch_warp<WR>(rec, u << j, count, key, tab, status, tree_logs + warp * 32 * kLogSlots, 1, guard);
        else
            tree_terms_warp<WR>(rec, u << j, count, key, tab, status, 4u, guard);
        __syncwarp();
    }
}

// Lanes per node for a launch of `nodes` nodes: the largest power of two up
// to 32 that keeps nodes * G within about four warps per SM, and at least 4
// (four lanes share a trial) up to 512 nodes per SM.  G >= 4: parallel
// terms and trials; G = 1: a node per lane with refill, which does the
// least FP64 work per trial and wins once a launch has more nodes than that.
uint32_t lanes_per_node(uint64_t nodes, int sms) {
    const uint64_t target = (uint64_t)sms * 4 * 32;
    uint32_t G = 1;
    while (G < 32 && nodes * G * 2 <= target) G *= 2;
    if (G < 4) G = nodes <= (uint64_t)sms * 512 ? 4 : 1;
    return G;
}

static int device_sms() {
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

// Splits nodes first .. first+nodes-1 (all on one level, parents done).
static void launch_nodes(NodeRec* rec, uint64_t first, uint64_t nodes, uint64_t seed, bool wr, const double* tab,
                         int* status, int sms, cudaStream_t st, bool guard) {
    const size_t smem = (size_t)kTreeWarps * 32 * kLogSlots * sizeof(double);
    // small launches: a group of G lanes per node runs trials in parallel;
    // then one node per lane until there are enough warps for every SM;
    // beyond that, batches grow (up to kTreeBatch) and lanes refill
    const uint32_t G = lanes_per_node(nodes, sms);
    uint32_t batch;
    if (G > 1) {
        // groups refill from batches of up to eight nodes per group while
        // that leaves about six warps per SM (measured best on GB300: the
        // longer the batch, the less the last nodes' trials idle the warp)
        const uint64_t per_sm = nodes * G / ((uint64_t)sms * 6 * 32);
        batch = (32 / G) * (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(8, per_sm));
    } else {
        uint64_t per = nodes / ((uint64_t)sms * kTreeWarps);   // one block per SM before the cap
        per = std::max<uint64_t>(32, std::min<uint64_t>(kTreeBatch, per & ~31ull));
        batch = (uint32_t)std::min<uint64_t>(per, nodes);
    }
    const uint64_t warps = (nodes + batch - 1) / batch;
    const unsigned blocks = (unsigned)((warps + kTreeWarps - 1) / kTreeWarps);
    if (G >= 4) {
        if (wr) tree_terms_kernel<true><<<blocks, kTreeWarps * 32, 0, st>>>(rec, first, nodes, batch, G, seed, tab, status, guard);
        else tree_terms_kernel<false><<<blocks, kTreeWarps * 32, 0, st>>>(rec, first, nodes, batch, G, seed, tab, status, guard);
    } else if (wr) {
        tree_level_kernel<true><<<blocks, kTreeWarps * 32, smem, st>>>(rec, first, nodes, batch, G, seed, tab, status, guard);
    } else {
        tree_level_kernel<false><<<blocks, kTreeWarps * 32, smem, st>>>(rec, first, nodes, batch, G, seed, tab, status, guard);
    }
}

cudaError_t launch_tree(NodeRec* rec, uint64_t n, uint64_t N, uint64_t seed, int D, bool with_replacement,
                        const double* tab, int* status, cudaStream_t st, bool guard) {
    return launch_tree_top(rec, n, N, seed, D, with_replacement, tab, status, st, guard);
}

// Whether the device takes cooperative launches of the fused top kernel
// (one block per SM).
static bool top_fusable() {
    int dev = 0, coop = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return false;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tree_top_kernel<false>, kTreeWarps * 32, 0) !=
            cudaSuccess || per_sm < 1)
        return false;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tree_top_kernel<true>, kTreeWarps * 32, 0) !=
            cudaSuccess || per_sm < 1)
        return false;
    return true;
}

cudaError_t launch_tree_top(NodeRec* rec, uint64_t n, uint64_t N, uint64_t seed, int levels, bool with_replacement,
                            const double* tab, int* status, cudaStream_t st, bool guard) {
    const int sms = device_sms();
    static const bool fusable = top_fusable();
    int level = 0;
    if (fusable && levels > 1) {
        int fused = levels < kTopFused ? levels : kTopFused;
        void* args[] = {&rec, &n, &N, &fused, &seed, &tab, &status, &guard};
        const void* kern = with_replacement ? (const void*)tree_top_kernel<true> : (const void*)tree_top_kernel<false>;
        const cudaError_t e = cudaLaunchCooperativeKernel(kern, dim3(sms), dim3(kTreeWarps * 32), args, 0, st);
        if (e != cudaSuccess) return e;
        level = fused;
    } else {
        tree_root_kernel<<<1, 32, 0, st>>>(rec, n, N);
    }
    // the last levels (at most kSubtreeLevels) as subtrees of one warp each
    const int L0 = levels - level >= 2 ? std::max(level, levels - kSubtreeLevels) : levels;
    for (; level < L0; ++level)
        launch_nodes(rec, 1ull << level, 1ull << level, seed, with_replacement, tab, status, sms, st, guard);
    if (L0 < levels) {
        const size_t smem = (size_t)kTreeWarps * 32 * kLogSlots * sizeof(double);
        const unsigned blocks = (unsigned)(((1ull << L0) + kTreeWarps - 1) / kTreeWarps);
        const int sub = levels - L0;
        if (with_replacement)
            tree_subtree_kernel<true><<<blocks, kTreeWarps * 32, smem, st>>>(rec, L0, sub, seed, tab, status, guard);
        else
            tree_subtree_kernel<false><<<blocks, kTreeWarps * 32, smem, st>>>(rec, L0, sub, seed, tab, status, guard);
    }
    return cudaGetLastError();
}

uint64_t tree_launches(int levels) {
    static const bool fusable = top_fusable();
    // one fused launch for the top levels, or the root kernel; then as launch_tree_top
    const int level = (fusable && levels > 1) ? std::min(levels, kTopFused) : 0;
    const int L0 = levels - level >= 2 ? std::max(level, levels - kSubtreeLevels) : levels;
    return 1 + (uint64_t)(L0 - level) + (L0 < levels ? 1 : 0);
}

cudaError_t launch_tree_part(NodeRec* rec, uint64_t seed, int D, int c, uint64_t part, bool with_replacement,
                             const double* tab, int* status, cudaStream_t st, bool guard) {
    const int sms = device_sms();
    for (int level = c; level < D; ++level) {
        const uint64_t per = 1ull << (level - c);
        launch_nodes(rec, (1ull << level) + part * per, per, seed, with_replacement, tab, status, sms, st, guard);
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
