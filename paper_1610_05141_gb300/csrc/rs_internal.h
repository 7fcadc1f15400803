// rs_internal.h -- host-side interfaces between the library's translation units.
#pragma once
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "rs_common.cuh"

namespace rs {

// Largest leaf selection of the shared-memory table of leaf H / leaf WR.
constexpr uint32_t kLeafFastCap = 4864;
// 64-bit keys: a table with room for 4,096 values fits three 256-thread
// blocks per SM instead of two (about 10 % faster leaves on GB300); leaves
// averaging at most 3,600 values take it (4,096 lies more than eight
// standard deviations of their counts above that mean).
constexpr uint32_t kCompact64Cap = 4096;
constexpr uint64_t kCompact64Mean = 3600;
// Largest selection the general (global-memory) leaf path accepts.
constexpr uint64_t kBigLeafMax = 1ull << 22;
// Deepest split tree the library builds (2^27 node records of 32 bytes).
constexpr int kMaxDepth = 26;

// Split-tree depth of (n, N, n0): the least D >= 0 with n <= n0 2^D, then
// lowered until 2^D <= N (Algorithm P's fixed tree, Sec. 3.2 and Sec. 4.5).
int tree_depth(uint64_t n, uint64_t N, uint32_t n0);

// Builds the ln i! table (i < 256) on the device with the library's own log.
cudaError_t launch_lf_table(double* tab, cudaStream_t st);

// Split tree: writes node records 1 .. 2^(D+1)-1 of `rec` level by level;
// the leaves are rec[2^D .. 2^(D+1)).  with_replacement selects binomial
// splits, else hypergeometric ones.  guard = false evaluates every
// ratio-of-uniforms test in FP64 (same output; the single-precision guard
// of rs_math.cuh otherwise decides the trials far from the boundary).
cudaError_t launch_tree(NodeRec* rec, uint64_t n, uint64_t N, uint64_t seed, int D, bool with_replacement,
                        const double* tab, int* status, cudaStream_t st, bool guard = true);
// The root and levels 0 .. levels-1.
cudaError_t launch_tree_top(NodeRec* rec, uint64_t n, uint64_t N, uint64_t seed, int levels, bool with_replacement,
                            const double* tab, int* status, cudaStream_t st, bool guard = true);
// Levels c .. D-1 of the subtree under node 2^c + part (its nodes on level l
// are 2^l + part 2^(l-c) .. + 2^(l-c) - 1); levels 0 .. c-1 must be done.
cudaError_t launch_tree_part(NodeRec* rec, uint64_t seed, int D, int c, uint64_t part, bool with_replacement,
                             const double* tab, int* status, cudaStream_t st, bool guard = true);

// Copies leaf records rec[2^D + i] to recs_out[4i .. 4i+3].
cudaError_t launch_export_leaves(const NodeRec* leaves, uint64_t nleaves, uint64_t* recs_out, cudaStream_t st);

struct LeafLaunch {
    const NodeRec* leaves;   // 2^D leaf records
    uint64_t nleaves;
    uint64_t first_id;       // heap id of leaf 0
    uint64_t seed;
    uint64_t smax;           // largest leaf size
    uint64_t* out;
    int* status;
    uint32_t* ovf_list;      // nleaves entries
    uint32_t* ovf_count;
    void* big_pool;          // scratch of big_pool_bytes(big_kmax) bytes, or null when big_kmax = 0
    uint64_t big_kmax;
    uint32_t cap;            // testing knob: largest selection of the shared-memory paths, 0 = the kernel's
    int sms;
    bool with_replacement;
    int blocks_per_sm = 0;   // leaf-kernel blocks per SM, 0 = as many as fit
    uint64_t mean_count = 0; // samples per leaf on average (picks the kernel's shape)
    bool pow2_leaves = false; // every leaf has the size smax, a power of two
};

// Leaf H (or leaf WR) for every leaf, then the general path for the leaves
// whose selection exceeded the capacity.
cudaError_t launch_leaves(const LeafLaunch& L, cudaStream_t st);
uint64_t big_pool_bytes(uint64_t kmax);

struct LeafBLaunch {
    const NodeRec* leaves;
    uint64_t nleaves;
    uint64_t first_id;
    uint64_t seed;
    uint64_t* out;
    int* status;
    int sms;
    const double* tab;       // the context's table (its logarithm)
    uint64_t smax;           // largest leaf size (32-bit positions up to 2^32)
    bool guard = true;       // skips decided in fixed and single precision where safe
};
// Algorithm B leaves (positions of one attempt live in shared memory).
cudaError_t launch_leaves_b(const LeafBLaunch& L, cudaStream_t st);

struct BernLaunch {
    double p;
    uint64_t N;
    uint64_t seed;
    int chunk_log2;
    uint64_t chunk_first;    // first chunk of the window
    uint64_t nchunks;        // chunks in the window
    uint64_t a, b;           // window of 0-based positions
    uint64_t* out;
    uint64_t cap;
    uint64_t* counts;        // nchunks + 1 words of scratch
    uint64_t* total;         // device word: number of positions in the window
    uint64_t* scan_scratch;  // scan_scratch_words(nchunks) words
    int* status;
    int sms;
    const double* tab;       // the context's table (its logarithm)
    uint64_t* stage;         // nchunks * stage_per words, or null
    uint64_t stage_per;      // staged positions per chunk
    bool guard = true;       // skips decided in fixed and single precision where safe
};
// With staging: one walk per chunk (positions staged, counted), exclusive
// scan of the counts, copy to the output (a chunk above stage_per positions
// walks again).  Without: count pass, scan, write pass.
cudaError_t launch_bernoulli(const BernLaunch& L, cudaStream_t st);
uint64_t scan_scratch_words(uint64_t n);
// Staged positions per chunk for an expected count mu: mu + 8 sqrt(mu) + 64,
// a multiple of 4.
uint64_t bern_stage_per(double mu);

struct BatchGroupView;
struct QueryBoundView;
struct QueryInnerView;
// Algorithm B leaves of a batch group, or of range queries (rs_bern.cu).
cudaError_t launch_batch_leaves_b(const BatchGroupView& G, const double* tab, int sms, cudaStream_t st);
cudaError_t launch_batch_leaves_b(const QueryBoundView& G, const double* tab, int sms, cudaStream_t st);
cudaError_t launch_batch_leaves_b(const QueryInnerView& G, const double* tab, int sms, cudaStream_t st);

}  // namespace rs
