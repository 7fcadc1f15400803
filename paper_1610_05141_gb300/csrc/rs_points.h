// rs_points.h -- launchers of rs_points.cu used by the C ABI.
#pragma once
#include "rs_common.cuh"

namespace rs {

constexpr uint32_t kPointsMaxDim = 4;

// A box [o_k, o_k + e_k) in every dimension k < d holding c points, written
// at out[off .. off + c) (points, d coordinates each).
struct __align__(16) BoxRec {
    uint64_t o[kPointsMaxDim], e[kPointsMaxDim], c, off;
};

struct BoxExtents {
    uint64_t e[kPointsMaxDim];
};

// The bisection tree: box records 1 .. 2^(D+1)-1 of `rec`, level by level
// (root: the box [0, E) with n points; node v halves its largest extent,
// lowest index on ties, and its left child gets BIN(c, floor(e/2), e) of
// the points from stream (SPLIT, v)).  1 + D launches.
cudaError_t launch_points_tree(BoxRec* rec, uint32_t d, const BoxExtents& E, uint64_t n, uint64_t seed, int D,
                               const double* tab, int* status, cudaStream_t st);

// Leaf records for the with-replacement leaf kernel: nr[i] = {0, volume, c,
// off} of leaf box i; stats[0] = the largest volume of a leaf with points,
// stats[1] = the largest count (both must be zero before the launch).
cudaError_t launch_points_leaf_recs(const BoxRec* leaves, uint64_t nleaves, uint32_t d, NodeRec* nr,
                                    unsigned long long* stats, cudaStream_t st);

// out[(off + j) d + k] = the coordinates of the leaf's j-th index idx[off +
// j] - 1, row-major in the leaf box (dimension 0 most significant).
cudaError_t launch_points_decode(const BoxRec* leaves, uint64_t nleaves, uint32_t d, const uint64_t* idx,
                                 uint64_t* out, int sms, cudaStream_t st);

}  // namespace rs
