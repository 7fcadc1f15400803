// rs_union.h -- launchers of rs_union.cu used by the C ABI.
#pragma once
#include "rs_common.cuh"

namespace rs {

// Samples per segment of a sample of n from the union of p segments of sizes
// L[0..p) (Sec. 4.3): node sums of the binary tree over the segments padded
// to P = 2^log2P (heap numbering, root 1, segment i at node P + i) are added
// bottom-up into sum[1 .. 2P), then, top-down, node v's cnt[v] samples split
// into HG(cnt[v], sum[2v], sum[v]) of stream (SPLIT, v) for its left child
// and the rest for its right child.  Segment i's count ends in cnt[P + i].
// sum and cnt: 2P words of device memory each; L: p words on the device.
// A failed deviate sets the status word.  1 + 2 log2P launches.
cudaError_t launch_union_counts(const uint64_t* L, uint32_t p, int log2P, uint64_t n, uint64_t seed, uint64_t* sum,
                                uint64_t* cnt, const double* tab, int* status, cudaStream_t st);

}  // namespace rs
