// rs_bern.h -- launchers of rs_bern.cu used by the C ABI beside those in
// rs_internal.h.
#pragma once
#include "rs_common.cuh"

namespace rs {

// One thread: *out = BIN(N, K / 2^62) of stream (SPLIT, 0) (N minus it when
// flip) -- the size of a Bernoulli sample drawn by its size (Sec. 4.7); a
// failed deviate sets the status word and gives 0.
cudaError_t launch_bernoulli_size(uint64_t seed, uint64_t N, uint64_t K, bool flip, const double* tab, uint64_t* out,
                                  int* status, cudaStream_t st);

}  // namespace rs
