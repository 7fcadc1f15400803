// rs_common.cuh -- shared device/host definitions of the CUDA sampler.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/rs.h"

#define RS_DEV __device__ __forceinline__
#define RS_HD __host__ __device__ __forceinline__

namespace rs {

// Stream tags: one per kind of random decision (split deviates, leaf
// candidates, Algorithm B attempts, the repair step, Bernoulli chunks).
enum : uint32_t { TAG_SPLIT = 1, TAG_LEAF_H = 2, TAG_LEAF_B = 3, TAG_FIXUP = 4, TAG_BERN = 5, TAG_LEAF_WR = 6 };

// A split-tree node: the 0-based positions [lo, lo+S) hold c samples that
// are written at out[off .. off+c).  Heap numbering: root 1, children 2v, 2v+1.
struct __align__(16) NodeRec {
    uint64_t lo, S, c, off;
};

// The table the library's math reads (one per context, on the device):
// ln i! for i < 256 (kTabLf), then for the 128 mantissa intervals of [1, 2)
// the reciprocal of the interval's centre and minus its logarithm as a
// double-double (kTabInv, kTabHi, kTabLo); see rs_math.cuh.  Then, from
// double slot kTabF on, ln i! (i < 256) rounded to single precision, for
// the single-precision guard of the ratio-of-uniforms test.  Then, for the
// fixed-point logarithm of the guarded geometric skips (rs_math.cuh
// qnlog_u57), 512 intervals of [1, 2) with left ends c = 1 + i/512: inv =
// ceil(2^64 / c) (kTabQInv, an unsigned 64-bit word per slot) and -ln(inv
// 2^-64) in Q63 (kTabQLn).
constexpr int kTabLf = 0;
constexpr int kTabInv = 256;
constexpr int kTabHi = 384;
constexpr int kTabLo = 512;
constexpr int kTabF = 640;
constexpr int kQLogIntervals = 512;
constexpr int kTabQInv = 768;
constexpr int kTabQLn = kTabQInv + kQLogIntervals;
constexpr int kTabWords = kTabQLn + kQLogIntervals;

// First error wins; later errors are dropped until the host clears the word.
RS_DEV void set_status(int* status, int code) {
    if (code != RS_OK) atomicCAS(status, RS_OK, code);
}

RS_DEV uint64_t umulhi64(uint64_t a, uint64_t b) { return __umul64hi(a, b); }

// Iteration caps of the method's loops: ratio-of-uniforms trials and
// inversion restarts per deviate (Sec. 3.1), Philox blocks per candidate or
// skip stream, Algorithm B attempts per leaf (Sec. 2).  The defaults are
// the definition's; rs_set_iteration_caps lowers them so that tests can
// reach the RS_EITER paths.
struct IterCaps {
    uint64_t rou_trials;
    uint64_t inv_restarts;
    uint64_t stream_blocks;
    uint64_t b_attempts;
};
#define RS_DEFAULT_CAPS {1ull << 20, 64ull, 1ull << 32, 64ull}

// Device code is compiled per translation unit: every unit holds its own
// copy of the caps in constant memory and registers, when the library is
// loaded, a host function that writes that copy on the current device.
static __constant__ IterCaps c_caps = RS_DEFAULT_CAPS;
using CapsWriter = cudaError_t (*)(const IterCaps&);
int register_caps_writer(CapsWriter w);
static cudaError_t write_caps_here(const IterCaps& c) { return cudaMemcpyToSymbol(c_caps, &c, sizeof(IterCaps)); }
[[maybe_unused]] static const int caps_writer_registered = register_caps_writer(&write_caps_here);

}  // namespace rs
