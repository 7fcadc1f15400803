// rs_bern.cu -- Bernoulli sampling by independent chunks (Sec. 4.7) and
// Algorithm B as the base case of the split tree (Sec. 2, Sec. 4.7).
//
// Geometric skips: with L = ln(1-p) and U uniform in (0,1], the skip
// floor(ln U / L) is Geometric(p), so a Bernoulli(p) sample of a range is the
// running sum of (skip + 1) while it stays inside the range (Sec. 2,
// Algorithm B).  The quotient is taken as ln U times R = RN(1/L), one
// division per range instead of one per draw (U = 1 gives skip 0 even where
// R overflows).  Draw j of a stream gives one skip.  A warp (Bernoulli
// chunks) or a block (leaf B) takes 32 or 512 consecutive draws at once and
// turns them into positions with an integer prefix sum, which is exact, so
// the positions are those of the sequential definition.  A draw with
// ln U / L >= 2^62 ends the range.
#include "rs_batch.cuh"
#include "rs_bern.h"
#include "rs_deviates.cuh"
#include "rs_hash_leaf.cuh"
#include "rs_math.cuh"

namespace rs {

constexpr uint64_t kSat = 1ull << 63;   // saturation of skip sums
constexpr double kTwo62 = 4611686018427387904.0;

RS_DEV uint64_t sat_add(uint64_t a, uint64_t b) { return a > kSat - b ? kSat : a + b; }

// Skip + 1 for one draw, or 0 with *stop when the draw ends the range.  The
// value is clamped to cmax, which exceeds every range length, so clamping
// never changes a decision.
RS_DEV uint64_t step_of(double q, uint64_t cmax, bool* stop) {
    *stop = !(q < kTwo62);
    if (*stop) return 0;
    const uint64_t f = (uint64_t)floor(q) + 1;
    return f < cmax ? f : cmax;
}

// q = ln U * R for the draw with 64-bit value x (U = u_open(x)); U = 1
// (the top 53 bits of x all ones) gives 0.
RS_DEV double skip_quotient(uint64_t x, double R, const double* __restrict__ tab) {
    if ((x >> 11) == (1ull << 53) - 1) return 0.0;
    return dlog(u_open(x), tab) * R;
}

// The skip of one draw decided without FP64 where that is safe.  The
// definition floors q64 = RN(dlog(U) R) (skip_quotient); here, with
// A = qnlog_u57(m) (U = m 2^-53, |A 2^-57 - |ln U|| <= 2^-55):
// - Lh + Lm = A 2^-57 (1 - tau), 0 <= tau < 2^-46: the top 47 of A's 63
//   bits as two exact singles, made from their bits;
// - rh + rl = |R| (1 + rho), |rho| <= 2^-48;
// - p = RN(Lh rh) and e = fma(Lh, rh, -p) + (Lh rl + Lm rh), whose roundings
//   stay below 2^-45 p; the dropped Lm rl is below 2^-48 p; so
//   |p + e - |ln U| |R|| <= |R| 2^-55 + p 2^-44.2;
// - dlog is within 2 ulp of ln U and the product is rounded once, so
//   |q64 - |ln U| |R|| <= 2^-50.6 q64;
// - r = RN((p - floor(p)) + e), p - floor(p) exact, rounds by 2^-24 |r|.
// Hence |floor(p) + r - q64| <= b / 2 for b = (|r| + 1) 2^-23 + p 2^-43 +
// |R| 2^-54, and when floor(r - b) = floor(r + b) (rounded outward) that is
// floor(q64 - floor(p)).  Otherwise, or for p >= 2^44 (skips that long
// need p below about 1e-12), the draw takes the FP64 definition.  The skips,
// and so the sample, are the definition's in every case.  No conversion
// instruction is used (they run on the slow FP64 pipe of this GPU): the
// singles are assembled from bits, and floors of x with |x| < 2^22 are
// (x + 1.5 2^23) - 1.5 2^23 with the sum rounded down.
struct SkipParams {
    double R;        // RN(1 / ln(1 - p)), negative
    float rh, rl;    // |R| as an unevaluated sum of two singles
    float rb;        // |R| 2^-54, rounded up
    bool fast;       // the single-precision decision may be taken
};

RS_DEV SkipParams skip_params(double R, bool guard) {
    SkipParams s;
    s.R = R;
    const double a = -R;
    s.fast = guard && a > 0.0 && a < 1e30;   // huge or infinite |R| (p near 0) takes FP64 only
    s.rh = __double2float_rn(s.fast ? a : 0.0);
    s.rl = __double2float_rn(s.fast ? a - (double)s.rh : 0.0);
    s.rb = __double2float_ru(s.fast ? a * 0x1p-54 : 0.0);
    return s;
}

// An integer-valued single in [0, 2^63) as a 64-bit integer, from its bits
// (the 64-bit conversion instructions would run on the FP64 pipe).
RS_DEV uint64_t f2u64_exact(float f) {
    const uint32_t b = __float_as_uint(f);
    const int e = (int)(b >> 23) - 127;
    if (e < 0) return 0;
    const uint64_t m = (b & 0x7FFFFFu) | 0x800000u;
    return e >= 23 ? m << (e - 23) : m >> (23 - e);
}

// Skip + 1 of the draw with 64-bit value x; false if it must take FP64.
RS_DEV bool skip_fast(uint64_t x, const SkipParams& sp, const double* __restrict__ tab, uint64_t* step) {
    const uint64_t m = (x >> 11) + 1;
    if (m == (1ull << 53)) {   // U = 1: skip 0, as in skip_quotient
        *step = 1;
        return true;
    }
    const int64_t A = qnlog_u57(m, tab);   // below 2^62.2 (|ln U| <= 53 ln 2)
    if (A <= 0) return false;
    const int lz = __clzll(A);
    const uint64_t nn = (uint64_t)A << lz;   // A 2^lz, top bit set: A 2^-57 = nn 2^(-57-lz)
    // Lh = bits 40..63 of nn times 2^(-17-lz): exponent field 127 + (6 - lz)
    const float Lh = __int_as_float(((133 - lz) << 23) | ((uint32_t)(nn >> 40) & 0x7FFFFFu));
    // Lm = bits 17..39 times 2^(-40-lz): 2^E (1 + f 2^-23) - 2^E, E = -17 - lz
    const float Lm = __int_as_float(((110 - lz) << 23) | ((uint32_t)(nn >> 17) & 0x7FFFFFu)) -
                     __int_as_float((110 - lz) << 23);
    const float p = Lh * sp.rh;
    const float e = __fmaf_rn(Lh, sp.rh, -p) + (Lh * sp.rl + Lm * sp.rh);
    if (!(p < 0x1p44f)) return false;
    const float fl = p < 0x1p23f ? __fadd_rd(p, 0x1p23f) - 0x1p23f : p;   // floor(p)
    const float r = (p - fl) + e;   // |r| < 2^21 + 1
    const float b = (fabsf(r) + 1.0f) * 0x1p-23f + p * 0x1p-43f + sp.rb;
    constexpr float kM = 12582912.0f;   // 1.5 2^23
    const float klo = __fadd_rd(__fadd_rd(r, -b), kM) - kM;   // floor(r - b)
    if (klo != __fadd_rd(__fadd_ru(r, b), kM) - kM) return false;
    const uint64_t k = klo < 0.0f ? 0 - f2u64_exact(-klo) : f2u64_exact(klo);   // mod 2^64
    *step = f2u64_exact(fl) + k + 1;
    return true;
}

// The FP64 definition of one draw's step, a call of its own so that the
// compiler cannot evaluate it, predicated off, for every draw: skip + 1
// clamped to cmax, or ~0 for a draw that ends the range.
__device__ __noinline__ uint64_t draw_step_fp64(uint64_t x, double R, uint64_t cmax, const double* __restrict__ tab) {
    bool stop;
    const uint64_t s = step_of(skip_quotient(x, R, tab), cmax, &stop);
    return stop ? ~0ull : s;
}

// Skip + 1 of one draw (or 0 with *stop), by skip_fast where it decides.
RS_DEV uint64_t draw_step(uint64_t x, const SkipParams& sp, uint64_t cmax, bool* stop,
                          const double* __restrict__ tab) {
    uint64_t s;
    if (sp.fast && skip_fast(x, sp, tab, &s)) {
        *stop = false;
        return s < cmax ? s : cmax;
    }
    s = draw_step_fp64(x, sp.R, cmax, tab);
    *stop = s == ~0ull;
    return *stop ? 0 : s;
}

RS_DEV uint64_t warp_inclusive_sat(uint64_t x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x = sat_add(x, y);
    }
    return x;
}

// The draws a lane (or a thread) takes per round of a walk: V consecutive
// draws from V/2 Philox blocks (block b gives draws 2b and 2b + 1, as in
// stream_value), so that no block is computed twice and a round's scan is
// shared by V draws.
constexpr int kWalkV = 4;

// Steps of draws j0 .. j0 + V - 1 (j0 even): step[q] (0 for a draw that
// ends the range), bit q of *endm set for a draw that ends the range or lies
// past the stream, bit q of *exhm for a draw past the stream.
template <int V>
RS_DEV void draw_steps(Key2 key, uint32_t tag, uint64_t id, const SkipParams& sp, uint64_t j0, uint64_t cmax,
                       const double* __restrict__ tab, uint64_t (&step)[V], uint32_t* endm, uint32_t* exhm) {
    uint32_t em = 0, xm = 0;
#pragma unroll
    for (int h = 0; h < V / 2; ++h) {
        const uint64_t blk = (j0 >> 1) + h;
        bool s0 = true, s1 = true;
        step[2 * h] = 0;
        step[2 * h + 1] = 0;
        if (blk < c_caps.stream_blocks) {
            const uint4 w = philox_block((uint32_t)blk, tag, id, key);
            step[2 * h] = draw_step(((uint64_t)w.y << 32) | w.x, sp, cmax, &s0, tab);
            step[2 * h + 1] = draw_step(((uint64_t)w.w << 32) | w.z, sp, cmax, &s1, tab);
        } else {
            xm |= 3u << (2 * h);
        }
        em |= (s0 ? 1u : 0u) << (2 * h);
        em |= (s1 ? 1u : 0u) << (2 * h + 1);
    }
    *endm = em;
    *exhm = xm;
}

// One warp walks the positions [start, end) with stream (tag, id): for each
// chosen position (0-based) emit(k, pos) is called, k its index in the
// range.  Returns the number of positions; *err is set if the stream ran out.
// Draw k of a round (lane k / V) lands on base - 1 plus the saturating sum of
// the round's steps up to k; the first draw that ends the range, lies past
// the stream or lands at or past `end` ends the walk.
template <typename Emit>
RS_DEV uint64_t warp_walk(Key2 key, uint32_t tag, uint64_t id, const SkipParams& sp, uint64_t start, uint64_t end,
                          const double* __restrict__ tab, bool* err, Emit&& emit) {
    constexpr int V = kWalkV;
    const int lane = threadIdx.x & 31;
    const uint64_t cmax = end - start + 2;
    uint64_t base = start;   // a step of 1 lands on `base`
    uint64_t count = 0;
    *err = false;
    for (uint64_t j = 0;; j += 32 * V) {
        uint64_t step[V];
        uint32_t endm, exhm;
        draw_steps<V>(key, tag, id, sp, j + (uint64_t)V * lane, cmax, tab, step, &endm, &exhm);
        uint64_t loc[V];   // the lane's own running sums
        loc[0] = step[0];
#pragma unroll
        for (int q = 1; q < V; ++q) loc[q] = sat_add(loc[q - 1], step[q]);
        const uint64_t lincl = warp_inclusive_sat(loc[V - 1]);
        uint64_t excl = __shfl_up_sync(0xFFFFFFFFu, lincl, 1);
        if (lane == 0) excl = 0;
        const uint64_t room = end - base;   // a draw fits while its sum is at most this
        uint32_t badm = endm;
#pragma unroll
        for (int q = 0; q < V; ++q)
            if (sat_add(excl, loc[q]) > room) badm |= 1u << q;
        const uint32_t lanes_bad = __ballot_sync(0xFFFFFFFFu, badm != 0);
        int first_bad = 32 * V;
        if (lanes_bad) {
            const int fl = __ffs(lanes_bad) - 1;
            const int qb = __ffs(__shfl_sync(0xFFFFFFFFu, badm, fl)) - 1;
            first_bad = fl * V + qb;
            *err = (__shfl_sync(0xFFFFFFFFu, exhm, fl) >> qb) & 1u;
        }
#pragma unroll
        for (int q = 0; q < V; ++q) {
            const int k = lane * V + q;
            if (k < first_bad) emit(count + k, base - 1 + sat_add(excl, loc[q]));
        }
        count += first_bad;
        if (first_bad < 32 * V) return count;
        base = base + __shfl_sync(0xFFFFFFFFu, lincl, 31);
    }
}

struct BernArgs {
    uint64_t* stage;
    uint64_t stage_per;
    Key2 key;
    double p;
    uint64_t N, C;
    int chunk_log2;
    uint64_t first, nchunks;
    uint64_t* counts;
    uint64_t* out;
    uint64_t cap;
    int* status;
    const double* tab;
    bool guard;   // skip_fast may decide
};

// The launch's skip parameters (FP64, the same for every chunk), by one
// thread per block: the FP64 pipe of this GPU is too slow to let every
// thread repeat them.  All threads of the block call it.
RS_DEV SkipParams block_skip_params(const BernArgs& A) {
    __shared__ SkipParams sh;
    if (threadIdx.x == 0) sh = skip_params(1.0 / dlog1p(-A.p, A.tab), A.guard);
    __syncthreads();
    return sh;
}

__global__ void bern_count_kernel(BernArgs A) {
    const SkipParams sp = block_skip_params(A);
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < A.nchunks; w += warps) {
        const uint64_t i = A.first + w;
        const uint64_t start = i << A.chunk_log2;
        const uint64_t end = min(start + A.C, A.N);
        bool err;
        const uint64_t c = warp_walk(A.key, TAG_BERN, i, sp, start, end, A.tab, &err, [](uint64_t, uint64_t) {});
        if ((threadIdx.x & 31) == 0) {
            A.counts[w] = c;
            if (err) set_status(A.status, RS_EITER);
        }
    }
}

__global__ void bern_write_kernel(BernArgs A) {
    const SkipParams sp = block_skip_params(A);
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < A.nchunks; w += warps) {
        const uint64_t i = A.first + w;
        const uint64_t start = i << A.chunk_log2;
        const uint64_t end = min(start + A.C, A.N);
        const uint64_t off = A.counts[w];
        if (off >= A.cap) continue;
        uint64_t* out = A.out;
        const uint64_t cap = A.cap;
        bool err;
        warp_walk(A.key, TAG_BERN, i, sp, start, end, A.tab, &err, [=](uint64_t k, uint64_t pos) {
            if (off + k < cap) out[off + k] = pos + 1;
        });
    }
}

// One walk per chunk: positions to the chunk's staging slots (the first
// stage_per of them), the count to counts[w].
__global__ void bern_stage_kernel(BernArgs A) {
    const SkipParams sp = block_skip_params(A);
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < A.nchunks; w += warps) {
        const uint64_t i = A.first + w;
        const uint64_t start = i << A.chunk_log2;
        const uint64_t end = min(start + A.C, A.N);
        uint64_t* slot = A.stage + w * A.stage_per;
        const uint64_t per = A.stage_per;
        bool err;
        const uint64_t c = warp_walk(A.key, TAG_BERN, i, sp, start, end, A.tab, &err, [=](uint64_t k, uint64_t pos) {
            if (k < per) slot[k] = pos + 1;
        });
        if ((threadIdx.x & 31) == 0) {
            A.counts[w] = c;
            if (err) set_status(A.status, RS_EITER);
        }
    }
}

// A block per chunk: the staged positions go to their place in the output;
// a chunk with more positions than its slots walks again with warp 0.
__global__ void bern_copy_kernel(BernArgs A) {
    const uint64_t w = blockIdx.x;
    const uint64_t off = A.counts[w];
    const uint64_t c = A.counts[w + 1] - off;
    if (off >= A.cap) return;
    const uint64_t n = min(c, A.cap - off);
    if (c <= A.stage_per) {
        const uint64_t* slot = A.stage + w * A.stage_per;
        for (uint64_t k = threadIdx.x; k < n; k += blockDim.x) A.out[off + k] = slot[k];
        return;
    }
    if (threadIdx.x >= 32) return;
    const SkipParams sp = skip_params(1.0 / dlog1p(-A.p, A.tab), A.guard);   // rare: one warp per restaged chunk
    const uint64_t i = A.first + w;
    const uint64_t start = i << A.chunk_log2;
    const uint64_t end = min(start + A.C, A.N);
    uint64_t* out = A.out;
    const uint64_t cap = A.cap;
    bool err;
    warp_walk(A.key, TAG_BERN, i, sp, start, end, A.tab, &err, [=](uint64_t k, uint64_t pos) {
        if (off + k < cap) out[off + k] = pos + 1;
    });
}

uint64_t bern_stage_per(double mu) {
    const double v = ceil(mu + 8.0 * sqrt(mu) + 64.0);
    const uint64_t s = v >= 9.0e18 ? (uint64_t)9e18 : (uint64_t)v;
    return (s + 3) & ~3ull;
}

// The size of a Bernoulli(p) sample drawn by its size (Sec. 4.7): BIN(N,
// K/2^62) from stream (SPLIT, 0), complemented to N - BIN when p > 1/2.
__global__ void bern_size_kernel(uint64_t seed, uint64_t N, uint64_t K, int flip, const double* tab, uint64_t* out,
                                 int* status) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    uint64_t c = 0;
    const int rc = binomial(make_key(seed), 0, N, K, 1ull << 62, tab, c);
    if (rc != RS_OK) {
        set_status(status, rc);
        c = 0;
    }
    *out = flip ? N - c : c;
}

cudaError_t launch_bernoulli_size(uint64_t seed, uint64_t N, uint64_t K, bool flip, const double* tab, uint64_t* out,
                                  int* status, cudaStream_t st) {
    bern_size_kernel<<<1, 32, 0, st>>>(seed, N, K, flip ? 1 : 0, tab, out, status);
    return cudaGetLastError();
}

__global__ void fill_range_kernel(uint64_t* out, uint64_t a, uint64_t n) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = a + i + 1;
}

__global__ void set_word_kernel(uint64_t* p, uint64_t v) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *p = v;
}

// --- exclusive scan of uint64 counts (tiles of 8192, recursive) ------------

constexpr int kScanThreads = 1024;
constexpr int kScanPer = 8;
constexpr uint64_t kScanTile = (uint64_t)kScanThreads * kScanPer;

__global__ void scan_tiles_kernel(uint64_t* data, uint64_t n, uint64_t* tile_sums) {
    __shared__ uint64_t warp_tot[kScanThreads / 32];
    const uint64_t i0 = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanPer;
    uint64_t v[kScanPer];
    uint64_t local = 0;
#pragma unroll
    for (int q = 0; q < kScanPer; ++q) {
        v[q] = (i0 + q < n) ? data[i0 + q] : 0;
        local += v[q];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint64_t w = warp_tot[lane];
        uint64_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
            if (lane >= o) wi += y;
        }
        warp_tot[lane] = wi - w;
        if (lane == 31) tile_sums[blockIdx.x] = wi;
    }
    __syncthreads();
    uint64_t run = warp_tot[warp] + incl - local;
#pragma unroll
    for (int q = 0; q < kScanPer; ++q) {
        if (i0 + q < n) data[i0 + q] = run;
        run += v[q];
    }
}

__global__ void scan_add_kernel(uint64_t* data, uint64_t n, const uint64_t* tile_offsets) {
    const uint64_t off = tile_offsets[blockIdx.x];
    const uint64_t t0 = (uint64_t)blockIdx.x * kScanTile;
    const uint64_t t1 = min(t0 + kScanTile, n);
    for (uint64_t i = t0 + threadIdx.x; i < t1; i += kScanThreads) data[i] += off;
}

uint64_t scan_scratch_words(uint64_t n) {
    uint64_t w = 0;
    while (n > 1) {
        n = (n + kScanTile - 1) / kScanTile;
        w += n + 1;
    }
    return w + 1;
}

// Exclusive scan of data[0..n) in place; data[n] receives the total.
static cudaError_t scan_u64(uint64_t* data, uint64_t n, uint64_t* scratch, cudaStream_t st) {
    const uint64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles <= 1) {
        scan_tiles_kernel<<<1, kScanThreads, 0, st>>>(data, n, data + n);
        return cudaGetLastError();
    }
    uint64_t* sums = scratch;   // tiles + 1 words
    scan_tiles_kernel<<<(unsigned)tiles, kScanThreads, 0, st>>>(data, n, sums);
    cudaError_t e = scan_u64(sums, tiles, scratch + tiles + 1, st);
    if (e != cudaSuccess) return e;
    scan_add_kernel<<<(unsigned)tiles, kScanThreads, 0, st>>>(data, n, sums);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(data + n, sums + tiles, sizeof(uint64_t), cudaMemcpyDeviceToDevice, st);
}

cudaError_t launch_bernoulli(const BernLaunch& L, cudaStream_t st) {
    if (L.p == 1.0) {
        const uint64_t n = L.b - L.a;
        const uint64_t w = std::min(n, L.cap);
        if (w > 0) {
            const unsigned blocks = (unsigned)std::min<uint64_t>((w + 255) / 256, 65535);
            fill_range_kernel<<<blocks, 256, 0, st>>>(L.out, L.a, w);
        }
        set_word_kernel<<<1, 32, 0, st>>>(L.total, n);
        return cudaGetLastError();
    }
    BernArgs A;
    A.key = make_key(L.seed);
    A.p = L.p;
    A.N = L.N;
    A.C = 1ull << L.chunk_log2;
    A.chunk_log2 = L.chunk_log2;
    A.first = L.chunk_first;
    A.nchunks = L.nchunks;
    A.counts = L.counts;
    A.out = L.out;
    A.cap = L.cap;
    A.status = L.status;
    A.tab = L.tab;
    A.stage = L.stage;
    A.stage_per = L.stage_per;
    A.guard = L.guard;
    const int threads = 256;
    const unsigned blocks = (unsigned)std::min<uint64_t>((L.nchunks * 32 + threads - 1) / threads,
                                                         (uint64_t)L.sms * 16);
    if (L.stage) {
        bern_stage_kernel<<<blocks, threads, 0, st>>>(A);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = scan_u64(L.counts, L.nchunks, L.scan_scratch, st);
        if (e != cudaSuccess) return e;
        for (uint64_t w0 = 0; w0 < L.nchunks; w0 += 65535u * 1024u) {   // grid x limit, in slices
            BernArgs S = A;
            const uint64_t m = std::min<uint64_t>(L.nchunks - w0, 65535u * 1024u);
            S.counts = A.counts + w0;
            S.first = A.first + w0;
            S.stage = A.stage + w0 * A.stage_per;
            bern_copy_kernel<<<(unsigned)m, 256, 0, st>>>(S);
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
        return cudaMemcpyAsync(L.total, L.counts + L.nchunks, sizeof(uint64_t), cudaMemcpyDeviceToDevice, st);
    }
    bern_count_kernel<<<blocks, threads, 0, st>>>(A);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = scan_u64(L.counts, L.nchunks, L.scan_scratch, st);
    if (e != cudaSuccess) return e;
    bern_write_kernel<<<blocks, threads, 0, st>>>(A);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(L.total, L.counts + L.nchunks, sizeof(uint64_t), cudaMemcpyDeviceToDevice, st);
}

// ---------------------------------------------------------------------------
// Leaf B: Bernoulli-sample the leaf with rate rho slightly above n'/s, retry
// if short, then drop the c - n' positions whose indices are the first
// c - n' distinct FIXUP candidates over [0, c) (Algorithm H on indices).
// rho = min(1, (n' + 3 sqrt(n') + 10) / s); attempt a uses LEAF_B + 256 a.
// ---------------------------------------------------------------------------

constexpr uint32_t kLeafBCap = 8192;   // positions of one attempt
constexpr int kLeafBThreads = 256;

// PosT: 32-bit positions when no leaf exceeds 2^32 positions.
template <typename PosT>
struct LeafBShared {
    PosT pos[kLeafBCap];              // the attempt's positions (offsets in the leaf), increasing
    uint32_t drop[kLeafBCap / 32];    // removed indices, as bits
    uint64_t warp_tot[kLeafBThreads / 32];
    uint32_t warp_cnt[kLeafBThreads / 32];
    uint32_t newcount[3];
    uint64_t last_incl;
    int first_bad;
    int err;
    int rho_one;                      // the leaf's rate is 1: every position
    SkipParams sp;                    // the leaf's skip parameters
};

// Geometric-skip walk of [0, s) by the whole block, V draws per thread per
// round as in warp_walk; positions go to sm.pos (up to the capacity).
// Returns the count; sets sm.err on a run-out stream.
template <int NT, typename PosT>
RS_DEV uint64_t block_walk(Key2 key, uint32_t tag, uint64_t id, const SkipParams& sp, uint64_t s, LeafBShared<PosT>& sm,
                           const double* __restrict__ tab) {
    constexpr int V = kWalkV;
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t cmax = s + 2;
    uint64_t base = 0, count = 0;
    for (uint64_t j = 0;; j += (uint64_t)NT * V) {
        uint64_t step[V];
        uint32_t endm, exhm;
        draw_steps<V>(key, tag, id, sp, j + (uint64_t)V * threadIdx.x, cmax, tab, step, &endm, &exhm);
        uint64_t loc[V];
        loc[0] = step[0];
#pragma unroll
        for (int q = 1; q < V; ++q) loc[q] = sat_add(loc[q - 1], step[q]);
        if (threadIdx.x == 0) sm.first_bad = NT * V;   // its last reads came before the last barrier
        // exclusive saturating sum of the threads' totals before this one
        const uint64_t wincl = warp_inclusive_sat(loc[V - 1]);
        uint64_t wexcl = __shfl_up_sync(0xFFFFFFFFu, wincl, 1);
        if (lane == 0) wexcl = 0;
        if (lane == 31) sm.warp_tot[warp] = wincl;
        __syncthreads();
        if (warp == 0) {
            const uint64_t w = lane < NW ? sm.warp_tot[lane] : 0;
            const uint64_t wi = warp_inclusive_sat(w);
            if (lane < NW) sm.warp_tot[lane] = wi;   // inclusive prefix of warp totals
        }
        __syncthreads();
        const uint64_t excl = sat_add(warp == 0 ? 0 : sm.warp_tot[warp - 1], wexcl);
        const uint64_t room = s - base;
        uint32_t badm = endm;
#pragma unroll
        for (int q = 0; q < V; ++q)
            if (sat_add(excl, loc[q]) > room) badm |= 1u << q;
        const int qb = __ffs(badm) - 1;
        if (badm) atomicMin(&sm.first_bad, (int)threadIdx.x * V + qb);
        if (threadIdx.x == NT - 1) sm.last_incl = sat_add(excl, loc[V - 1]);
        __syncthreads();
        const int fb = sm.first_bad;
#pragma unroll
        for (int q = 0; q < V; ++q) {
            const int k = (int)threadIdx.x * V + q;
            if (k < fb && count + k < kLeafBCap) sm.pos[count + k] = (PosT)(base - 1 + sat_add(excl, loc[q]));
        }
        if (badm && (int)threadIdx.x * V + qb == fb && ((exhm >> qb) & 1u)) sm.err = 1;
        count += fb;
        const uint64_t last = sm.last_incl;
        __syncthreads();
        if (fb < NT * V) return count;
        base += last;
    }
}

struct LeafBArgs {
    const NodeRec* leaves;
    uint64_t nleaves, first_id;
    Key2 key;
    uint64_t* out;
    int* status;
    const double* tab;
    bool guard;
};

// One leaf of Algorithm B, by the whole block: the walk (retried while
// short), then the c - n' removed indices -- the first c - n' distinct valid
// candidates of stream (FIXUP, id) over [0, c), Algorithm H on indices -- as
// bits, and the kept positions written in order (a kept index's place is
// the number of kept indices below it).
template <int NT, typename PosT>
RS_DEV void leaf_b_one(LeafBShared<PosT>& sm, const NodeRec& r, uint64_t id, Key2 key, uint64_t* __restrict__ out,
                       int* status, const double* __restrict__ tab, bool guard) {
    constexpr int NW = NT / 32;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (r.c == 0) return;
    // the leaf's rate and skip parameters in FP64, once, by thread 0 (the
    // FP64 pipe of this GPU is too slow to let every thread repeat them);
    // the last reads of these fields came before the last leaf's final barrier
    if (tid == 0) {
        const double dn = (double)r.c;
        const double rho = (dn + 3.0 * sqrt(dn) + 10.0) / (double)r.S;
        sm.rho_one = rho >= 1.0;
        if (rho < 1.0) sm.sp = skip_params(1.0 / dlog1p(-rho, tab), guard);
        sm.err = 0;
    }
    uint64_t c = 0;
    int attempt = 0;
    bool fail = false;
    __syncthreads();
    if (sm.rho_one) {
        c = r.S;
        const uint64_t fill = c < kLeafBCap ? c : kLeafBCap;
        for (uint64_t i = tid; i < fill; i += NT) sm.pos[i] = (PosT)i;
        __syncthreads();
    } else {
        const SkipParams sp = sm.sp;
        for (attempt = 0; (uint64_t)attempt < c_caps.b_attempts; ++attempt) {
            c = block_walk<NT>(key, TAG_LEAF_B + 256u * (uint32_t)attempt, id, sp, r.S, sm, tab);
            if (sm.err) break;
            if (c >= r.c) break;
        }
        if (sm.err || (uint64_t)attempt == c_caps.b_attempts) {
            if (tid == 0) set_status(status, RS_EITER);
            fail = true;
        }
    }
    if (!fail && c > kLeafBCap) {
        if (tid == 0) set_status(status, RS_ECAPACITY);
        fail = true;
    }
    if (fail) {
        __syncthreads();
        return;
    }
    const uint32_t cc = (uint32_t)c, drop = (uint32_t)(c - r.c);
    const uint32_t words = (cc + 31) >> 5;
    for (uint32_t i = tid; i < words; i += NT) sm.drop[i] = 0;
    if (tid < 3) sm.newcount[tid] = 0;
    __syncthreads();
    const LeafRec fr{0, c, drop, 0, id};
    const bool ok = distinct_rounds<NT, 0>(
        sm.newcount, fr, lemire_threshold(c), key, TAG_FIXUP, drop, status, tid,
        [&](uint64_t v) -> uint32_t {
            const uint32_t bit = 1u << (v & 31);
            return (atomicOr(&sm.drop[v >> 5], bit) & bit) ? 0u : 1u;
        },
        [] { return false; });
    if (!ok) return;
    // kept indices: each warp takes a contiguous run of words, one bit per
    // lane of the current word so that the stores are coalesced
    auto kept = [&](uint32_t w) {
        uint32_t bits = ~sm.drop[w];
        if (w * 32 + 32 > cc) bits &= (1u << (cc & 31)) - 1u;   // beyond the attempt
        return bits;
    };
    const uint32_t per = (words + NW - 1) / NW;
    const uint32_t w0 = min(warp * per, words), w1 = min(w0 + per, words);
    uint32_t cnt = 0;
    for (uint32_t w = w0 + lane; w < w1; w += 32) cnt += __popc(kept(w));
    cnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
    if (lane == 0) sm.warp_cnt[warp] = cnt;
    __syncthreads();
    uint32_t base = 0;
    for (uint32_t i = 0; i < warp; ++i) base += sm.warp_cnt[i];
    uint64_t* dst = out + r.off;
    const uint64_t lo1 = r.lo + 1;
    for (uint32_t w = w0; w < w1; ++w) {
        const uint32_t bits = kept(w);
        if ((bits >> lane) & 1u) dst[base + __popc(bits & ((1u << lane) - 1u))] = lo1 + sm.pos[w * 32 + lane];
        base += __popc(bits);
    }
    __syncthreads();
}

template <typename PosT>
__global__ void __launch_bounds__(kLeafBThreads) leaf_b_kernel(LeafBArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto& sm = *reinterpret_cast<LeafBShared<PosT>*>(smem_raw);
    for (uint64_t leaf = blockIdx.x; leaf < A.nleaves; leaf += gridDim.x)
        leaf_b_one<kLeafBThreads>(sm, A.leaves[leaf], A.first_id + leaf, A.key, A.out, A.status, A.tab, A.guard);
}

// Algorithm B leaves of a batch group or of range queries (leaf sizes not
// bounded in advance: 64-bit positions).
template <class View>
__global__ void __launch_bounds__(kLeafBThreads) group_leaf_b_kernel(View G, const double* tab) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto& sm = *reinterpret_cast<LeafBShared<uint64_t>*>(smem_raw);
    for (uint64_t g = blockIdx.x; g < G.nleaves; g += gridDim.x) {
        const ResolvedLeaf L = resolve_leaf(G, g);
        leaf_b_one<kLeafBThreads>(sm, L.rec, L.id, make_key(L.seed), L.out, L.status, tab, true);
    }
}

template <class View>
static cudaError_t launch_group_leaves_b(const View& G, const double* tab, int sms, cudaStream_t st) {
    const size_t smem = sizeof(LeafBShared<uint64_t>);
    auto kern = group_leaf_b_kernel<View>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kLeafBThreads, smem);
    if (e != cudaSuccess) return e;
    const uint64_t grid = std::min<uint64_t>(G.nleaves, (uint64_t)sms * std::max(per_sm, 1));
    if (grid == 0) return cudaSuccess;
    kern<<<(unsigned)grid, kLeafBThreads, smem, st>>>(G, tab);
    return cudaGetLastError();
}

cudaError_t launch_batch_leaves_b(const BatchGroupView& G, const double* tab, int sms, cudaStream_t st) {
    return launch_group_leaves_b(G, tab, sms, st);
}
cudaError_t launch_batch_leaves_b(const QueryBoundView& G, const double* tab, int sms, cudaStream_t st) {
    return launch_group_leaves_b(G, tab, sms, st);
}
cudaError_t launch_batch_leaves_b(const QueryInnerView& G, const double* tab, int sms, cudaStream_t st) {
    return launch_group_leaves_b(G, tab, sms, st);
}

template <typename PosT>
static cudaError_t launch_leaves_b_t(const LeafBLaunch& L, cudaStream_t st) {
    const size_t smem = sizeof(LeafBShared<PosT>);
    auto kern = leaf_b_kernel<PosT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kLeafBThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    LeafBArgs A{L.leaves, L.nleaves, L.first_id, make_key(L.seed), L.out, L.status, L.tab, L.guard};
    const uint64_t grid = std::min<uint64_t>(L.nleaves, (uint64_t)L.sms * per_sm);
    kern<<<(unsigned)grid, kLeafBThreads, smem, st>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_leaves_b(const LeafBLaunch& L, cudaStream_t st) {
    if (L.smax <= (1ull << 32)) return launch_leaves_b_t<uint32_t>(L, st);
    return launch_leaves_b_t<uint64_t>(L, st);
}

}  // namespace rs
