// rs_leaf.cu -- base-case kernels: leaf H (without replacement) and leaf WR
// (with replacement), plus the sorted write-out.
//
// Leaf H is Algorithm H (Sec. 2) with sorted output (Sec. 4.1): the leaf's
// selection is the first k distinct valid candidates of its LEAF_H stream,
// k = n' (or s - n' when more than half the leaf is taken, whose complement
// is then written: Sec. 2's n > N/2 rule applied per leaf).
//
// Leaf WR (Sec. 4.6) is the same machinery without the distinctness rule:
// the first n' valid candidates of its LEAF_WR stream, sorted as a multiset.
#include "rs_big_leaf.cuh"
#include "rs_hash_leaf.cuh"

namespace rs {

struct LeafJob {
    const NodeRec* leaves;   // leaf records, leaf i at leaves[i]
    uint64_t nleaves;
    uint64_t first_id;       // heap id of leaf 0 (= 2^D)
    uint64_t seed;
    uint64_t* out;
    int* status;
    uint32_t* ovf_list;      // leaves left to the general path
    uint32_t* ovf_count;
    uint32_t cap;            // largest selection handled here
    RoundKeys rk;            // the seed's Philox round keys
};

// Two shapes of the leaf kernel: 256 threads with room for 4,864 values
// (leaves of about 4,096 samples, 4 blocks per SM), and 512 threads with
// room for 9,728 (leaves of about 8,192, 2 blocks per SM): the same warps per
// SM, half the per-leaf fixed costs per sample for the larger leaves.
constexpr int kHashThreads = 256;
constexpr int kLargeThreads = 512;
constexpr uint32_t kLargeCap = 2 * kLeafFastCap;

// One block per leaf at a time, persistent over the leaves; leaves the
// shared-memory table cannot take go to the general path's list.
// The job is a __grid_constant__ parameter so that the Philox rounds read
// their keys from the parameter bank.
// Copies a leaf record (32 bytes) into shared memory asynchronously.
RS_DEV void prefetch_record(NodeRec* dst, const NodeRec* src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n\t"
                 "cp.async.cg.shared.global [%2], [%3], 16;\n\t"
                 "cp.async.commit_group;" ::"r"(d), "l"(src), "r"(d + 16),
                 "l"(reinterpret_cast<const unsigned char*>(src) + 16)
                 : "memory");
}
RS_DEV void prefetch_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <typename KeyT, bool WR, int NT, uint32_t CAP, bool POW2>
__global__ void __launch_bounds__(NT, 1024 / NT) leaf_kernel(const __grid_constant__ LeafJob job) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto& sm = *reinterpret_cast<HashShared<KeyT, NT / 32, CAP>*>(smem_raw);
    // the next leaf's record is copied in (thread 0, cp.async) while this
    // leaf runs; the wait and a barrier at the end of the leaf make it visible
    __shared__ __align__(16) NodeRec recbuf[2];
    if (blockIdx.x >= job.nleaves) return;
    if (threadIdx.x == 0) {
        prefetch_record(&recbuf[0], &job.leaves[blockIdx.x]);
        prefetch_wait();
    }
    __syncthreads();
    uint32_t par = 0;
    for (uint64_t leaf = blockIdx.x; leaf < job.nleaves; leaf += gridDim.x, par ^= 1u) {
        const NodeRec r = recbuf[par];
        if (threadIdx.x == 0 && leaf + gridDim.x < job.nleaves)
            prefetch_record(&recbuf[par ^ 1u], &job.leaves[leaf + gridDim.x]);
        if (r.c != 0) {
            const LeafRec lr{r.lo, r.S, r.c, r.off, job.first_id + leaf};
            if (!hash_leaf<KeyT, NT, 0, WR, CAP, RoundKeys, POW2, true>(sm, lr, job.rk, job.out, job.status,
                                                                       threadIdx.x, job.cap)) {
                if (threadIdx.x == 0) job.ovf_list[atomicAdd(job.ovf_count, 1u)] = (uint32_t)leaf;
            }
        }
        if (threadIdx.x == 0) prefetch_wait();
        __syncthreads();
    }
}

template <bool WR>
__global__ void __launch_bounds__(kBigThreads) big_leaf_kernel(LeafJob job, BigScratch sc) {
    __shared__ uint32_t tmp[kBigThreads / 32 + 1];
    const Key2 key = make_key(job.seed);
    const uint32_t count = *job.ovf_count;
    for (uint32_t t = 0; t < count; ++t) {
        const uint64_t leaf = job.ovf_list[t];
        const NodeRec r = job.leaves[leaf];
        const bool comp = !WR && (r.c > r.S - r.c);
        const uint64_t k = comp ? r.S - r.c : r.c;
        if (k > sc.kmax) {
            if (threadIdx.x == 0) set_status(job.status, RS_ECAPACITY);
            continue;
        }
        if (!big_select<WR>(r, job.first_id + leaf, key, k, sc, tmp, job.status)) continue;
        uint64_t* dst = job.out + r.off;
        if (!comp) {
            for (uint64_t i = threadIdx.x; i < k; i += kBigThreads) dst[i] = r.lo + 1 + sc.keys[i];
        } else {
            const uint64_t nout = r.S - k;
            for (uint64_t o = threadIdx.x; o < nout; o += kBigThreads) {
                uint64_t lo = 0, hi = k;
                while (lo < hi) {
                    const uint64_t mid = (lo + hi) >> 1;
                    if (sc.keys[mid] - mid <= o) lo = mid + 1; else hi = mid;
                }
                dst[o] = r.lo + 1 + o + lo;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------

template <typename KeyT, bool WR, int NT, uint32_t CAP, bool POW2>
static cudaError_t launch_fast(LeafJob job, uint32_t cap_knob, int sms, int per_sm_cap, cudaStream_t st) {
    job.cap = cap_knob ? std::min<uint32_t>(cap_knob, CAP) : CAP;
    const size_t smem = sizeof(HashShared<KeyT, NT / 32, CAP>);
    auto kern = leaf_kernel<KeyT, WR, NT, CAP, POW2>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm_cap > 0 && per_sm > per_sm_cap) per_sm = per_sm_cap;
    if (per_sm < 1) per_sm = 1;
    const uint64_t grid = std::min<uint64_t>(job.nleaves, (uint64_t)sms * per_sm);
    kern<<<(unsigned)grid, NT, smem, st>>>(job);
    return cudaGetLastError();
}

// Launches whose leaves all have the same power-of-two size (N a power of
// two times the leaf count, as in the benchmark's 2^50) take a kernel
// without the code for void candidates, which would otherwise cost the
// power-of-two path registers and time.
template <bool WR, int NT, uint32_t CAP>
static cudaError_t launch_shape(const LeafJob& job, const LeafLaunch& L, cudaStream_t st) {
    if (L.smax <= (1ull << 32)) {
        if (L.pow2_leaves) return launch_fast<uint32_t, WR, NT, CAP, true>(job, L.cap, L.sms, L.blocks_per_sm, st);
        return launch_fast<uint32_t, WR, NT, CAP, false>(job, L.cap, L.sms, L.blocks_per_sm, st);
    }
    if (NT == kHashThreads && L.mean_count <= kCompact64Mean) {   // 64-bit keys: the compact table
        if (L.pow2_leaves)
            return launch_fast<uint64_t, WR, NT, kCompact64Cap, true>(job, L.cap, L.sms, L.blocks_per_sm, st);
        return launch_fast<uint64_t, WR, NT, kCompact64Cap, false>(job, L.cap, L.sms, L.blocks_per_sm, st);
    }
    if (L.pow2_leaves) return launch_fast<uint64_t, WR, NT, CAP, true>(job, L.cap, L.sms, L.blocks_per_sm, st);
    return launch_fast<uint64_t, WR, NT, CAP, false>(job, L.cap, L.sms, L.blocks_per_sm, st);
}

cudaError_t launch_leaves(const LeafLaunch& L, cudaStream_t st) {
    LeafJob job{L.leaves, L.nleaves, L.first_id, L.seed, L.out, L.status, L.ovf_list, L.ovf_count, 0,
                RoundKeys::of(L.seed)};
    cudaError_t e = cudaMemsetAsync(L.ovf_count, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    // leaves averaging well above the small shape's room take the large one
    const bool large = L.mean_count * 20 > (uint64_t)kLeafFastCap * 17;
    if (L.with_replacement)
        e = large ? launch_shape<true, kLargeThreads, kLargeCap>(job, L, st)
                  : launch_shape<true, kHashThreads, kLeafFastCap>(job, L, st);
    else
        e = large ? launch_shape<false, kLargeThreads, kLargeCap>(job, L, st)
                  : launch_shape<false, kHashThreads, kLeafFastCap>(job, L, st);
    if (e != cudaSuccess) return e;
    if (L.big_kmax == 0) return cudaSuccess;   // no leaf can exceed the capacity
    const BigScratch sc = carve_big_scratch(L.big_pool, L.big_kmax);
    if (L.with_replacement) big_leaf_kernel<true><<<1, kBigThreads, 0, st>>>(job, sc);
    else big_leaf_kernel<false><<<1, kBigThreads, 0, st>>>(job, sc);
    return cudaGetLastError();
}

uint64_t big_pool_bytes(uint64_t kmax) {
    uint64_t tmax = 32;
    while (tmax < kmax) tmax <<= 1;
    return kmax * (8 + 8 + 8 + 4 + 4) + (tmax + 1) * 4;
}

}  // namespace rs
