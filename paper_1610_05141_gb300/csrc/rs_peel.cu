// rs_peel.cu -- online sorted sampling by peeling (Sec. 4.1): the sample in
// increasing order as a sequence of batches of about n0 values, each batch
// made in O(n0) work.
//
// With n_t samples left among the N_t positions after lo_t, batch t splits
// off the next m_t = ceil(N_t n0 / n_t) positions and takes HG(n_t, m_t, N_t)
// of the samples (stream (SPLIT, t + 1)); once m_t >= N_t the batch is the
// rest.  Its values are leaf H of node t + 1 over [lo_t, lo_t + m_t).  The
// chain of deviates is sequential by definition: one warp walks it for the
// batches of a call (each deviate's trials spread over its lanes), then one
// leaf launch makes all their values.
#include <new>

#include "rs_deviates.cuh"
#include "rs_internal.h"

namespace rs {
int ctx_device(rs_ctx* ctx);
int ctx_sms(rs_ctx* ctx);
const double* ctx_tab(rs_ctx* ctx);
void ctx_count_launches(rs_ctx* ctx, uint64_t n);

struct PeelState {
    uint64_t n, N, lo, t;   // samples left, positions left, positions done, batches done
};

// info: batches, values, largest range, largest selection, the count of the
// batch that did not fit (0 if none), then the new state's n, N, t.
__global__ void peel_chain_kernel(PeelState* st, uint32_t n0, uint64_t seed, uint32_t max_batches, uint64_t cap,
                                  NodeRec* rec, uint64_t* info, const double* __restrict__ tab, int* status) {
    // one warp: the state is the same in every lane, the lanes share each
    // deviate's trials, lane 0 writes
    if (blockIdx.x != 0 || threadIdx.x >= 32) return;
    const bool lead = threadIdx.x == 0;
    PeelState s = *st;
    const Key2 key = make_key(seed);
    uint64_t off = 0, maxm = 0, maxk = 0, need = 0;
    uint32_t b = 0;
    while (b < max_batches && s.n > 0) {
        const unsigned __int128 m128 = ((unsigned __int128)s.N * n0 + (s.n - 1)) / s.n;
        uint64_t m, c;
        if (m128 >= s.N) {
            m = s.N;
            c = s.n;
        } else {
            m = (uint64_t)m128;
            const int rc = hypergeometric_warp(key, s.t + 1, s.n, m, s.N, tab, c);
            if (rc != RS_OK) {
                if (lead) set_status(status, rc);
                break;
            }
        }
        if (off + c > cap) {
            need = c;
            break;
        }
        if (lead) rec[b] = NodeRec{s.lo, m, c, off};
        off += c;
        ++b;
        const uint64_t k = c < m - c ? c : m - c;
        maxm = m > maxm ? m : maxm;
        maxk = k > maxk ? k : maxk;
        s.lo += m;
        s.N -= m;
        s.n -= c;
        s.t += 1;
    }
    if (!lead) return;
    *st = s;
    info[0] = b;
    info[1] = off;
    info[2] = maxm;
    info[3] = maxk;
    info[4] = need;
    info[5] = s.n;
    info[6] = s.N;
    info[7] = s.t;
}

}  // namespace rs

struct rs_peel {
    rs_ctx* ctx = nullptr;
    int device = 0;
    uint64_t n = 0, N = 0, seed = 0;
    uint32_t n0 = 0, max_batches = 0;
    uint64_t n_left = 0, N_left = 0, t = 0;   // host copy of the state after the last call
    rs::PeelState* state = nullptr;
    rs::NodeRec* rec = nullptr;
    uint64_t* info = nullptr;                // 8 words
    uint64_t* info_host = nullptr;           // 8 words, pinned
    uint32_t* ovf = nullptr;                 // max_batches + 1 words (the last one counts)
    int* status = nullptr;
    void* big_pool = nullptr;
    uint64_t big_pool_bytes = 0;
};

namespace {

struct PeelGuard {
    int prev = -1;
    bool ok = false;
    explicit PeelGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~PeelGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

int peel_rc(cudaError_t e) {
    if (e == cudaSuccess) return RS_OK;
    return e == cudaErrorMemoryAllocation ? RS_ENOMEM : RS_ECUDA;
}

void peel_free(rs_peel* it) {
    cudaFree(it->state);
    cudaFree(it->rec);
    cudaFree(it->info);
    cudaFreeHost(it->info_host);
    cudaFree(it->ovf);
    cudaFree(it->status);
    cudaFree(it->big_pool);
    delete it;
}

}  // namespace

extern "C" {

int rs_peel_create(rs_ctx* ctx, uint64_t n, uint64_t N, uint64_t seed, uint32_t n0, uint32_t max_batches,
                   rs_peel** out) {
    if (!out) return RS_EINVAL;
    *out = nullptr;
    if (!ctx || n0 == 0 || N > (1ull << 62) || n > N || max_batches == 0 || max_batches > (1u << 20))
        return RS_EINVAL;
    const int dev = rs::ctx_device(ctx);
    PeelGuard g(dev);
    if (!g.ok) return RS_ECUDA;
    rs_peel* it = new (std::nothrow) rs_peel;
    if (!it) return RS_ENOMEM;
    it->ctx = ctx;
    it->device = dev;
    it->n = it->n_left = n;
    it->N = it->N_left = N;
    it->seed = seed;
    it->n0 = n0;
    it->max_batches = max_batches;
    int rc = peel_rc(cudaMalloc(&it->state, sizeof(rs::PeelState)));
    if (!rc) rc = peel_rc(cudaMalloc(&it->rec, max_batches * sizeof(rs::NodeRec)));
    if (!rc) rc = peel_rc(cudaMalloc(&it->info, 8 * sizeof(uint64_t)));
    if (!rc) rc = peel_rc(cudaMallocHost(&it->info_host, 8 * sizeof(uint64_t)));
    if (!rc) rc = peel_rc(cudaMalloc(&it->ovf, (max_batches + 1) * sizeof(uint32_t)));
    if (!rc) rc = peel_rc(cudaMalloc(&it->status, sizeof(int)));
    const rs::PeelState s0{n, N, 0, 0};
    if (!rc) rc = peel_rc(cudaMemcpy(it->state, &s0, sizeof(s0), cudaMemcpyHostToDevice));
    if (!rc) rc = peel_rc(cudaMemset(it->status, 0, sizeof(int)));
    if (rc) {
        peel_free(it);
        return rc;
    }
    *out = it;
    return RS_OK;
}

int rs_peel_next(rs_peel* it, uint64_t* out_dev, uint64_t cap, uint64_t* count_out, uint32_t* batches_out,
                 void* stream) {
    if (!it || !count_out || !batches_out) return RS_EINVAL;
    *count_out = 0;
    *batches_out = 0;
    if (cap > 0 && (!out_dev || ((uintptr_t)out_dev & 7))) return RS_EINVAL;
    if (it->n_left == 0) return RS_OK;
    PeelGuard g(it->device);
    if (!g.ok) return RS_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint64_t t0 = it->t;
    rs::peel_chain_kernel<<<1, 32, 0, st>>>(it->state, it->n0, it->seed, it->max_batches, cap, it->rec, it->info,
                                            rs::ctx_tab(it->ctx), it->status);
    int rc = peel_rc(cudaGetLastError());
    if (!rc) rc = peel_rc(cudaMemcpyAsync(it->info_host, it->info, 8 * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    if (!rc) rc = peel_rc(cudaStreamSynchronize(st));
    rs::ctx_count_launches(it->ctx, 1);
    if (rc) return rc;
    const uint64_t* inf = it->info_host;
    const uint64_t b = inf[0], total = inf[1], maxm = inf[2], maxk = inf[3], need = inf[4];
    it->n_left = inf[5];
    it->N_left = inf[6];
    it->t = inf[7];
    if (b > 0) {
        // The general path must be ready for any leaf the shared-memory
        // table cannot take (a large selection, or a complement whose range
        // does not fit the bitmap).
        const uint64_t big_kmax = std::min<uint64_t>(std::max<uint64_t>(maxk, 64), rs::kBigLeafMax);
        const uint64_t bytes = rs::big_pool_bytes(big_kmax);
        if (it->big_pool_bytes < bytes) {
            cudaFree(it->big_pool);
            it->big_pool = nullptr;
            it->big_pool_bytes = 0;
            rc = peel_rc(cudaMalloc(&it->big_pool, bytes));
            if (rc) return rc;
            it->big_pool_bytes = bytes;
        }
        rs::LeafLaunch L{};
        L.leaves = it->rec;
        L.nleaves = b;
        L.first_id = t0 + 1;
        L.seed = it->seed;
        L.smax = maxm;
        L.out = out_dev;
        L.status = it->status;
        L.ovf_list = it->ovf;
        L.ovf_count = it->ovf + it->max_batches;
        L.big_pool = it->big_pool;
        L.big_kmax = big_kmax;
        L.cap = 0;
        L.sms = rs::ctx_sms(it->ctx);
        L.with_replacement = false;
        L.mean_count = total / b;
        rc = peel_rc(rs::launch_leaves(L, st));
        rs::ctx_count_launches(it->ctx, 2);
        if (rc) return rc;
    }
    int h = 0;
    rc = peel_rc(cudaMemcpyAsync(&h, it->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (!rc) rc = peel_rc(cudaStreamSynchronize(st));
    if (rc) return rc;
    if (h != RS_OK) return h;
    *count_out = total;
    *batches_out = (uint32_t)b;
    if (b == 0 && need > 0) {
        *count_out = need;   // the next batch's size
        return RS_ECAPACITY;
    }
    return RS_OK;
}

int rs_peel_state(rs_peel* it, uint64_t* n_left, uint64_t* N_left, uint64_t* batches_done) {
    if (!it || !n_left || !N_left || !batches_done) return RS_EINVAL;
    *n_left = it->n_left;
    *N_left = it->N_left;
    *batches_done = it->t;
    return RS_OK;
}

int rs_peel_destroy(rs_peel* it) {
    if (!it) return RS_EINVAL;
    PeelGuard g(it->device);
    cudaDeviceSynchronize();
    peel_free(it);
    return RS_OK;
}

}  // extern "C"
