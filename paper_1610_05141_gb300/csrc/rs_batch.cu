// rs_batch.cu -- many independent sampling requests in one device run.
//
// A plan (host) validates the requests, computes every tree depth and lays
// out: the node records of all requests in one scratch array, per tree level
// a list of warp items (request, first node, count), and the leaves grouped
// by kind and key width.  A run (device only) is a fixed sequence of
// launches -- roots, one launch per tree level across all requests, one
// persistent leaf kernel per group, the general path for oversized leaves --
// that is captured once into a CUDA graph and replayed.  Each request's
// output equals its own rs_sample / rs_sample_with_replacement / rs_sample_b
// output: the sample is a function of the request alone (Sec. 4.5).
#include <cstring>
#include <new>
#include <vector>

#include "rs_batch.cuh"
#include "rs_big_leaf.cuh"
#include "rs_hash_leaf.cuh"
#include "rs_internal.h"
#include "rs_tree_warp.cuh"

namespace rs {

constexpr int kBatchTreeWarps = 4;
constexpr int kBatchLeafThreads = 256;
constexpr uint32_t kBatchTreeBatch = 128;

__global__ void batch_init_kernel(const BatchReq* __restrict__ reqs, uint32_t R, NodeRec* __restrict__ nodes,
                                  int* __restrict__ status) {
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
        const BatchReq q = reqs[r];
        status[r] = q.status0;
        if (q.D >= 0) nodes[q.node_base + 1] = NodeRec{0, q.N, q.n, 0};
    }
}

__global__ void __launch_bounds__(kBatchTreeWarps * 32) batch_tree_kernel(const BatchReq* __restrict__ reqs,
                                                                          const BatchTreeItem* __restrict__ items,
                                                                          uint32_t nitems, NodeRec* nodes,
                                                                          const double* __restrict__ tab,
                                                                          int* status) {
    extern __shared__ double tree_logs[];
    const uint32_t warp = threadIdx.x >> 5;
    const uint32_t it = blockIdx.x * kBatchTreeWarps + warp;
    if (it >= nitems) return;
    const BatchTreeItem e = items[it];
    const BatchReq q = reqs[e.req];
    double* logs = tree_logs + warp * 32 * kLogSlots;
    if (q.kind == RS_KIND_WR)
        tree_batch_warp<true>(nodes + q.node_base, e.v0, e.count, make_key(q.seed), tab, status + e.req, logs);
    else
        tree_batch_warp<false>(nodes + q.node_base, e.v0, e.count, make_key(q.seed), tab, status + e.req, logs);
}

template <typename KeyT, bool WR>
__global__ void __launch_bounds__(kBatchLeafThreads) batch_leaf_kernel(BatchGroupView G, uint32_t* ovf_list,
                                                                       uint32_t* ovf_count, uint32_t cap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto& sm = *reinterpret_cast<HashShared<KeyT, kBatchLeafThreads / 32>*>(smem_raw);
    for (uint64_t g = blockIdx.x; g < G.nleaves; g += gridDim.x) {
        const ResolvedLeaf L = resolve_leaf(G, g);
        if (L.rec.c == 0) continue;
        const LeafRec lr{L.rec.lo, L.rec.S, L.rec.c, L.rec.off, L.id};
        if (!hash_leaf<KeyT, kBatchLeafThreads, 0, WR>(sm, lr, make_key(L.seed), L.out, L.status, threadIdx.x, cap)) {
            if (threadIdx.x == 0) ovf_list[atomicAdd(ovf_count, 1u)] = (uint32_t)g;
        }
    }
}

template <bool WR>
__global__ void __launch_bounds__(kBigThreads) batch_big_kernel(BatchGroupView G, const uint32_t* ovf_list,
                                                                const uint32_t* ovf_count, BigScratch sc) {
    __shared__ uint32_t tmp[kBigThreads / 32 + 1];
    const uint32_t count = *ovf_count;
    for (uint32_t t = 0; t < count; ++t) {
        const ResolvedLeaf L = resolve_leaf(G, ovf_list[t]);
        const NodeRec& r = L.rec;
        const bool comp = !WR && (r.c > r.S - r.c);
        const uint64_t k = comp ? r.S - r.c : r.c;
        if (k > sc.kmax) {
            if (threadIdx.x == 0) set_status(L.status, RS_ECAPACITY);
            continue;
        }
        if (!big_select<WR>(r, L.id, make_key(L.seed), k, sc, tmp, L.status)) continue;
        big_write(r, k, comp, sc, L.out + r.off);
        __syncthreads();
    }
}

}  // namespace rs

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------

namespace {

struct Group {
    int kind = 0;
    bool wide = false;
    uint32_t m = 0;
    uint64_t nleaves = 0;
    uint32_t* req_of = nullptr;    // device
    uint64_t* prefix = nullptr;    // device, m + 1
    uint32_t* ovf = nullptr;       // device, nleaves + 1 (list, then count)
    int grid_per_sm = 0;           // leaf kernel blocks per SM (0 = occupancy limit)
};

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? RS_OK : (e == cudaErrorMemoryAllocation ? RS_ENOMEM : RS_ECUDA); }

int depth_for(uint64_t n, uint64_t N, uint32_t n0) {
    int D = 0;
    while ((unsigned __int128)n > ((unsigned __int128)n0 << D)) ++D;
    while (D > 0 && ((unsigned __int128)1 << D) > (unsigned __int128)N) --D;
    return D;
}

template <typename T>
int upload(T** dst, const std::vector<T>& v) {
    *dst = nullptr;
    if (v.empty()) return RS_OK;
    int rc = cuda_rc(cudaMalloc((void**)dst, v.size() * sizeof(T)));
    if (rc) return rc;
    return cuda_rc(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
}

}  // namespace

struct rs_batchplan {
    int device = 0;
    int sms = 0;
    uint32_t R = 0;
    const double* tab = nullptr;   // the context's ln i! table
    rs::BatchReq* reqs = nullptr;
    rs::NodeRec* nodes = nullptr;
    std::vector<std::pair<rs::BatchTreeItem*, uint32_t>> levels;   // device items, count
    Group groups[5];
    void* big_pool = nullptr;
    uint64_t big_kmax = 0;
    // graph of the last run
    bool ran_eagerly = false;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t capture_stream = nullptr;
    uint64_t* graph_pool = nullptr;
    int32_t* graph_status = nullptr;
    uint64_t launches_per_run = 0;
};

namespace {

// The device work of a run, issued on `st`.
int issue_run(rs_batchplan* B, uint64_t* pool, int32_t* status, cudaStream_t st, uint64_t* launches) {
    uint64_t nl = 0;
    int* stat = reinterpret_cast<int*>(status);
    rs::batch_init_kernel<<<(B->R + 255) / 256, 256, 0, st>>>(B->reqs, B->R, B->nodes, stat);
    ++nl;
    const size_t tree_smem = (size_t)rs::kBatchTreeWarps * 32 * rs::kLogSlots * sizeof(double);
    for (auto& lv : B->levels) {
        const unsigned blocks = (lv.second + rs::kBatchTreeWarps - 1) / rs::kBatchTreeWarps;
        rs::batch_tree_kernel<<<blocks, rs::kBatchTreeWarps * 32, tree_smem, st>>>(B->reqs, lv.first, lv.second,
                                                                                   B->nodes, B->tab, stat);
        ++nl;
    }
    for (Group& G : B->groups) {
        if (G.nleaves == 0) continue;
        rs::BatchGroupView V{B->reqs, G.req_of, G.prefix, G.m, G.nleaves, B->nodes, pool, stat};
        if (G.kind == RS_KIND_B) {
            if (rs::launch_batch_leaves_b(V, B->sms, st) != cudaSuccess) return RS_ECUDA;
            ++nl;
            continue;
        }
        if (cudaMemsetAsync(G.ovf + G.nleaves, 0, sizeof(uint32_t), st) != cudaSuccess) return RS_ECUDA;
        const bool wr = G.kind == RS_KIND_WR;
        void (*kern)(rs::BatchGroupView, uint32_t*, uint32_t*, uint32_t);
        size_t smem;
        if (G.wide) {
            kern = wr ? rs::batch_leaf_kernel<uint64_t, true> : rs::batch_leaf_kernel<uint64_t, false>;
            smem = sizeof(rs::HashShared<uint64_t, rs::kBatchLeafThreads / 32>);
        } else {
            kern = wr ? rs::batch_leaf_kernel<uint32_t, true> : rs::batch_leaf_kernel<uint32_t, false>;
            smem = sizeof(rs::HashShared<uint32_t, rs::kBatchLeafThreads / 32>);
        }
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return RS_ECUDA;
        int per_sm = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, rs::kBatchLeafThreads, smem) != cudaSuccess)
            return RS_ECUDA;
        if (G.grid_per_sm > 0) per_sm = std::min(per_sm, G.grid_per_sm);
        const uint64_t grid = std::min<uint64_t>(G.nleaves, (uint64_t)B->sms * std::max(per_sm, 1));
        kern<<<(unsigned)grid, rs::kBatchLeafThreads, smem, st>>>(V, G.ovf, G.ovf + G.nleaves, rs::kLeafFastCap);
        ++nl;
        if (B->big_kmax) {
            rs::BigScratch sc;
            uint64_t tmax = 32;
            while (tmax < B->big_kmax) tmax <<= 1;
            unsigned char* p = static_cast<unsigned char*>(B->big_pool);
            sc.keys = reinterpret_cast<uint64_t*>(p); p += B->big_kmax * 8;
            sc.cand = reinterpret_cast<uint64_t*>(p); p += B->big_kmax * 8;
            sc.tmp = reinterpret_cast<uint64_t*>(p); p += B->big_kmax * 8;
            sc.bkt = reinterpret_cast<uint32_t*>(p); p += B->big_kmax * 4;
            sc.arr = reinterpret_cast<uint32_t*>(p); p += B->big_kmax * 4;
            sc.cnt = reinterpret_cast<uint32_t*>(p);
            sc.kmax = B->big_kmax;
            if (wr) rs::batch_big_kernel<true><<<1, rs::kBigThreads, 0, st>>>(V, G.ovf, G.ovf + G.nleaves, sc);
            else rs::batch_big_kernel<false><<<1, rs::kBigThreads, 0, st>>>(V, G.ovf, G.ovf + G.nleaves, sc);
            ++nl;
        }
    }
    *launches = nl;
    return cuda_rc(cudaGetLastError());
}

struct Guard {
    int prev = -1;
    bool ok = false;
    explicit Guard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~Guard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

// Internal hooks from rs_capi.cu.
namespace rs {
int ctx_device(rs_ctx* ctx);
int ctx_sms(rs_ctx* ctx);
const double* ctx_tab(rs_ctx* ctx);
void ctx_count_launches(rs_ctx* ctx, uint64_t n);
}  // namespace rs

extern "C" {

int rs_batch_destroy(rs_batchplan* B) {
    if (!B) return RS_OK;
    Guard g(B->device);
    cudaDeviceSynchronize();
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->capture_stream) cudaStreamDestroy(B->capture_stream);
    cudaFree(B->reqs);
    cudaFree(B->nodes);
    for (auto& lv : B->levels) cudaFree(lv.first);
    for (Group& G : B->groups) {
        cudaFree(G.req_of);
        cudaFree(G.prefix);
        cudaFree(G.ovf);
    }
    cudaFree(B->big_pool);
    delete B;
    return RS_OK;
}

int rs_batch_plan(rs_ctx* ctx, const rs_request* reqs, uint32_t R, rs_batchplan** out) {
    if (!ctx || !out || (R > 0 && !reqs)) return RS_EINVAL;
    *out = nullptr;
    Guard g(rs::ctx_device(ctx));
    if (!g.ok) return RS_ECUDA;
    rs_batchplan* B = new (std::nothrow) rs_batchplan();
    if (!B) return RS_ENOMEM;
    B->device = rs::ctx_device(ctx);
    B->sms = rs::ctx_sms(ctx);
    B->tab = rs::ctx_tab(ctx);
    B->R = R;
    std::vector<rs::BatchReq> h(R);
    uint64_t nodes = 0, bound = 0;
    int Dmax = -1;
    std::vector<uint32_t> req_of[5];
    std::vector<uint64_t> prefix[5];
    auto group_of = [](uint32_t kind, bool wide) { return kind == RS_KIND_B ? 4 : (int)kind * 2 + (wide ? 1 : 0); };
    for (uint32_t r = 0; r < R; ++r) {
        const rs_request& q = reqs[r];
        rs::BatchReq& b = h[r];
        b.n = q.n;
        b.N = q.N;
        b.seed = q.seed;
        b.out_off = q.out_off;
        b.n0 = q.n0;
        b.kind = q.kind;
        b.D = -1;
        b.node_base = 0;
        b.status0 = RS_OK;
        const bool wr = q.kind == RS_KIND_WR;
        if (q.kind > RS_KIND_B || q.n0 == 0 || q.N > (1ull << 62) || (q.n > 0 && q.N == 0) || (!wr && q.n > q.N)) {
            b.status0 = RS_EINVAL;
            continue;
        }
        if (q.n == 0) continue;
        const int D = depth_for(q.n, q.N, q.n0);
        if (D > rs::kMaxDepth) {
            b.status0 = RS_ECAPACITY;
            continue;
        }
        b.D = D;
        b.node_base = nodes;
        nodes += 2ull << D;
        Dmax = std::max(Dmax, D);
        const uint64_t nleaves = 1ull << D;
        const uint64_t smax = (q.N >> D) + ((q.N & (nleaves - 1)) ? 1 : 0);
        const int gi = group_of(q.kind, smax > (1ull << 32));
        if (prefix[gi].empty()) prefix[gi].push_back(0);
        req_of[gi].push_back(r);
        prefix[gi].push_back(prefix[gi].back() + nleaves);
        if (q.kind != RS_KIND_B) bound = std::max<uint64_t>(bound, wr ? q.n : std::min<uint64_t>(q.n, smax - smax / 2));
    }
    int rc = upload(&B->reqs, h);
    if (!rc && nodes) rc = cuda_rc(cudaMalloc(&B->nodes, nodes * sizeof(rs::NodeRec)));
    // tree levels: warp items of up to kBatchTreeBatch consecutive nodes
    for (int level = 0; !rc && level < Dmax; ++level) {
        std::vector<rs::BatchTreeItem> items;
        const uint64_t cnt = 1ull << level;
        const uint32_t per = (uint32_t)std::min<uint64_t>(cnt, rs::kBatchTreeBatch);
        for (uint32_t r = 0; r < R; ++r) {
            if (h[r].D <= level) continue;
            for (uint64_t s = 0; s < cnt; s += per)
                items.push_back(rs::BatchTreeItem{r, (uint32_t)std::min<uint64_t>(per, cnt - s), cnt + s});
        }
        rs::BatchTreeItem* d = nullptr;
        rc = upload(&d, items);
        if (!rc) B->levels.emplace_back(d, (uint32_t)items.size());
    }
    for (int gi = 0; !rc && gi < 5; ++gi) {
        Group& G = B->groups[gi];
        G.kind = gi == 4 ? RS_KIND_B : gi / 2;
        G.wide = gi < 4 && (gi & 1);
        G.m = (uint32_t)req_of[gi].size();
        if (G.m == 0) continue;
        G.nleaves = prefix[gi].back();
        rc = upload(&G.req_of, req_of[gi]);
        if (!rc) rc = upload(&G.prefix, prefix[gi]);
        if (!rc && G.kind != RS_KIND_B) rc = cuda_rc(cudaMalloc(&G.ovf, (G.nleaves + 1) * sizeof(uint32_t)));
    }
    if (!rc && bound > 64) {
        B->big_kmax = std::min<uint64_t>(bound, rs::kBigLeafMax);
        rc = cuda_rc(cudaMalloc(&B->big_pool, rs::big_pool_bytes(B->big_kmax)));
    }
    if (rc) {
        rs_batch_destroy(B);
        return rc;
    }
    *out = B;
    return RS_OK;
}

int rs_batch_run(rs_batchplan* B, uint64_t* out_pool_dev, int32_t* status_dev, void* stream) {
    if (!B || !status_dev) return RS_EINVAL;
    if (((uintptr_t)out_pool_dev & 7) != 0) return RS_EINVAL;
    Guard g(B->device);
    if (!g.ok) return RS_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!B->ran_eagerly) {
        // first run: plain launches (this also sets the kernels' attributes)
        uint64_t nl = 0;
        int rc = issue_run(B, out_pool_dev, status_dev, st, &nl);
        B->launches_per_run = nl;
        B->ran_eagerly = true;
        return rc;
    }
    if (!B->exec || B->graph_pool != out_pool_dev || B->graph_status != status_dev) {
        if (B->exec) {
            cudaGraphExecDestroy(B->exec);
            B->exec = nullptr;
        }
        if (!B->capture_stream && cudaStreamCreateWithFlags(&B->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
            return RS_ECUDA;
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(B->capture_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return RS_ECUDA;
        uint64_t nl = 0;
        const int rc = issue_run(B, out_pool_dev, status_dev, B->capture_stream, &nl);
        const cudaError_t e = cudaStreamEndCapture(B->capture_stream, &graph);
        if (rc || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return rc ? rc : RS_ECUDA;
        }
        const cudaError_t ei = cudaGraphInstantiate(&B->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) return RS_ECUDA;
        B->graph_pool = out_pool_dev;
        B->graph_status = status_dev;
    }
    return cuda_rc(cudaGraphLaunch(B->exec, st));
}

int rs_batch_launch_count(rs_batchplan* B, uint64_t* per_run) {
    if (!B || !per_run) return RS_EINVAL;
    *per_run = B->launches_per_run;
    return RS_OK;
}

int rs_batch_tune(rs_batchplan* B, uint64_t* out_pool_dev, int32_t* status_dev, void* stream) {
    if (!B || !status_dev) return RS_EINVAL;
    Guard g(B->device);
    if (!g.ok) return RS_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return RS_ECUDA;
    // Output-invariant knob: leaf blocks per SM (the leaf-to-block schedule
    // does not change any value).  Try each setting on the whole run.
    int best = 0;
    float best_ms = 1e30f;
    for (int per : {0, 4, 3, 2, 1}) {
        for (Group& G : B->groups) G.grid_per_sm = per;
        uint64_t nl = 0;
        int rc = issue_run(B, out_pool_dev, status_dev, st, &nl);   // warm
        cudaEventRecord(e0, st);
        if (!rc) rc = issue_run(B, out_pool_dev, status_dev, st, &nl);
        cudaEventRecord(e1, st);
        if (rc || cudaEventSynchronize(e1) != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return rc ? rc : RS_ECUDA;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best = per;
        }
    }
    for (Group& G : B->groups) G.grid_per_sm = best;
    if (B->exec) {
        cudaGraphExecDestroy(B->exec);
        B->exec = nullptr;
    }
    B->ran_eagerly = true;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return RS_OK;
}

int rs_batch(rs_ctx* ctx, const rs_request* reqs_dev, uint32_t R, uint64_t* out_pool_dev, int32_t* status_dev,
             void* stream) {
    if (!ctx || (R > 0 && !reqs_dev) || !status_dev) return RS_EINVAL;
    if (R == 0) return RS_OK;
    Guard g(rs::ctx_device(ctx));
    if (!g.ok) return RS_ECUDA;
    std::vector<rs_request> h(R);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(h.data(), reqs_dev, R * sizeof(rs_request), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return RS_ECUDA;
    rs_batchplan* B = nullptr;
    int rc = rs_batch_plan(ctx, h.data(), R, &B);
    if (rc) return rc;
    rc = rs_batch_run(B, out_pool_dev, status_dev, stream);
    if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = RS_ECUDA;
    rs::ctx_count_launches(ctx, B->launches_per_run);
    rs_batch_destroy(B);
    return rc;
}

}  // extern "C"
