// rs_query.cu -- resident split trees and online sorted range queries.
//
// A resident tree keeps the leaf records (lo, s, n', offset) of one sample's
// split tree in device memory (Sec. 3.1 Algorithm R, Sec. 4.5: they fix
// every leaf's share and output position).  A query for the values in
// [a, b) regenerates only the leaves whose ranges overlap [a, b) -- each
// leaf's sample is a function of its record and id alone -- and writes the
// values in range, in increasing order: the sorted, online generation of a
// contiguous piece of the sample (Sec. 4.1), without producing the rest.
#include <cstring>
#include <new>

#include "rs_group.h"

namespace rs {
int ctx_device(rs_ctx* ctx);
int ctx_sms(rs_ctx* ctx);
const double* ctx_tab(rs_ctx* ctx);
void ctx_count_launches(rs_ctx* ctx, uint64_t n);
int ctx_build_tree(rs_ctx* ctx, uint64_t n, uint64_t N, uint64_t seed, uint32_t n0, int kind, cudaStream_t st,
                   int* D, NodeRec** nodes);

// Largest leaf count and largest leaf selection (the count, or for leaves
// written as a complement, the complement's size) over the leaves.
__global__ void leaf_stats_kernel(const NodeRec* __restrict__ leaves, uint64_t nleaves, int with_replacement,
                                  unsigned long long* __restrict__ out) {
    unsigned long long mc = 0, mk = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nleaves;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const NodeRec r = leaves[i];
        const uint64_t k = (!with_replacement && r.c > r.S - r.c) ? r.S - r.c : r.c;
        mc = r.c > mc ? r.c : mc;
        mk = k > mk ? k : mk;
    }
    for (int o = 16; o > 0; o >>= 1) {
        mc = max(mc, __shfl_xor_sync(0xFFFFFFFFu, mc, o));
        mk = max(mk, __shfl_xor_sync(0xFFFFFFFFu, mk, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&out[0], mc);
        atomicMax(&out[1], mk);
    }
}

}  // namespace rs

struct rs_tree {
    rs_ctx* ctx = nullptr;
    int device = 0;
    int sms = 0;
    uint64_t n = 0;
    rs::TreeInfo info{};
    rs::NodeRec* leaves = nullptr;
    // single-query workspace, grown on demand
    unsigned char* up = nullptr;
    uint64_t up_cap = 0;
    unsigned char* work = nullptr;
    uint64_t work_cap = 0;
    void* big = nullptr;
    uint64_t big_cap = 0;
    unsigned char* img = nullptr;   // pinned upload image
    uint64_t img_cap = 0;
    rs::QueryRes* res_host = nullptr;   // pinned
};

namespace {

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

int cuda_rc(cudaError_t e) {
    if (e == cudaSuccess) return RS_OK;
    return e == cudaErrorMemoryAllocation ? RS_ENOMEM : RS_ECUDA;
}

int grow_dev(unsigned char*& p, uint64_t& cap, uint64_t need) {
    if (cap >= need) return RS_OK;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    int rc = cuda_rc(cudaMalloc(&p, need));
    if (!rc) cap = need;
    return rc;
}

int grow_host(unsigned char*& p, uint64_t& cap, uint64_t need) {
    if (cap >= need) return RS_OK;
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
    int rc = cuda_rc(cudaMallocHost(&p, need));
    if (!rc) cap = need;
    return rc;
}

}  // namespace

namespace rs {
// Tree description for the server (rs_serve.cu).
const TreeInfo* tree_info(const rs_tree* t) { return &t->info; }
int tree_device(const rs_tree* t) { return t->device; }
uint64_t tree_samples(const rs_tree* t) { return t->n; }
}  // namespace rs

extern "C" {

int rs_tree_destroy(rs_tree* t) {
    if (!t) return RS_OK;
    Guard g(t->device);
    int rc = cuda_rc(cudaDeviceSynchronize());
    cudaFree(t->leaves);
    cudaFree(t->up);
    cudaFree(t->work);
    cudaFree(t->big);
    if (t->img) cudaFreeHost(t->img);
    if (t->res_host) cudaFreeHost(t->res_host);
    delete t;
    return rc;
}

int rs_tree_create(rs_ctx* ctx, uint64_t n, uint64_t N, uint64_t seed, uint32_t n0, int kind, void* stream,
                   rs_tree** out) {
    if (!ctx || !out) return RS_EINVAL;
    *out = nullptr;
    const bool wr = kind == RS_KIND_WR;
    if (kind < RS_KIND_H || kind > RS_KIND_B || n0 == 0 || N > (1ull << 62) || (n > 0 && N == 0) || (!wr && n > N))
        return RS_EINVAL;
    const int D = rs::plan_depth(n, N, n0);
    if (D > rs::kMaxDepth) return RS_ECAPACITY;
    Guard g(rs::ctx_device(ctx));
    if (!g.ok) return RS_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rs_tree* t = new (std::nothrow) rs_tree();
    if (!t) return RS_ENOMEM;
    t->ctx = ctx;
    t->device = rs::ctx_device(ctx);
    t->sms = rs::ctx_sms(ctx);
    t->n = n;
    const uint64_t nleaves = 1ull << D;
    const uint64_t smax = N == 0 ? 0 : (N >> D) + ((N & (nleaves - 1)) ? 1 : 0);
    t->info.N = N;
    t->info.seed = seed;
    t->info.D = D;
    t->info.kind = kind;
    t->info.wide = smax > (1ull << 32);
    int rc = cuda_rc(cudaMalloc(&t->leaves, nleaves * sizeof(rs::NodeRec)));
    if (!rc) rc = cuda_rc(cudaMallocHost(&t->res_host, sizeof(rs::QueryRes)));
    unsigned long long* stats = nullptr;
    if (!rc) rc = cuda_rc(cudaMalloc(&stats, 2 * sizeof(unsigned long long)));
    if (!rc && n > 0) {
        int Dt = 0;
        rs::NodeRec* nodes = nullptr;
        rc = rs::ctx_build_tree(ctx, n, N, seed, n0, kind, st, &Dt, &nodes);
        if (!rc)
            rc = cuda_rc(cudaMemcpyAsync(t->leaves, nodes + nleaves, nleaves * sizeof(rs::NodeRec),
                                         cudaMemcpyDeviceToDevice, st));
        if (!rc) rc = cuda_rc(cudaMemsetAsync(stats, 0, 2 * sizeof(unsigned long long), st));
        if (!rc) {
            const unsigned blocks = (unsigned)std::min<uint64_t>((nleaves + 255) / 256, 1024);
            rs::leaf_stats_kernel<<<blocks, 256, 0, st>>>(t->leaves, nleaves, wr ? 1 : 0, stats);
            rs::ctx_count_launches(ctx, 1);
            rc = cuda_rc(cudaGetLastError());
        }
        unsigned long long h[2] = {0, 0};
        if (!rc) rc = cuda_rc(cudaMemcpyAsync(h, stats, sizeof(h), cudaMemcpyDeviceToHost, st));
        if (!rc) rc = rs_sync(ctx, stream);   // waits; a device error of the tree build ends the call
        t->info.maxc = h[0];
        t->info.maxk = h[1];
    }
    cudaFree(stats);
    t->info.leaves = t->leaves;
    if (rc) {
        rs_tree_destroy(t);
        return rc;
    }
    *out = t;
    return RS_OK;
}

int rs_tree_query(rs_tree* t, uint64_t a, uint64_t b, uint64_t* out_dev, uint64_t cap, uint64_t* count_out,
                  void* stream) {
    if (!t || !count_out) return RS_EINVAL;
    *count_out = 0;
    if (cap > 0 && (!out_dev || ((uintptr_t)out_dev & 7))) return RS_EINVAL;
    const uint64_t lo = a < 1 ? 1 : a;
    const uint64_t hi = b > t->info.N + 1 ? t->info.N + 1 : b;
    if (t->n == 0 || lo >= hi) return RS_OK;
    Guard g(t->device);
    if (!g.ok) return RS_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = RS_OK;
    try {
        rs::GroupPlan plan;
        const rs::GroupQuery q{&t->info, lo, hi, out_dev, cap};
        plan.build(nullptr, nullptr, 0, &q, 1);
        rc = grow_dev(t->up, t->up_cap, plan.upload_bytes());
        if (!rc) rc = grow_dev(t->work, t->work_cap, plan.work_bytes());
        if (!rc) rc = grow_host(t->img, t->img_cap, plan.upload_bytes());
        const uint64_t big_bytes = plan.big_kmax() ? rs::big_pool_bytes(plan.big_kmax()) : 0;
        if (!rc && big_bytes > t->big_cap) {
            unsigned char* p = static_cast<unsigned char*>(t->big);
            rc = grow_dev(p, t->big_cap, big_bytes);
            t->big = p;
        }
        if (rc) return rc;
        plan.bind(t->up, t->work, t->big, t->img);
        rc = cuda_rc(cudaMemcpyAsync(t->up, t->img, plan.upload_bytes(), cudaMemcpyHostToDevice, st));
        uint64_t nl = 0;
        if (!rc) rc = plan.issue(rs::ctx_tab(t->ctx), t->sms, nullptr, nullptr, st, &nl);
        rs::ctx_count_launches(t->ctx, nl);
        if (!rc)
            rc = cuda_rc(cudaMemcpyAsync(t->res_host, plan.query_results(), sizeof(rs::QueryRes),
                                         cudaMemcpyDeviceToHost, st));
        if (!rc) rc = cuda_rc(cudaStreamSynchronize(st));
    } catch (const std::bad_alloc&) {
        rc = RS_ENOMEM;
    }
    if (rc) return rc;
    *count_out = t->res_host->count;
    return t->res_host->status;
}

int rs_tree_info(rs_tree* t, int* depth, uint64_t* max_leaf_count) {
    if (!t || !depth || !max_leaf_count) return RS_EINVAL;
    *depth = t->info.D;
    *max_leaf_count = t->info.maxc;
    return RS_OK;
}

}  // extern "C"
