// rs_capi.cu -- the C ABI declared in include/rs.h.
//
// Host side of the sampler: argument checks, the plan (tree depth), scratch
// memory, and the launch sequence tree -> leaves on the caller's stream.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "rs_bern.h"
#include "rs_internal.h"
#include "rs_points.h"
#include "rs_union.h"

namespace rs {
// Kernel launches that launch_tree_top(..., levels, ...) issues (rs_tree.cu).
uint64_t tree_launches(int levels);
}  // namespace rs

struct rs_ctx {
    int device = 0;
    int sms = 0;
    double* tab = nullptr;          // ln i!, i < 256
    int* status = nullptr;          // first device-side error
    rs::NodeRec* nodes = nullptr;   // heap-numbered node records
    uint64_t nodes_cap = 0;         // records
    uint32_t* ovf = nullptr;        // overflow list + its counter
    uint64_t ovf_cap = 0;           // words
    void* big_pool = nullptr;
    uint64_t big_pool_bytes = 0;
    uint64_t* words = nullptr;      // general scratch (Bernoulli chunk counts, leaf B positions)
    uint64_t words_cap = 0;
    uint64_t* boxes = nullptr;      // box records of the multi-dimensional sampler
    uint64_t boxes_cap = 0;         // words
    uint64_t* stage = nullptr;      // Bernoulli: positions staged per chunk by the single walk
    uint64_t stage_cap = 0;
    uint64_t stage_max_words = 1ull << 31;   // rs_set_bernoulli_staging
    uint64_t stage_slots = 0;
    uint32_t leaf_cap = 0;          // testing knob, 0 = default
    bool guard = true;              // guarded fast paths of the deviates and skips (rs_set_exact_deviates)
    // pipelining of deep trees: 2^pipe_log2 subtrees, each built on the tree
    // stream while the caller's stream runs the leaves of the ones before
    int pipe_log2 = 0;
    int pipe_leaf_blocks = 3;       // leaf blocks per SM while tree work may run beside them (off by default:
                                    // on GB300 the issue-bound leaves starve the tree blocks)
    cudaStream_t tree_stream = nullptr;
    cudaEvent_t ev_fork = nullptr;
    std::vector<cudaEvent_t> ev_part;
    // copies of the sample to host memory while it is produced
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_copied = nullptr;
    uint64_t* bounds_dev = nullptr;     // output offsets at part boundaries
    uint64_t* bounds_host = nullptr;    // pinned
    bool profiling = false;
    struct PhaseRec {               // event indices of one profiled call
        size_t start, tree_end, end;
        std::vector<std::pair<size_t, size_t>> leaves;
    };
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<PhaseRec> prof_calls;
    uint64_t launches = 0;
};

namespace {

// Makes ctx->device current for the duration of a call, then restores the
// caller's device.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

int cuda_rc(cudaError_t e) {
    if (e == cudaSuccess) return RS_OK;
    if (e == cudaErrorMemoryAllocation) return RS_ENOMEM;
    return RS_ECUDA;
}

// Grows a device buffer to at least `need` elements (contents not kept).
template <typename T>
int ensure(T*& ptr, uint64_t& cap, uint64_t need) {
    if (cap >= need) return RS_OK;
    if (ptr) {
        cudaError_t e = cudaFree(ptr);   // synchronizes the device
        ptr = nullptr;
        cap = 0;
        if (e != cudaSuccess) return RS_ECUDA;
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, need * sizeof(T));
    if (e != cudaSuccess) return cuda_rc(e);
    ptr = static_cast<T*>(p);
    cap = need;
    return RS_OK;
}

// Records the next event of the profiling pool on `st` and returns its
// index (events are created on demand and reused after rs_set_profiling).
size_t record_event(rs_ctx* ctx, cudaStream_t st) {
    while (ctx->ev_pool.size() <= ctx->ev_used) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            ctx->profiling = false;
            return 0;
        }
        ctx->ev_pool.push_back(e);
    }
    cudaEventRecord(ctx->ev_pool[ctx->ev_used], st);
    return ctx->ev_used++;
}

constexpr int kCopyParts = 8;   // pieces of a sample copied to the host while the next ones are made

// Output offsets of the first leaf of each of `parts` equal runs of leaves,
// then n: the pieces of the output the leaves of each run write.
__global__ void part_bounds_kernel(const rs::NodeRec* __restrict__ leaves, uint64_t per_part, uint32_t parts,
                                   uint64_t n, uint64_t* __restrict__ bounds) {
    const uint32_t j = threadIdx.x;
    if (j < parts) bounds[j] = leaves[(uint64_t)j * per_part].off;
    if (j == parts) bounds[j] = n;
}

int ensure_copy(rs_ctx* ctx, size_t parts) {
    if (!ctx->copy_stream && cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
        return RS_ECUDA;
    if (!ctx->ev_copied && cudaEventCreateWithFlags(&ctx->ev_copied, cudaEventDisableTiming) != cudaSuccess)
        return RS_ECUDA;
    if (!ctx->bounds_dev && cudaMalloc(&ctx->bounds_dev, 65 * sizeof(uint64_t)) != cudaSuccess) return RS_ENOMEM;
    if (!ctx->bounds_host && cudaMallocHost(&ctx->bounds_host, 65 * sizeof(uint64_t)) != cudaSuccess)
        return RS_ENOMEM;
    while (ctx->ev_part.size() < parts) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return RS_ECUDA;
        ctx->ev_part.push_back(e);
    }
    return RS_OK;
}

// The tree stream (highest priority) and its events, made on first use.
int ensure_pipeline(rs_ctx* ctx, size_t parts) {
    if (!ctx->tree_stream) {
        int least = 0, greatest = 0;
        if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) return RS_ECUDA;
        if (cudaStreamCreateWithPriority(&ctx->tree_stream, cudaStreamNonBlocking, greatest) != cudaSuccess)
            return RS_ECUDA;
    }
    if (!ctx->ev_fork && cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess)
        return RS_ECUDA;
    while (ctx->ev_part.size() < parts) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return RS_ECUDA;
        ctx->ev_part.push_back(e);
    }
    return RS_OK;
}

int depth_of(uint64_t n, uint64_t N, uint32_t n0) { return rs::tree_depth(n, N, n0); }

int check_sample_args(uint64_t n, uint64_t N, uint32_t n0, bool with_replacement, const void* out) {
    if (n0 == 0) return RS_EINVAL;
    if (N > (1ull << 62)) return RS_EINVAL;
    if (n > 0 && N == 0) return RS_EINVAL;
    if (!with_replacement && n > N) return RS_EINVAL;
    if (n > 0 && out == nullptr) return RS_EINVAL;
    if (out && ((uintptr_t)out & 7)) return RS_EINVAL;
    return RS_OK;
}

// Builds the split tree for (n, N, seed, n0) into ctx->nodes.  kind selects
// binomial (RS_KIND_WR) or hypergeometric splits.
int build_tree(rs_ctx* ctx, uint64_t n, uint64_t N, uint64_t seed, uint32_t n0, int kind, cudaStream_t st,
               int* D_out) {
    const int D = depth_of(n, N, n0);
    if (D > rs::kMaxDepth) return RS_ECAPACITY;
    int rc = ensure(ctx->nodes, ctx->nodes_cap, 2ull << D);
    if (rc) return rc;
    *D_out = D;
    ctx->launches += rs::tree_launches(D);
    return cuda_rc(rs::launch_tree(ctx->nodes, n, N, seed, D, kind == RS_KIND_WR, ctx->tab, ctx->status, st, ctx->guard));
}

int sample_impl(rs_ctx* ctx, uint64_t n, uint64_t N, uint64_t seed, uint32_t n0, int kind, uint64_t* out,
                void* stream, uint64_t* host_out = nullptr) {
    if (!ctx) return RS_EINVAL;
    int rc = check_sample_args(n, N, n0, kind == RS_KIND_WR, out);
    if (rc || n == 0) return rc;
    DeviceGuard g(ctx->device);
    if (!g.ok) return RS_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int D = depth_of(n, N, n0);
    if (D > rs::kMaxDepth) return RS_ECAPACITY;
    rc = ensure(ctx->nodes, ctx->nodes_cap, 2ull << D);
    if (rc) return rc;
    const bool wr = kind == RS_KIND_WR;
    const uint64_t nleaves = 1ull << D;
    // Deep trees: the subtrees under level c are built one after another on
    // the tree stream, and the leaves of each start on `st` as soon as its
    // subtree is done, beside the FP64 work of the next subtrees.
    const int c = (!host_out && ctx->pipe_log2 > 0 && D >= ctx->pipe_log2 + 9) ? ctx->pipe_log2 : 0;
    // copying to the host: the leaves run in pieces, each copied as soon as it is done
    const int cc = host_out ? std::min(D, 3) : 0;
    const uint64_t parts = 1ull << (c + cc), per_part = nleaves >> (c + cc);
    if (c) {
        rc = ensure_pipeline(ctx, parts);
        if (rc) return rc;
    }
    if (host_out) {
        rc = ensure_copy(ctx, parts);
        if (rc) return rc;
    }
    size_t prof = 0;
    if (ctx->profiling) {
        ctx->prof_calls.emplace_back();
        prof = ctx->prof_calls.size();
        ctx->prof_calls[prof - 1].start = record_event(ctx, st);
    }
    if (c == 0) {
        rc = cuda_rc(rs::launch_tree(ctx->nodes, n, N, seed, D, wr, ctx->tab, ctx->status, st, ctx->guard));
        ctx->launches += rs::tree_launches(D);
        if (prof) ctx->prof_calls[prof - 1].tree_end = record_event(ctx, st);
    } else {
        cudaStream_t ts = ctx->tree_stream;
        rc = cuda_rc(cudaEventRecord(ctx->ev_fork, st));
        if (!rc) rc = cuda_rc(cudaStreamWaitEvent(ts, ctx->ev_fork, 0));
        if (!rc) rc = cuda_rc(rs::launch_tree_top(ctx->nodes, n, N, seed, c, wr, ctx->tab, ctx->status, ts, ctx->guard));
        for (uint64_t j = 0; !rc && j < parts; ++j) {
            rc = cuda_rc(rs::launch_tree_part(ctx->nodes, seed, D, c, j, wr, ctx->tab, ctx->status, ts, ctx->guard));
            if (!rc) rc = cuda_rc(cudaEventRecord(ctx->ev_part[j], ts));
        }
        ctx->launches += rs::tree_launches(c) + parts * (uint64_t)(D - c);
        if (prof) ctx->prof_calls[prof - 1].tree_end = record_event(ctx, ts);
    }
    if (rc) return rc;
    if (host_out) {
        // where each piece of the output starts: known once the tree is done
        part_bounds_kernel<<<1, 128, 0, st>>>(ctx->nodes + nleaves, per_part, (uint32_t)parts, n, ctx->bounds_dev);
        ctx->launches += 1;
        rc = cuda_rc(cudaMemcpyAsync(ctx->bounds_host, ctx->bounds_dev, (parts + 1) * sizeof(uint64_t),
                                     cudaMemcpyDeviceToHost, st));
        if (!rc) rc = cuda_rc(cudaStreamSynchronize(st));
        if (rc) return rc;
    }
    const uint64_t smax = (N >> D) + ((N & (nleaves - 1)) ? 1 : 0);
    rs::LeafLaunch L{};
    uint64_t big_kmax = 0;
    if (kind != RS_KIND_B) {
        rc = ensure(ctx->ovf, ctx->ovf_cap, nleaves + 1);
        if (rc) return rc;
        // Largest selection any leaf can need: k <= n and, without
        // replacement, k <= s/2 (the complement rule).  A leaf also leaves
        // the fast path when a complement does not fit the bitmap or a probe
        // runs past the table: keep the general path ready whenever a leaf
        // can hold more than a handful of values.
        uint64_t bound = n;
        if (!wr) bound = std::min<uint64_t>(bound, smax - smax / 2);
        if (bound > 64) {
            big_kmax = std::min<uint64_t>(bound, rs::kBigLeafMax);
            const uint64_t bytes = rs::big_pool_bytes(big_kmax);
            if (ctx->big_pool_bytes < bytes) {
                if (ctx->big_pool) cudaFree(ctx->big_pool);
                ctx->big_pool = nullptr;
                ctx->big_pool_bytes = 0;
                cudaError_t e = cudaMalloc(&ctx->big_pool, bytes);
                if (e != cudaSuccess) return cuda_rc(e);
                ctx->big_pool_bytes = bytes;
            }
        }
        L.seed = seed;
        L.smax = smax;
        L.out = out;
        L.status = ctx->status;
        L.ovf_list = ctx->ovf;
        L.ovf_count = ctx->ovf + nleaves;
        L.big_pool = ctx->big_pool;
        L.big_kmax = big_kmax;
        L.cap = ctx->leaf_cap;
        L.mean_count = n >> D;
        L.pow2_leaves = (N & (nleaves - 1)) == 0 && (smax & (smax - 1)) == 0;
        L.sms = ctx->sms;
        L.with_replacement = wr;
    }
    for (uint64_t j = 0; !rc && j < parts; ++j) {
        if (c) rc = cuda_rc(cudaStreamWaitEvent(st, ctx->ev_part[j], 0));
        if (rc) break;
        const size_t a = prof ? record_event(ctx, st) : 0;
        const uint64_t first = j * per_part;
        if (kind == RS_KIND_B) {
            rs::LeafBLaunch LB{ctx->nodes + nleaves + first, per_part, nleaves + first, seed, out, ctx->status,
                               ctx->sms, ctx->tab, smax, ctx->guard};
            ctx->launches += 1;
            rc = cuda_rc(rs::launch_leaves_b(LB, st));
        } else {
            L.leaves = ctx->nodes + nleaves + first;
            L.nleaves = per_part;
            L.first_id = nleaves + first;
            L.blocks_per_sm = (c && j + 1 < parts) ? ctx->pipe_leaf_blocks : 0;
            ctx->launches += big_kmax ? 2 : 1;
            rc = cuda_rc(rs::launch_leaves(L, st));
        }
        if (prof) {
            const size_t b = record_event(ctx, st);
            ctx->prof_calls[prof - 1].leaves.emplace_back(a, b);
            ctx->prof_calls[prof - 1].end = b;
        }
        if (!rc && host_out) {
            const uint64_t b0 = ctx->bounds_host[j], b1 = ctx->bounds_host[j + 1];
            rc = cuda_rc(cudaEventRecord(ctx->ev_part[j], st));
            if (!rc) rc = cuda_rc(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_part[j], 0));
            if (!rc && b1 > b0)
                rc = cuda_rc(cudaMemcpyAsync(host_out + b0, out + b0, (b1 - b0) * sizeof(uint64_t),
                                             cudaMemcpyDeviceToHost, ctx->copy_stream));
        }
    }
    if (!rc && host_out) {
        // later work on `stream` (and rs_sync) waits for the copies
        rc = cuda_rc(cudaEventRecord(ctx->ev_copied, ctx->copy_stream));
        if (!rc) rc = cuda_rc(cudaStreamWaitEvent(st, ctx->ev_copied, 0));
    }
    return rc;
}

}  // namespace

namespace rs {
static std::vector<CapsWriter>& caps_writers() {
    static std::vector<CapsWriter> v;
    return v;
}
int register_caps_writer(CapsWriter w) {
    caps_writers().push_back(w);
    return 1;
}
int tree_depth(uint64_t n, uint64_t N, uint32_t n0) {
    int D = 0;
    while ((unsigned __int128)n > ((unsigned __int128)n0 << D)) ++D;
    while (D > 0 && ((unsigned __int128)1 << D) > (unsigned __int128)N) --D;
    return D;
}
// Accessors for the other translation units (the batch planner).
int ctx_device(rs_ctx* ctx) { return ctx->device; }
int ctx_sms(rs_ctx* ctx) { return ctx->sms; }
const double* ctx_tab(rs_ctx* ctx) { return ctx->tab; }
void ctx_count_launches(rs_ctx* ctx, uint64_t n) { ctx->launches += n; }
// Builds the split tree of (n, N, seed, n0) in the context's node records
// (leaves at (*nodes)[2^D ..)); valid until the context's next call.
int ctx_build_tree(rs_ctx* ctx, uint64_t n, uint64_t N, uint64_t seed, uint32_t n0, int kind, cudaStream_t st,
                   int* D, NodeRec** nodes) {
    const int rc = build_tree(ctx, n, N, seed, n0, kind, st, D);
    *nodes = ctx->nodes;
    return rc;
}
}  // namespace rs

extern "C" {

int rs_create(rs_ctx** out, int device) {
    if (!out) return RS_EINVAL;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) return RS_ECUDA;
    DeviceGuard g(device);
    if (!g.ok) return RS_ECUDA;
    rs_ctx* ctx = new (std::nothrow) rs_ctx();
    if (!ctx) return RS_ENOMEM;
    ctx->device = device;
    int rc = RS_OK;
    if (cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) rc = RS_ECUDA;
    if (!rc) rc = cuda_rc(cudaMalloc(&ctx->tab, rs::kTabWords * sizeof(double)));
    if (!rc) rc = cuda_rc(cudaMalloc(&ctx->status, sizeof(int)));
    if (!rc) rc = cuda_rc(cudaMemset(ctx->status, 0, sizeof(int)));
    if (!rc) rc = cuda_rc(rs::launch_lf_table(ctx->tab, 0));
    if (!rc) rc = cuda_rc(cudaDeviceSynchronize());
    if (rc) {
        rs_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return RS_OK;
}

int rs_destroy(rs_ctx* ctx) {
    if (!ctx) return RS_OK;
    DeviceGuard g(ctx->device);
    int rc = cuda_rc(cudaDeviceSynchronize());
    cudaFree(ctx->tab);
    cudaFree(ctx->status);
    cudaFree(ctx->nodes);
    cudaFree(ctx->ovf);
    cudaFree(ctx->big_pool);
    cudaFree(ctx->words);
    cudaFree(ctx->stage);
    cudaFree(ctx->boxes);
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->ev_part) cudaEventDestroy(e);
    if (ctx->ev_copied) cudaEventDestroy(ctx->ev_copied);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    cudaFree(ctx->bounds_dev);
    if (ctx->bounds_host) cudaFreeHost(ctx->bounds_host);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->tree_stream) cudaStreamDestroy(ctx->tree_stream);
    delete ctx;
    return rc;
}

int rs_plan(uint64_t n, uint64_t N, uint32_t n0, int* depth_out) {
    if (!depth_out || n0 == 0) return RS_EINVAL;
    *depth_out = depth_of(n, N, n0);
    return RS_OK;
}

int rs_sample(rs_ctx* ctx, uint64_t n, uint64_t N, uint64_t seed, uint32_t n0, uint64_t* out_dev, void* stream) {
    return sample_impl(ctx, n, N, seed, n0, RS_KIND_H, out_dev, stream);
}

int rs_sample_with_replacement(rs_ctx* ctx, uint64_t n, uint64_t N, uint64_t seed, uint32_t n0, uint64_t* out_dev,
                               void* stream) {
    return sample_impl(ctx, n, N, seed, n0, RS_KIND_WR, out_dev, stream);
}

int rs_sample_b(rs_ctx* ctx, uint64_t n, uint64_t N, uint64_t seed, uint32_t n0, uint64_t* out_dev, void* stream) {
    return sample_impl(ctx, n, N, seed, n0, RS_KIND_B, out_dev, stream);
}

int rs_sample_to_host(rs_ctx* ctx, int kind, uint64_t n, uint64_t N, uint64_t seed, uint32_t n0, uint64_t* out_dev,
                      uint64_t* out_host, void* stream) {
    if (kind < RS_KIND_H || kind > RS_KIND_B || (n > 0 && !out_host)) return RS_EINVAL;
    return sample_impl(ctx, n, N, seed, n0, kind, out_dev, stream, out_host);
}

int rs_split_tree(rs_ctx* ctx, uint64_t n, uint64_t N, uint64_t seed, uint32_t n0, int kind, uint64_t* recs_dev,
                  uint64_t max_leaves, void* stream) {
    if (!ctx || kind < RS_KIND_H || kind > RS_KIND_B) return RS_EINVAL;
    int rc = check_sample_args(n, N, n0, kind == RS_KIND_WR, recs_dev);
    if (rc) return rc;
    if (!recs_dev) return RS_EINVAL;
    const int D = depth_of(n, N, n0);
    if ((1ull << D) > max_leaves) return RS_ECAPACITY;
    if (N == 0) return RS_OK;
    DeviceGuard g(ctx->device);
    if (!g.ok) return RS_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int Dt;
    rc = build_tree(ctx, n, N, seed, n0, kind, st, &Dt);
    if (rc) return rc;
    return cuda_rc(rs::launch_export_leaves(ctx->nodes + (1ull << D), 1ull << D, recs_dev, st));
}

int rs_bernoulli(rs_ctx* ctx, double p, uint64_t N, uint64_t seed, uint32_t n0, uint64_t a, uint64_t b,
                 uint64_t* out_dev, uint64_t cap, uint64_t* count_out, void* stream) {
    if (!ctx || !count_out) return RS_EINVAL;
    *count_out = 0;
    if (!(p >= 0.0 && p <= 1.0) || n0 == 0 || N > (1ull << 62) || a > b || b > N) return RS_EINVAL;
    int c = 0;
    while (c < 62 && ldexp(1.0, c) * p < (double)n0) ++c;
    const uint64_t C = 1ull << c;
    if (a % C != 0 || (b % C != 0 && b != N)) return RS_EINVAL;
    if (cap > 0 && (!out_dev || ((uintptr_t)out_dev & 7))) return RS_EINVAL;
    if (p == 0.0 || a == b) return RS_OK;
    DeviceGuard g(ctx->device);
    if (!g.ok) return RS_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint64_t first = a >> c;
    const uint64_t nchunks = ((b - 1) >> c) - first + 1;
    int rc = ensure(ctx->words, ctx->words_cap, nchunks + 2 + rs::scan_scratch_words(nchunks));
    if (rc) return rc;
    // one walk per chunk with its positions staged (about 1.1 times the
    // output), unless that needs more than the staging limit or cannot be
    // allocated: then a count walk and a write walk
    uint64_t* stage = nullptr;
    const uint64_t per = ctx->stage_slots ? ctx->stage_slots : rs::bern_stage_per(ldexp(1.0, c) * p);
    if (p < 1.0 && per <= ctx->stage_max_words / nchunks) {
        if (ensure(ctx->stage, ctx->stage_cap, nchunks * per) == RS_OK) stage = ctx->stage;
        else (void)cudaGetLastError();
    }
    rs::BernLaunch L{p, N, seed, c, first, nchunks, a, b, out_dev, cap, ctx->words, ctx->words + nchunks + 1,
                     ctx->words + nchunks + 2, ctx->status, ctx->sms, ctx->tab, stage, per, ctx->guard};
    rc = cuda_rc(rs::launch_bernoulli(L, st));
    if (rc) return rc;
    uint64_t total = 0;
    rc = cuda_rc(cudaMemcpyAsync(&total, ctx->words + nchunks + 1, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    if (!rc) rc = cuda_rc(cudaStreamSynchronize(st));
    if (rc) return rc;
    *count_out = total;
    return total > cap ? RS_ECAPACITY : RS_OK;
}

int rs_bernoulli_size(rs_ctx* ctx, double p, uint64_t N, uint64_t seed, uint64_t* count_out, void* stream) {
    if (!ctx || !count_out) return RS_EINVAL;
    *count_out = 0;
    if (!(p >= 0.0 && p <= 1.0) || N > (1ull << 62)) return RS_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return RS_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // p as K / 2^62, K = floor(q 2^62 + 1/2) with q = p or 1 - p (whichever is at most 1/2)
    const bool flip = p > 0.5;
    const double q = flip ? 1.0 - p : p;
    const uint64_t K = (uint64_t)floor(q * 0x1p62 + 0.5);
    int rc = ensure(ctx->words, ctx->words_cap, 1);
    if (rc) return rc;
    rc = cuda_rc(rs::launch_bernoulli_size(seed, N, K, flip, ctx->tab, ctx->words, ctx->status, st));
    ctx->launches += 1;
    if (rc) return rc;
    uint64_t c = 0;
    rc = cuda_rc(cudaMemcpyAsync(&c, ctx->words, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    if (rc) return rc;
    rc = rs_sync(ctx, stream);
    if (rc) return rc;
    *count_out = c;
    return RS_OK;
}

int rs_bernoulli_by_size(rs_ctx* ctx, double p, uint64_t N, uint64_t seed, uint32_t n0, uint64_t a, uint64_t b,
                         uint64_t* out_dev, uint64_t cap, uint64_t* count_out, uint64_t* total_out, void* stream) {
    if (!ctx || !count_out || !total_out) return RS_EINVAL;
    *count_out = 0;
    *total_out = 0;
    if (n0 == 0 || a > b || b > N) return RS_EINVAL;
    if (cap > 0 && (!out_dev || ((uintptr_t)out_dev & 7))) return RS_EINVAL;
    uint64_t n = 0;
    int rc = rs_bernoulli_size(ctx, p, N, seed, &n, stream);
    if (rc) return rc;
    *total_out = n;
    if (n == 0 || a == b) return RS_OK;
    if (a == 0 && b == N) {   // the whole sample
        *count_out = n;
        if (n > cap) return RS_ECAPACITY;
        return rs_sample(ctx, n, N, seed, n0, out_dev, stream);
    }
    rs_tree* tree = nullptr;
    rc = rs_tree_create(ctx, n, N, seed, n0, RS_KIND_H, stream, &tree);
    if (rc) return rc;
    rc = rs_tree_query(tree, a + 1, b + 1, out_dev, cap, count_out, stream);
    const int rd = rs_tree_destroy(tree);
    return rc ? rc : rd;
}

namespace {
constexpr uint32_t kUnionMaxSegments = 1u << 24;
constexpr uint64_t kUnionWeyl = 0x9E3779B97F4A7C15ull;

// Validates the segments and runs the count tree; counts_host[i] = segment
// i's count.  *total_out = the union's size.
int union_counts(rs_ctx* ctx, const uint64_t* L_host, uint32_t p, uint64_t n, uint64_t seed,
                 uint64_t* counts_host, cudaStream_t st) {
    if (p > kUnionMaxSegments || (p > 0 && (!L_host || !counts_host))) return RS_EINVAL;
    unsigned __int128 total = 0;
    for (uint32_t i = 0; i < p; ++i) total += L_host[i];
    if (total > ((unsigned __int128)1 << 62) || n > (uint64_t)total) return RS_EINVAL;
    if (p == 0) return RS_OK;
    int log2P = 0;
    while ((1ull << log2P) < p) ++log2P;
    const uint64_t P = 1ull << log2P;
    int rc = ensure(ctx->words, ctx->words_cap, p + 4 * P);
    if (rc) return rc;
    uint64_t* L = ctx->words;
    uint64_t* sum = L + p;
    uint64_t* cnt = sum + 2 * P;
    rc = cuda_rc(cudaMemcpyAsync(L, L_host, p * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
    if (rc) return rc;
    rc = cuda_rc(rs::launch_union_counts(L, p, log2P, n, seed, sum, cnt, ctx->tab, ctx->status, st));
    ctx->launches += 1 + 2 * (uint64_t)log2P;
    if (rc) return rc;
    rc = cuda_rc(cudaMemcpyAsync(counts_host, cnt + P, p * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    if (rc) return rc;
    return rs_sync(ctx, st);
}
}  // namespace

int rs_union_counts(rs_ctx* ctx, const uint64_t* L_host, uint32_t p, uint64_t n, uint64_t seed,
                    uint64_t* counts_host, void* stream) {
    if (!ctx) return RS_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return RS_ECUDA;
    return union_counts(ctx, L_host, p, n, seed, counts_host, static_cast<cudaStream_t>(stream));
}

uint64_t rs_union_key(uint64_t seed, uint32_t i) { return seed + ((uint64_t)i + 1) * kUnionWeyl; }

int rs_union_sample(rs_ctx* ctx, const uint64_t* L_host, uint32_t p, uint64_t n, uint64_t seed, uint32_t n0,
                    uint64_t* out_dev, uint64_t* counts_host, void* stream) {
    if (!ctx || n0 == 0) return RS_EINVAL;
    if (n > 0 && (!out_dev || ((uintptr_t)out_dev & 7))) return RS_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return RS_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = union_counts(ctx, L_host, p, n, seed, counts_host, st);
    if (rc || n == 0) return rc;
    // one request per segment with samples, output segment after segment
    std::vector<rs_request> req;
    uint64_t off = 0;
    for (uint32_t i = 0; i < p; ++i) {
        if (counts_host[i])
            req.push_back(rs_request{counts_host[i], L_host[i], rs_union_key(seed, i), off, n0, RS_KIND_H});
        off += counts_host[i];
    }
    const uint32_t R = (uint32_t)req.size();
    rs_batchplan* B = nullptr;
    rc = rs_batch_plan(ctx, req.data(), R, &B);
    if (rc) return rc;
    // the count tree's scratch is free again: the requests' status words
    int32_t* status = reinterpret_cast<int32_t*>(ctx->words);
    rc = rs_batch_run(B, out_dev, status, st);
    uint64_t per_run = 0;
    if (!rc && !rs_batch_launch_count(B, &per_run)) ctx->launches += per_run;
    std::vector<int32_t> sh(R);
    if (!rc) rc = cuda_rc(cudaMemcpyAsync(sh.data(), status, R * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    if (!rc) rc = rs_sync(ctx, st);
    const int rd = rs_batch_destroy(B);
    for (uint32_t r = 0; !rc && r < R; ++r) rc = sh[r];
    return rc ? rc : rd;
}

int rs_points(rs_ctx* ctx, uint32_t d, const uint64_t* extents_host, uint64_t n, uint64_t seed, uint32_t n0,
              uint64_t* out_dev, void* stream) {
    if (!ctx || d == 0 || d > rs::kPointsMaxDim || !extents_host || n0 == 0) return RS_EINVAL;
    if (n > 0 && (!out_dev || ((uintptr_t)out_dev & 7))) return RS_EINVAL;
    rs::BoxExtents E{};
    unsigned __int128 V = 1;
    for (uint32_t k = 0; k < d; ++k) {
        if (extents_host[k] == 0) return RS_EINVAL;
        E.e[k] = extents_host[k];
        V *= extents_host[k];
        if (V > ((unsigned __int128)1 << 62)) return RS_EINVAL;
    }
    if (n == 0) return RS_OK;
    DeviceGuard g(ctx->device);
    if (!g.ok) return RS_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int D = depth_of(n, (uint64_t)V, n0);
    if (D > rs::kMaxDepth) return RS_ECAPACITY;
    const uint64_t nleaves = 1ull << D;
    constexpr uint64_t kBoxWords = sizeof(rs::BoxRec) / sizeof(uint64_t);
    int rc = ensure(ctx->boxes, ctx->boxes_cap, kBoxWords * 2 * nleaves);
    if (!rc) rc = ensure(ctx->nodes, ctx->nodes_cap, nleaves);
    if (!rc) rc = ensure(ctx->words, ctx->words_cap, n + 2);
    if (!rc) rc = ensure(ctx->ovf, ctx->ovf_cap, nleaves + 1);
    if (rc) return rc;
    rs::BoxRec* boxes = reinterpret_cast<rs::BoxRec*>(ctx->boxes);
    uint64_t* idx = ctx->words;
    unsigned long long* stats = reinterpret_cast<unsigned long long*>(ctx->words + n);
    rc = cuda_rc(rs::launch_points_tree(boxes, d, E, n, seed, D, ctx->tab, ctx->status, st));
    if (!rc) rc = cuda_rc(cudaMemsetAsync(stats, 0, 2 * sizeof(uint64_t), st));
    if (!rc) rc = cuda_rc(rs::launch_points_leaf_recs(boxes + nleaves, nleaves, d, ctx->nodes, stats, st));
    ctx->launches += 2 + (uint64_t)D;
    uint64_t sh[2] = {0, 0};
    if (!rc) rc = cuda_rc(cudaMemcpyAsync(sh, stats, sizeof(sh), cudaMemcpyDeviceToHost, st));
    if (!rc) rc = cuda_rc(cudaStreamSynchronize(st));
    if (rc) return rc;
    // the general path takes leaves above the shared-memory table's room
    const uint64_t big_kmax = std::min<uint64_t>(std::max<uint64_t>(sh[1], 64), rs::kBigLeafMax);
    const uint64_t bytes = rs::big_pool_bytes(big_kmax);
    if (ctx->big_pool_bytes < bytes) {
        if (ctx->big_pool) cudaFree(ctx->big_pool);
        ctx->big_pool = nullptr;
        ctx->big_pool_bytes = 0;
        rc = cuda_rc(cudaMalloc(&ctx->big_pool, bytes));
        if (rc) return rc;
        ctx->big_pool_bytes = bytes;
    }
    rs::LeafLaunch L{};
    L.leaves = ctx->nodes;
    L.nleaves = nleaves;
    L.first_id = nleaves;
    L.seed = seed;
    L.smax = sh[0];
    L.out = idx;
    L.status = ctx->status;
    L.ovf_list = ctx->ovf;
    L.ovf_count = ctx->ovf + nleaves;
    L.big_pool = ctx->big_pool;
    L.big_kmax = big_kmax;
    L.cap = ctx->leaf_cap;
    L.sms = ctx->sms;
    L.with_replacement = true;
    L.mean_count = n >> D;
    rc = cuda_rc(rs::launch_leaves(L, st));
    if (!rc) rc = cuda_rc(rs::launch_points_decode(boxes + nleaves, nleaves, d, idx, out_dev, ctx->sms, st));
    ctx->launches += 3;
    return rc;
}

int rs_sync(rs_ctx* ctx, void* stream) {
    if (!ctx) return RS_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return RS_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(st) != cudaSuccess) return RS_ECUDA;
    int h = 0;
    if (cudaMemcpy(&h, ctx->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return RS_ECUDA;
    if (h != RS_OK && cudaMemset(ctx->status, 0, sizeof(int)) != cudaSuccess) return RS_ECUDA;
    return h;
}

const char* rs_strerror(int code) {
    switch (code) {
        case RS_OK: return "ok";
        case RS_EINVAL: return "invalid argument";
        case RS_ECAPACITY: return "result exceeds the buffer or a size limit";
        case RS_ENOMEM: return "out of memory";
        case RS_ECUDA: return "CUDA runtime error";
        case RS_ETIMEOUT: return "bounded wait gave up";
        case RS_EITER: return "iteration cap reached";
        default: return "unknown error code";
    }
}

int rs_set_profiling(rs_ctx* ctx, int on) {
    if (!ctx) return RS_EINVAL;
    ctx->profiling = on != 0;
    ctx->ev_used = 0;
    ctx->prof_calls.clear();
    return RS_OK;
}

int rs_phase_totals(rs_ctx* ctx, double* tree_ms, double* leaf_ms, uint64_t* calls) {
    if (!ctx || !tree_ms || !leaf_ms || !calls) return RS_EINVAL;
    DeviceGuard g(ctx->device);
    *tree_ms = 0.0;
    *leaf_ms = 0.0;
    *calls = ctx->prof_calls.size();
    for (const auto& c : ctx->prof_calls) {
        float t = 0.f;
        if (cudaEventSynchronize(ctx->ev_pool[c.end]) != cudaSuccess) return RS_ECUDA;
        if (cudaEventSynchronize(ctx->ev_pool[c.tree_end]) != cudaSuccess) return RS_ECUDA;
        if (cudaEventElapsedTime(&t, ctx->ev_pool[c.start], ctx->ev_pool[c.tree_end]) != cudaSuccess) return RS_ECUDA;
        *tree_ms += t;
        for (const auto& ab : c.leaves) {
            float l = 0.f;
            if (cudaEventElapsedTime(&l, ctx->ev_pool[ab.first], ctx->ev_pool[ab.second]) != cudaSuccess)
                return RS_ECUDA;
            *leaf_ms += l;
        }
    }
    return RS_OK;
}

int rs_set_pipeline(rs_ctx* ctx, int log2_parts, int leaf_blocks_per_sm) {
    if (!ctx || log2_parts < 0 || log2_parts > 6 || leaf_blocks_per_sm < 0) return RS_EINVAL;
    ctx->pipe_log2 = log2_parts;
    ctx->pipe_leaf_blocks = leaf_blocks_per_sm;
    return RS_OK;
}

int rs_set_bernoulli_staging(rs_ctx* ctx, uint64_t max_bytes, uint64_t slots_per_chunk) {
    if (!ctx) return RS_EINVAL;
    ctx->stage_max_words = max_bytes / sizeof(uint64_t);
    ctx->stage_slots = slots_per_chunk;
    return RS_OK;
}

int rs_launch_count(rs_ctx* ctx, uint64_t* count) {
    if (!ctx || !count) return RS_EINVAL;
    *count = ctx->launches;
    return RS_OK;
}

int rs_set_leaf_capacity(rs_ctx* ctx, uint32_t cap) {
    if (!ctx) return RS_EINVAL;
    ctx->leaf_cap = cap;
    return RS_OK;
}

int rs_set_iteration_caps(uint64_t rou_trials, uint64_t inv_restarts, uint64_t stream_blocks, uint64_t b_attempts) {
    const rs::IterCaps def = RS_DEFAULT_CAPS;
    auto pick = [](uint64_t v, uint64_t d) { return v > d ? d : v; };
    const rs::IterCaps c{pick(rou_trials, def.rou_trials), pick(inv_restarts, def.inv_restarts),
                         pick(stream_blocks, def.stream_blocks), pick(b_attempts, def.b_attempts)};
    for (rs::CapsWriter w : rs::caps_writers())
        if (w(c) != cudaSuccess) return RS_ECUDA;
    return RS_OK;
}

int rs_set_exact_deviates(rs_ctx* ctx, int on) {
    if (!ctx) return RS_EINVAL;
    ctx->guard = on == 0;
    return RS_OK;
}

}  // extern "C"
