// rs_batch.cu -- groups of device work: many independent sampling requests
// (the batch API) and range queries on resident trees, each group one fixed
// sequence of launches on one stream.
//
// A plan (host) validates the requests, computes every tree depth and lays
// out: the node records of all requests in one array, per tree level a list
// of warp items (request, first node, count), and the leaves grouped by kind
// and key width; for queries, their boundary leaves, interior leaves and
// results.  The batch API issues a plan once with plain launches, then
// captures the sequence into a CUDA graph and replays it.  Each request's
// output equals its own rs_sample / rs_sample_with_replacement / rs_sample_b
// output: the sample is a function of the request alone (Sec. 4.5).
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include "rs_big_leaf.cuh"
#include "rs_group.h"
#include "rs_hash_leaf.cuh"
#include "rs_tree_warp.cuh"

namespace rs {

constexpr int kBatchTreeWarps = 4;
constexpr int kBatchLeafThreads = 256;
constexpr uint32_t kBatchTreeBatch = 128;
constexpr int kLocateThreads = 256;

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

// A level whose items hold at most 8 nodes of one request: 32 / count lanes
// per node, four lanes per trial (rs_tree_warp.cuh: tree_terms_warp).
__global__ void __launch_bounds__(kBatchTreeWarps * 32) batch_terms_kernel(const BatchReq* __restrict__ reqs,
                                                                           const BatchTreeItem* __restrict__ items,
                                                                           uint32_t nitems, NodeRec* nodes,
                                                                           const double* __restrict__ tab,
                                                                           int* status) {
    const uint32_t warp = threadIdx.x >> 5;
    const uint32_t it = blockIdx.x * kBatchTreeWarps + warp;
    if (it >= nitems) return;
    const BatchTreeItem e = items[it];
    const BatchReq q = reqs[e.req];
    const uint32_t G = 32 / e.count;
    if (q.kind == RS_KIND_WR)
        tree_terms_warp<true>(nodes + q.node_base, e.v0, e.count, make_key(q.seed), tab, status + e.req, G);
    else
        tree_terms_warp<false>(nodes + q.node_base, e.v0, e.count, make_key(q.seed), tab, status + e.req, G);
}

// Leaf H / leaf WR over the leaves of a view, one block per leaf at a time;
// leaves the shared-memory table cannot take go to the overflow list.  Two
// shapes as in the single-request path: 256 threads with room for 4,864
// values, 512 with room for 9,728.
// Copies `bytes` (a multiple of 16, both addresses 16-byte aligned) into
// shared memory asynchronously; prefetch_all_wait() completes every copy
// this thread started.
RS_DEV void prefetch_bytes(void* dst, const void* src, int bytes) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    const unsigned char* p = static_cast<const unsigned char*>(src);
    for (int o = 0; o < bytes; o += 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + o), "l"(p + o) : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
}
RS_DEV void prefetch_all_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <typename KeyT, bool WR, class View, int NT, uint32_t CAP>
__global__ void __launch_bounds__(NT, 1024 / NT) group_leaf_kernel(View G, uint32_t* ovf_list, uint32_t* ovf_count,
                                                                  uint32_t cap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto& sm = *reinterpret_cast<HashShared<KeyT, NT / 32, CAP>*>(smem_raw);
    if constexpr (std::is_same<View, BatchGroupView>::value) {
        // A batch's leaf is resolved by three dependent loads (descriptor,
        // then request and node record); thread 0 fetches them ahead by
        // cp.async while the block works: the descriptor two leaves ahead
        // (three slots) and the request and record one leaf ahead (two),
        // each slot last read before the previous leaf's final barrier.
        __shared__ __align__(16) LeafDesc dbuf[3];
        __shared__ __align__(16) NodeRec rbuf[2];
        __shared__ __align__(16) BatchReq qbuf[2];
        const uint64_t n = G.nleaves, step = gridDim.x, g0 = blockIdx.x;
        if (g0 >= n) return;
        if (threadIdx.x == 0) {
            prefetch_bytes(&dbuf[0], &G.desc[g0], sizeof(LeafDesc));
            prefetch_all_wait();
            prefetch_bytes(&rbuf[0], &G.nodes[dbuf[0].node], sizeof(NodeRec));
            prefetch_bytes(&qbuf[0], &G.reqs[dbuf[0].req], sizeof(BatchReq));
            if (g0 + step < n) prefetch_bytes(&dbuf[1], &G.desc[g0 + step], sizeof(LeafDesc));
            prefetch_all_wait();
        }
        __syncthreads();
        uint32_t t = 0;
        for (uint64_t g = g0; g < n; g += step, ++t) {
            const LeafDesc d = dbuf[t % 3];
            const NodeRec rec = rbuf[t & 1];
            const BatchReq& q = qbuf[t & 1];
            const uint64_t id = (1ull << q.D) + d.i, seed = q.seed;
            uint64_t* out = q.out_ptr ? q.out_ptr : G.pool + q.out_off;
            int* status = G.status + d.req;
            if (threadIdx.x == 0) {
                if (g + step < n) {   // its descriptor arrived with the last leaf
                    const LeafDesc& dn = dbuf[(t + 1) % 3];
                    prefetch_bytes(&rbuf[(t + 1) & 1], &G.nodes[dn.node], sizeof(NodeRec));
                    prefetch_bytes(&qbuf[(t + 1) & 1], &G.reqs[dn.req], sizeof(BatchReq));
                }
                if (g + 2 * step < n) prefetch_bytes(&dbuf[(t + 2) % 3], &G.desc[g + 2 * step], sizeof(LeafDesc));
            }
            if (rec.c != 0) {
                const LeafRec lr{rec.lo, rec.S, rec.c, rec.off, id};
                if (!hash_leaf<KeyT, NT, 0, WR, CAP>(sm, lr, make_key(seed), out, status, threadIdx.x, cap)) {
                    if (threadIdx.x == 0) ovf_list[atomicAdd(ovf_count, 1u)] = (uint32_t)g;
                }
            }
            if (threadIdx.x == 0) prefetch_all_wait();
            __syncthreads();
        }
        return;
    }
    for (uint64_t g = blockIdx.x; g < G.nleaves; g += gridDim.x) {
        const ResolvedLeaf L = resolve_leaf(G, g);
        if (L.rec.c == 0) continue;
        const LeafRec lr{L.rec.lo, L.rec.S, L.rec.c, L.rec.off, L.id};
        if (!hash_leaf<KeyT, NT, 0, WR, CAP>(sm, lr, make_key(L.seed), L.out, L.status, threadIdx.x, cap)) {
            if (threadIdx.x == 0) ovf_list[atomicAdd(ovf_count, 1u)] = (uint32_t)g;
        }
    }
}

// The general path for the overflow list of a view.
template <bool WR, class View>
__global__ void __launch_bounds__(kBigThreads) group_big_kernel(View G, const uint32_t* ovf_list,
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

// Index of the first of the sorted x[0..n) that is >= key, by one warp:
// 32-way splits of the range, then one probe per lane.
RS_DEV uint64_t warp_lower_bound(const uint64_t* __restrict__ x, uint64_t n, uint64_t key) {
    const uint32_t lane = threadIdx.x & 31;
    uint64_t lo = 0, hi = n;
    while (hi - lo > 32) {
        const uint64_t step = (hi - lo + 31) / 32;
        const uint64_t p = lo + lane * step;
        const uint32_t t = __popc(__ballot_sync(0xFFFFFFFFu, p < hi && x[p] < key));
        if (t == 0) return lo;   // x[lo] >= key
        const uint64_t next = lo + (uint64_t)t * step;   // first probe >= key, or past hi
        lo = lo + (uint64_t)(t - 1) * step + 1;
        if (next < hi) hi = next;
    }
    const uint64_t p = lo + lane;
    return lo + __popc(__ballot_sync(0xFFFFFFFFu, p < hi && x[p] < key));
}

// Locate step of each query (one block per query): where [a, b) starts in
// boundary leaf i0 and ends in leaf i0+m-1, the count, the base offset; the
// boundary parts are copied to the output if the count fits.
__global__ void __launch_bounds__(kLocateThreads) query_locate_kernel(const QueryDesc* __restrict__ qs,
                                                                      QueryRes* __restrict__ res, uint32_t nq) {
    __shared__ uint64_t sh_k[2];
    const uint32_t warp = threadIdx.x >> 5;
    for (uint32_t qi = blockIdx.x; qi < nq; qi += gridDim.x) {
        const QueryDesc& Q = qs[qi];
        const NodeRec r0 = Q.leaves[Q.i0];
        const NodeRec r1 = Q.leaves[Q.i0 + Q.m - 1];
        const uint64_t* hi_part = Q.m == 1 ? Q.scratch : Q.scratch + r0.c;
        const uint64_t hi_n = Q.m == 1 ? r0.c : r1.c;
        if (warp == 0) {
            const uint64_t k = warp_lower_bound(Q.scratch, r0.c, Q.a);
            if ((threadIdx.x & 31) == 0) sh_k[0] = k;
        } else if (warp == 1) {
            const uint64_t k = warp_lower_bound(hi_part, hi_n, Q.b);
            if ((threadIdx.x & 31) == 0) sh_k[1] = k;
        }
        __syncthreads();
        const uint64_t k_lo = sh_k[0], k_hi = sh_k[1];
        const uint64_t base = r0.off + k_lo;
        const uint64_t end = (Q.m == 1 ? r0.off : r1.off) + k_hi;
        const uint64_t count = end - base;
        int st = res[qi].status;   // errors of the boundary leaves
        if (st == RS_OK && count > Q.cap) st = RS_ECAPACITY;
        if (threadIdx.x == 0) {
            res[qi].count = count;
            res[qi].base = base;
            res[qi].status = st;
            res[qi].go = (st == RS_OK && Q.m > 2) ? 1 : 0;
        }
        if (st == RS_OK) {
            if (Q.m == 1) {
                for (uint64_t i = threadIdx.x; i < count; i += kLocateThreads) Q.out[i] = Q.scratch[k_lo + i];
            } else {
                const uint64_t n0 = r0.c - k_lo;
                for (uint64_t i = threadIdx.x; i < n0; i += kLocateThreads) Q.out[i] = Q.scratch[k_lo + i];
                uint64_t* dst = Q.out + (r1.off - base);
                for (uint64_t i = threadIdx.x; i < k_hi; i += kLocateThreads) dst[i] = hi_part[i];
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Host side: the group planner.
// ---------------------------------------------------------------------------

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// Leaf groups: kind (H, WR) x key width x size class (the large class:
// leaves averaging more than the 256-thread shape comfortably holds),
// Algorithm B (group 4), and for requests with 64-bit keys and small means
// the compact table (groups 9 and 10).
int group_of(int kind, bool wide, bool large, bool compact = false) {
    if (kind == RS_KIND_B) return 4;
    if (compact && wide && !large) return 9 + kind;
    return kind * 2 + (wide ? 1 : 0) + (large ? 5 : 0);
}
bool large_class(uint64_t mean_count) { return mean_count * 20 > (uint64_t)kLeafFastCap * 17; }

// Counter slots of the zeroed block: sample leaf groups, query boundary
// subgroups, query interior subgroups.
constexpr int kCounters = 3 * GroupPlan::kGroups + 1;
int counter_of(int part, int gi) { return part * GroupPlan::kGroups + gi; }

int cuda_rc(cudaError_t e) {
    if (e == cudaSuccess) return RS_OK;
    return e == cudaErrorMemoryAllocation ? RS_ENOMEM : RS_ECUDA;
}

// Largest number of blocks of `kern` per SM on the current device (sets the
// kernel's shared-memory limit first), cached per kernel and device.
int blocks_per_sm(const void* kern, size_t smem, int threads) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find({kern, dev});
    if (it != cache.end()) return it->second;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -1;
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem) != cudaSuccess) return -1;
    per = std::max(per, 1);
    cache[{kern, dev}] = per;
    return per;
}

// The leaf kernel of one shape for a view: its function, shared memory and
// capacity.
template <class View, int NT, uint32_t CAP>
void leaf_flavour(bool wide, bool wr, void (**kern)(View, uint32_t*, uint32_t*, uint32_t), size_t* smem,
                  uint32_t* cap) {
    if (wide) {
        *kern = wr ? group_leaf_kernel<uint64_t, true, View, NT, CAP> : group_leaf_kernel<uint64_t, false, View, NT, CAP>;
        *smem = sizeof(HashShared<uint64_t, NT / 32, CAP>);
    } else {
        *kern = wr ? group_leaf_kernel<uint32_t, true, View, NT, CAP> : group_leaf_kernel<uint32_t, false, View, NT, CAP>;
        *smem = sizeof(HashShared<uint32_t, NT / 32, CAP>);
    }
    *cap = CAP;
}

// The compact 64-bit-key shape (256 threads, room for kCompact64Cap
// values), built for request groups only.
template <class View>
void compact_flavour(bool wr, void (**kern)(View, uint32_t*, uint32_t*, uint32_t), size_t* smem, uint32_t* cap) {
    if constexpr (std::is_same<View, BatchGroupView>::value) {
        *kern = wr ? group_leaf_kernel<uint64_t, true, View, kBatchLeafThreads, kCompact64Cap>
                   : group_leaf_kernel<uint64_t, false, View, kBatchLeafThreads, kCompact64Cap>;
        *smem = sizeof(HashShared<uint64_t, kBatchLeafThreads / 32, kCompact64Cap>);
        *cap = kCompact64Cap;
    } else {
        leaf_flavour<View, kBatchLeafThreads, kLeafFastCap>(true, wr, kern, smem, cap);
    }
}

// One leaf kernel (+ the general path) over the leaves of a view; `threads`
// picks the shape (256 or 512), `compact` the compact 64-bit table at 256.
template <class View>
int issue_leaves(const View& V, int kind, bool wide, int threads, bool compact, uint32_t* ovf, uint32_t* ovf_count,
                 void* big, uint64_t big_kmax, int per_sm_cap, bool persistent, const double* tab, int sms,
                 cudaStream_t st, uint64_t* nl) {
    if (V.nleaves == 0) return RS_OK;
    if (kind == RS_KIND_B) {
        ++*nl;
        return cuda_rc(launch_batch_leaves_b(V, tab, sms, st));
    }
    const bool wr = kind == RS_KIND_WR;
    void (*kern)(View, uint32_t*, uint32_t*, uint32_t);
    size_t smem;
    uint32_t cap;
    if (threads == 512) leaf_flavour<View, 512, 2 * kLeafFastCap>(wide, wr, &kern, &smem, &cap);
    else if (compact && wide) compact_flavour<View>(wr, &kern, &smem, &cap);
    else leaf_flavour<View, kBatchLeafThreads, kLeafFastCap>(wide, wr, &kern, &smem, &cap);
    int per = blocks_per_sm(reinterpret_cast<const void*>(kern), smem, threads == 512 ? 512 : kBatchLeafThreads);
    if (per < 0) return RS_ECUDA;
    if (per_sm_cap > 0) per = std::min(per, per_sm_cap);
    const uint64_t grid = persistent ? std::min<uint64_t>(V.nleaves, (uint64_t)sms * per)
                                     : std::min<uint64_t>(V.nleaves, 0x7FFFFFFFull);
    kern<<<(unsigned)grid, threads == 512 ? 512 : kBatchLeafThreads, smem, st>>>(V, ovf, ovf_count, cap);
    ++*nl;
    if (big_kmax) {
        const BigScratch sc = carve_big_scratch(big, big_kmax);
        if (wr) group_big_kernel<true, View><<<1, kBigThreads, 0, st>>>(V, ovf, ovf_count, sc);
        else group_big_kernel<false, View><<<1, kBigThreads, 0, st>>>(V, ovf, ovf_count, sc);
        ++*nl;
    }
    return cuda_rc(cudaGetLastError());
}

}  // namespace

int plan_depth(uint64_t n, uint64_t N, uint32_t n0) {
    int D = 0;
    while ((unsigned __int128)n > ((unsigned __int128)n0 << D)) ++D;
    while (D > 0 && ((unsigned __int128)1 << D) > (unsigned __int128)N) --D;
    return D;
}

uint64_t leaf_of_position(uint64_t N, int D, uint64_t pos) {
    uint64_t lo = 0, S = N, idx = 0;
    for (int l = 0; l < D; ++l) {
        const uint64_t K = S / 2;
        if (pos < lo + K) {
            idx = 2 * idx;
            S = K;
        } else {
            idx = 2 * idx + 1;
            lo += K;
            S -= K;
        }
    }
    return idx;
}

void GroupPlan::request_cost(const rs_request& q, uint64_t* up, uint64_t* work) {
    *up = sizeof(BatchReq);
    *work = 0;
    if (q.n == 0 || q.n0 == 0) return;
    const int D = plan_depth(q.n, q.N, q.n0);
    uint64_t items = 0;
    for (int l = 0; l < D; ++l) items += std::max<uint64_t>(1, (1ull << l) / kBatchTreeBatch);
    *up += items * sizeof(BatchTreeItem) + (1ull << D) * sizeof(LeafDesc);
    *work = (2ull << D) * sizeof(NodeRec) + (1ull << D) * 4;
}

void GroupPlan::query_cost(const TreeInfo& t, uint64_t a, uint64_t b, uint64_t* up, uint64_t* work) {
    *up = sizeof(QueryDesc) + 24;
    *work = sizeof(QueryRes) + 2 * t.maxc * 8 + 16;
    if (t.D < 0 || a >= b) return;
    const uint64_t i0 = leaf_of_position(t.N, t.D, a - 1);
    const uint64_t i1 = leaf_of_position(t.N, t.D, b - 2);
    *work += (i1 - i0 + 1) * 4;
}

void GroupPlan::build(const rs_request* reqs, uint64_t* const* out_ptrs, uint32_t R, const GroupQuery* qs,
                      uint32_t Q) {
    R_ = R;
    Q_ = Q;
    reqs_.assign(R, BatchReq{});
    levels_.clear();
    qdesc_.clear();
    qscratch_.clear();
    for (int gi = 0; gi < kGroups; ++gi) {
        groups_[gi] = Sub{};
        groups_[gi].kind = gi == 4 ? RS_KIND_B : (gi % 5) / 2;
        groups_[gi].wide = gi != 4 && ((gi % 5) & 1);
        groups_[gi].large = gi > 4 && gi < 9;
        if (gi >= 9) {
            groups_[gi].kind = gi - 9;
            groups_[gi].wide = true;
            groups_[gi].compact = true;
        }
        qgroups_[gi] = groups_[gi];
        qgroups_[gi].compact = false;   // (query groups 9 and 10 stay empty)
    }
    nodes_ = 0;
    uint64_t bound = 0;
    int Dmax = -1;
    for (uint32_t r = 0; r < R; ++r) {
        const rs_request& q = reqs[r];
        BatchReq& b = reqs_[r];
        b.n = q.n;
        b.N = q.N;
        b.seed = q.seed;
        b.out_off = q.out_off;
        b.out_ptr = out_ptrs ? out_ptrs[r] : nullptr;
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
        const int D = plan_depth(q.n, q.N, q.n0);
        if (D > kMaxDepth) {
            b.status0 = RS_ECAPACITY;
            continue;
        }
        b.D = D;
        b.node_base = nodes_;
        nodes_ += 2ull << D;
        Dmax = std::max(Dmax, D);
        const uint64_t nleaves = 1ull << D;
        const uint64_t smax = (q.N >> D) + ((q.N & (nleaves - 1)) ? 1 : 0);
        Sub& G = groups_[group_of((int)q.kind, smax > (1ull << 32), large_class(q.n >> D),
                                  (q.n >> D) <= kCompact64Mean)];
        for (uint64_t i = 0; i < nleaves; ++i) G.desc.push_back(LeafDesc{b.node_base + nleaves + i, r, (uint32_t)i});
        G.n1 += nleaves;
        if (q.kind != RS_KIND_B) bound = std::max<uint64_t>(bound, wr ? q.n : std::min<uint64_t>(q.n, smax - smax / 2));
    }
    // tree levels: warp items of up to kBatchTreeBatch consecutive nodes
    for (int level = 0; level < Dmax; ++level) {
        std::vector<BatchTreeItem> items;
        const uint64_t cnt = 1ull << level;
        const uint32_t per = (uint32_t)std::min<uint64_t>(cnt, kBatchTreeBatch);
        for (uint32_t r = 0; r < R; ++r) {
            if (reqs_[r].D <= level) continue;
            for (uint64_t s = 0; s < cnt; s += per)
                items.push_back(BatchTreeItem{r, (uint32_t)std::min<uint64_t>(per, cnt - s), cnt + s});
        }
        levels_.push_back(std::move(items));
    }
    // queries
    for (uint32_t qi = 0; qi < Q; ++qi) {
        const GroupQuery& g = qs[qi];
        const TreeInfo& t = *g.tree;
        QueryDesc d{};
        d.leaves = t.leaves;
        d.first_id = 1ull << t.D;
        d.seed = t.seed;
        d.a = g.a;
        d.b = g.b;
        d.i0 = leaf_of_position(t.N, t.D, g.a - 1);
        d.m = leaf_of_position(t.N, t.D, g.b - 2) - d.i0 + 1;
        d.out = g.out;
        d.cap = g.cap;
        d.scratch_cap = (d.m == 1 ? 1 : 2) * t.maxc;
        qdesc_.push_back(d);
        qscratch_.push_back(std::max<uint64_t>(d.scratch_cap, 1));
        Sub& G = qgroups_[group_of(t.kind, t.wide, t.maxk > kLeafFastCap)];
        G.a32.push_back(qi << 1);
        if (d.m > 1) G.a32.push_back((qi << 1) | 1);
        G.n1 = G.a32.size();
        if (d.m > 2) {
            if (G.p64.empty()) G.p64.push_back(0);
            G.b32.push_back(qi);
            G.p64.push_back(G.p64.back() + (d.m - 2));
            G.n2 += d.m - 2;
        }
        if (t.kind != RS_KIND_B) bound = std::max<uint64_t>(bound, t.maxk);
    }
    big_kmax_ = bound > 64 ? std::min<uint64_t>(bound, kBigLeafMax) : 0;
    layout();
}

bool GroupPlan::has_class(bool large) const {
    for (int gi = 0; gi < kGroups; ++gi)
        if (groups_[gi].large == large && gi != 4 && (groups_[gi].n1 || qgroups_[gi].n1 || qgroups_[gi].n2)) return true;
    return false;
}

void GroupPlan::layout() {
    size_t up = 0, work = 0;
    auto take = [](size_t& at, size_t bytes) {
        const size_t o = at;
        at = align_up(at + bytes);
        return o;
    };
    o_reqs_ = take(up, reqs_.size() * sizeof(BatchReq));
    o_levels_.clear();
    for (auto& lv : levels_) o_levels_.push_back(take(up, lv.size() * sizeof(BatchTreeItem)));
    for (Sub& G : groups_) G.o_desc = take(up, G.desc.size() * sizeof(LeafDesc));
    o_qdesc_ = take(up, qdesc_.size() * sizeof(QueryDesc));
    for (Sub& G : qgroups_) {
        G.o_a32 = take(up, G.a32.size() * 4);
        G.o_b32 = take(up, G.b32.size() * 4);
        G.o_p64 = take(up, G.p64.size() * 8);
    }
    o_nodes_ = take(work, nodes_ * sizeof(NodeRec));
    o_zero_ = work;
    zero_bytes_ = kCounters * 4 + Q_ * sizeof(QueryRes);
    o_qres_ = o_zero_ + kCounters * 4;
    take(work, zero_bytes_);
    for (Sub& G : groups_) G.o_ovf1 = take(work, G.n1 * 4);
    for (Sub& G : qgroups_) {
        G.o_ovf1 = take(work, G.n1 * 4);
        G.o_ovf2 = take(work, G.n2 * 4);
    }
    uint64_t scr = 0;
    for (uint64_t s : qscratch_) scr += s;
    o_qscr_ = take(work, scr * 8);
    up_bytes_ = std::max<size_t>(up, kAlign);
    work_bytes_ = std::max<size_t>(work, kAlign);
}

void GroupPlan::bind(unsigned char* up, unsigned char* work, void* big, unsigned char* img) {
    up_ = up;
    work_ = work;
    big_ = big;
    qres_ = reinterpret_cast<QueryRes*>(work + o_qres_);
    uint64_t at = 0;
    for (uint32_t qi = 0; qi < Q_; ++qi) {
        qdesc_[qi].scratch = reinterpret_cast<uint64_t*>(work + o_qscr_) + at;
        at += qscratch_[qi];
    }
    auto put = [img](size_t o, const void* src, size_t bytes) {
        if (bytes) std::memcpy(img + o, src, bytes);
    };
    put(o_reqs_, reqs_.data(), reqs_.size() * sizeof(BatchReq));
    for (size_t l = 0; l < levels_.size(); ++l)
        put(o_levels_[l], levels_[l].data(), levels_[l].size() * sizeof(BatchTreeItem));
    for (const Sub& G : groups_) put(G.o_desc, G.desc.data(), G.desc.size() * sizeof(LeafDesc));
    put(o_qdesc_, qdesc_.data(), qdesc_.size() * sizeof(QueryDesc));
    for (const Sub& G : qgroups_) {
        put(G.o_a32, G.a32.data(), G.a32.size() * 4);
        put(G.o_b32, G.b32.data(), G.b32.size() * 4);
        put(G.o_p64, G.p64.data(), G.p64.size() * 8);
    }
}

int GroupPlan::issue(const double* tab, int sms, uint64_t* pool, int* status, cudaStream_t st, uint64_t* launches) {
    uint64_t nl = 0;
    int rc = cuda_rc(cudaMemsetAsync(work_ + o_zero_, 0, zero_bytes_, st));
    uint32_t* counters = reinterpret_cast<uint32_t*>(work_ + o_zero_);
    const BatchReq* reqs = reinterpret_cast<const BatchReq*>(up_ + o_reqs_);
    NodeRec* nodes = reinterpret_cast<NodeRec*>(work_ + o_nodes_);
    if (!rc && R_ > 0) {
        batch_init_kernel<<<(R_ + 255) / 256, 256, 0, st>>>(reqs, R_, nodes, status);
        ++nl;
        const size_t tree_smem = (size_t)kBatchTreeWarps * 32 * kLogSlots * sizeof(double);
        for (size_t l = 0; l < levels_.size(); ++l) {
            const uint32_t n = (uint32_t)levels_[l].size();
            if (n == 0) continue;
            const auto* items = reinterpret_cast<const BatchTreeItem*>(up_ + o_levels_[l]);
            const unsigned blocks = (n + kBatchTreeWarps - 1) / kBatchTreeWarps;
            // items of level l hold min(2^l, kBatchTreeBatch) nodes each
            if ((1ull << l) <= 8)
                batch_terms_kernel<<<blocks, kBatchTreeWarps * 32, 0, st>>>(reqs, items, n, nodes, tab, status);
            else
                batch_tree_kernel<<<blocks, kBatchTreeWarps * 32, tree_smem, st>>>(reqs, items, n, nodes, tab, status);
            ++nl;
        }
        for (int gi = 0; !rc && gi < kGroups; ++gi) {
            const Sub& G = groups_[gi];
            if (G.n1 == 0) continue;
            BatchGroupView V{reqs, reinterpret_cast<const LeafDesc*>(up_ + G.o_desc), G.n1, nodes, pool, status};
            rc = issue_leaves(V, G.kind, G.wide, threads_of(G), G.compact,
                              reinterpret_cast<uint32_t*>(work_ + G.o_ovf1), counters + counter_of(0, gi), big_, big_kmax_, per_sm_, persistent_, tab, sms, st, &nl);
        }
    }
    if (!rc && Q_ > 0) {
        const QueryDesc* qd = reinterpret_cast<const QueryDesc*>(up_ + o_qdesc_);
        for (int gi = 0; !rc && gi < kGroups; ++gi) {
            const Sub& G = qgroups_[gi];
            if (G.n1 == 0) continue;
            QueryBoundView V{qd, qres_, reinterpret_cast<const uint32_t*>(up_ + G.o_a32), G.n1};
            rc = issue_leaves(V, G.kind, G.wide, threads_of(G), false,
                              reinterpret_cast<uint32_t*>(work_ + G.o_ovf1), counters + counter_of(1, gi), big_, big_kmax_, per_sm_, persistent_, tab, sms, st, &nl);
        }
        if (!rc) {
            const unsigned grid = (unsigned)std::min<uint64_t>(Q_, (uint64_t)sms * 8);
            query_locate_kernel<<<grid, kLocateThreads, 0, st>>>(qd, qres_, Q_);
            ++nl;
        }
        for (int gi = 0; !rc && gi < kGroups; ++gi) {
            const Sub& G = qgroups_[gi];
            if (G.n2 == 0) continue;
            QueryInnerView V{qd,
                             qres_,
                             reinterpret_cast<const uint32_t*>(up_ + G.o_b32),
                             reinterpret_cast<const uint64_t*>(up_ + G.o_p64),
                             (uint32_t)G.b32.size(),
                             G.n2};
            rc = issue_leaves(V, G.kind, G.wide, threads_of(G), false, reinterpret_cast<uint32_t*>(work_ + G.o_ovf2),
                              counters + counter_of(2, gi), big_, big_kmax_, per_sm_, persistent_, tab, sms, st, &nl);
        }
    }
    if (launches) *launches = nl;
    if (rc) return rc;
    return cuda_rc(cudaGetLastError());
}

}  // namespace rs

// ---------------------------------------------------------------------------
// The batch API.
// ---------------------------------------------------------------------------

struct rs_batchplan {
    int device = 0;
    int sms = 0;
    const double* tab = nullptr;   // the context's ln i! table
    rs::GroupPlan plan;
    unsigned char* up = nullptr;
    unsigned char* work = nullptr;
    void* big_pool = nullptr;
    // graph of the last run
    bool ran_eagerly = false;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t capture_stream = nullptr;
    uint64_t* graph_pool = nullptr;
    int32_t* graph_status = nullptr;
    uint64_t launches_per_run = 0;
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

int issue_run(rs_batchplan* B, uint64_t* pool, int32_t* status, cudaStream_t st, uint64_t* launches) {
    return B->plan.issue(B->tab, B->sms, pool, reinterpret_cast<int*>(status), st, launches);
}

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
    cudaFree(B->up);
    cudaFree(B->work);
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
    int rc = RS_OK;
    try {
        B->plan.build(reqs, nullptr, R, nullptr, 0);
        std::vector<unsigned char> img(B->plan.upload_bytes());
        rc = rs::cuda_rc(cudaMalloc(&B->up, B->plan.upload_bytes()));
        if (!rc) rc = rs::cuda_rc(cudaMalloc(&B->work, B->plan.work_bytes()));
        if (!rc && B->plan.big_kmax())
            rc = rs::cuda_rc(cudaMalloc(&B->big_pool, rs::big_pool_bytes(B->plan.big_kmax())));
        if (!rc) {
            B->plan.bind(B->up, B->work, B->big_pool, img.data());
            rc = rs::cuda_rc(cudaMemcpy(B->up, img.data(), img.size(), cudaMemcpyHostToDevice));
        }
    } catch (const std::bad_alloc&) {
        rc = RS_ENOMEM;
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
    return rs::cuda_rc(cudaGraphLaunch(B->exec, st));
}

int rs_batch_set_leaf_launch(rs_batchplan* B, int small_threads, int large_threads, int blocks_per_sm) {
    auto ok = [](int t) { return t == 0 || t == 256 || t == 512; };
    if (!B || !ok(small_threads) || !ok(large_threads) || blocks_per_sm < 0) return RS_EINVAL;
    B->plan.set_leaf_threads(small_threads, large_threads);
    B->plan.set_blocks_per_sm(blocks_per_sm);
    if (B->exec) {   // the next run captures its graph again
        cudaGraphExecDestroy(B->exec);
        B->exec = nullptr;
    }
    return RS_OK;
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
    // Output-invariant knobs (the leaf-to-block schedule and the block's
    // shape never change a value): leaf blocks per SM, then each size
    // class's leaf shape, each setting timed on the whole run.
    auto timed = [&](float* ms) {
        uint64_t nl = 0;
        int rc = issue_run(B, out_pool_dev, status_dev, st, &nl);   // warm
        cudaEventRecord(e0, st);
        if (!rc) rc = issue_run(B, out_pool_dev, status_dev, st, &nl);
        cudaEventRecord(e1, st);
        if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = RS_ECUDA;
        if (!rc) cudaEventElapsedTime(ms, e0, e1);
        return rc;
    };
    int best = 0, rc = RS_OK;
    float best_ms = 1e30f;
    for (int per : {0, 4, 3, 2, 1}) {
        B->plan.set_blocks_per_sm(per);
        float ms = 0.f;
        if ((rc = timed(&ms)) != RS_OK) break;
        if (ms < best_ms) {
            best_ms = ms;
            best = per;
        }
    }
    B->plan.set_blocks_per_sm(best);
    int threads[2] = {0, 0};
    for (int cls = 0; rc == RS_OK && cls < 2; ++cls) {
        if (!B->plan.has_class(cls == 1)) continue;
        int trial[2] = {threads[0], threads[1]};
        trial[cls] = cls ? 256 : 512;   // the other shape
        B->plan.set_leaf_threads(trial[0], trial[1]);
        float ms = 0.f;
        if ((rc = timed(&ms)) != RS_OK) break;
        if (ms < best_ms) {
            best_ms = ms;
            threads[cls] = trial[cls];
        }
    }
    B->plan.set_leaf_threads(threads[0], threads[1]);
    if (rc) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return rc;
    }
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
