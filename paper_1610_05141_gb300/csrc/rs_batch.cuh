// rs_batch.cuh -- device view of a planned batch of independent requests.
//
// Every request is its own sample (its own split tree and leaves, keyed by
// its own seed), so requests need no coordination at all (Sec. 3.2: no
// communication besides the parameters); a batch only flattens their work:
// the tree nodes of all requests level by level, and their leaves in groups
// of equal kind and key width.
#pragma once
#include "rs_common.cuh"

namespace rs {

struct BatchReq {
    uint64_t n, N, seed, out_off;
    uint64_t node_base;   // this request's node records start at nodes + node_base (heap id 0 unused)
    uint32_t n0, kind;
    int32_t D;            // tree depth, -1 if the request does no work
    int32_t status0;      // argument check result, copied to the status array at the start of a run
};

// One warp's share of a tree level: `count` consecutive nodes of request
// `req` starting at heap id `v0`.
struct BatchTreeItem {
    uint32_t req, count;
    uint64_t v0;
};

// The leaves of a group: requests req_of[0..m) in order, request req_of[i]
// owning group leaves [prefix[i], prefix[i+1]).
struct BatchGroupView {
    const BatchReq* reqs;
    const uint32_t* req_of;
    const uint64_t* prefix;
    uint32_t m;
    uint64_t nleaves;
    NodeRec* nodes;
    uint64_t* pool;
    int* status;
};

struct ResolvedLeaf {
    NodeRec rec;
    uint64_t id;       // heap id of the leaf in its request's tree
    uint64_t seed;
    uint64_t* out;     // the request's output
    int* status;       // the request's status word
};

RS_DEV ResolvedLeaf resolve_leaf(const BatchGroupView& G, uint64_t g) {
    uint32_t lo = 0, hi = G.m;   // last i with prefix[i] <= g
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (G.prefix[mid] <= g) lo = mid; else hi = mid;
    }
    const uint32_t r = G.req_of[lo];
    const BatchReq q = G.reqs[r];
    const uint64_t first = 1ull << q.D;
    const uint64_t id = first + (g - G.prefix[lo]);
    ResolvedLeaf L;
    L.rec = G.nodes[q.node_base + id];
    L.id = id;
    L.seed = q.seed;
    L.out = G.pool + q.out_off;
    L.status = G.status + r;
    return L;
}

}  // namespace rs
