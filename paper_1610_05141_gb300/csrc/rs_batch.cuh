// rs_batch.cuh -- device views of grouped work: planned batches of
// independent requests, and range queries on resident split trees.
//
// Every request is its own sample (its own split tree and leaves, keyed by
// its own seed), so requests need no coordination at all (Sec. 3.2: no
// communication besides the parameters); a batch only flattens their work:
// the tree nodes of all requests level by level, and their leaves in groups
// of equal kind and key width.
//
// A range query regenerates only the leaves whose positions overlap the
// queried values (Sec. 4.1: a leaf's sample is a function of its record and
// its id, so any leaf can be produced alone, in sorted order).  The leaf
// kernels see a query's leaves through the same resolve_leaf() interface as
// a batch's: a record, its heap id, a seed, and where to write.
#pragma once
#include "rs_common.cuh"

namespace rs {

struct BatchReq {
    uint64_t n, N, seed, out_off;
    uint64_t* out_ptr;    // output address, or null: the run's pool + out_off
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

// Group leaf g: its node record nodes[node], request req, leaf index i of
// that request (heap id 2^D + i).
struct __align__(16) LeafDesc {
    uint64_t node;
    uint32_t req, i;
};

// The leaves of a group, one descriptor each (one load resolves a leaf).
struct BatchGroupView {
    const BatchReq* reqs;
    const LeafDesc* desc;
    uint64_t nleaves;
    NodeRec* nodes;
    uint64_t* pool;
    int* status;
};

struct ResolvedLeaf {
    NodeRec rec;       // rec.off is relative to `out`; rec.c = 0 means nothing to do
    uint64_t id;       // heap id of the leaf in its request's tree
    uint64_t seed;
    uint64_t* out;     // where the leaf's output offsets count from
    int* status;       // the request's status word
};

// Last i with prefix[i] <= g (prefix[0] = 0 <= g < prefix[m]).
RS_DEV uint32_t owner_of(const uint64_t* __restrict__ prefix, uint32_t m, uint64_t g) {
    uint32_t lo = 0, hi = m;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (prefix[mid] <= g) lo = mid; else hi = mid;
    }
    return lo;
}

RS_DEV ResolvedLeaf resolve_leaf(const BatchGroupView& G, uint64_t g) {
    const LeafDesc d = G.desc[g];
    const BatchReq& q = G.reqs[d.req];
    ResolvedLeaf L;
    L.rec = G.nodes[d.node];
    L.id = (1ull << q.D) + d.i;
    L.seed = q.seed;
    L.out = q.out_ptr ? q.out_ptr : G.pool + q.out_off;
    L.status = G.status + d.req;
    return L;
}

// ---------------------------------------------------------------------------
// Range queries.  Values in [a, b) of a tree's sample lie in the leaves
// i0 .. i0+m-1 (leaf ranges follow from N and the depth alone).  A query
// runs in three steps: the boundary leaves i0 and i0+m-1 are generated into
// scratch; the locate step finds where [a, b) starts and ends in them, which
// fixes the global output offset `base` of the first value in range and the
// count, and copies the boundary parts to the output; the interior leaves
// are then generated straight into the output at (their offset - base).
// ---------------------------------------------------------------------------

struct QueryDesc {
    const NodeRec* leaves;   // the tree's 2^D leaf records
    uint64_t first_id;       // heap id of leaf 0 (2^D)
    uint64_t seed;
    uint64_t a, b;           // values in [a, b), 1 <= a < b <= N + 1
    uint64_t i0, m;          // overlapping leaves, m >= 1
    uint64_t* out;           // the caller's buffer
    uint64_t cap;            // its capacity in values
    uint64_t* scratch;       // room for the boundary leaves' full output
    uint64_t scratch_cap;    // values
};

struct QueryRes {
    uint64_t count;   // values in [a, b)
    uint64_t base;    // global output offset (in the tree's full sample) of the first of them
    int32_t status;   // RS_OK or the first error of the query
    int32_t go;       // set by the locate step: 1 = write the interior leaves
};

// The boundary leaves of a set of queries: item t is (query << 1) | side,
// side 0 = leaf i0 (scratch offset 0), side 1 = leaf i0+m-1 (after leaf i0).
struct QueryBoundView {
    const QueryDesc* q;
    QueryRes* res;
    const uint32_t* items;
    uint64_t nleaves;
};

RS_DEV ResolvedLeaf resolve_leaf(const QueryBoundView& V, uint64_t g) {
    const uint32_t t = V.items[g];
    const uint32_t qi = t >> 1;
    const QueryDesc& Q = V.q[qi];
    const bool hi_side = (t & 1) != 0;
    const uint64_t i = Q.i0 + (hi_side ? Q.m - 1 : 0);
    ResolvedLeaf L;
    L.rec = Q.leaves[i];
    L.rec.off = hi_side ? Q.leaves[Q.i0].c : 0;
    L.id = Q.first_id + i;
    L.seed = Q.seed;
    L.out = Q.scratch;
    L.status = &V.res[qi].status;
    if (L.rec.off + L.rec.c > Q.scratch_cap) {   // sized from the tree's largest leaf: cannot happen
        set_status(L.status, RS_ECAPACITY);
        L.rec.c = 0;
    }
    return L;
}

// The interior leaves (m - 2 per query) of a set of queries: queries
// q_of[0..nq) in order, query q_of[i] owning items [prefix[i], prefix[i+1]).
// They run after the locate step, which has set each query's base and `go`
// (read instead of the status word, which other blocks may still change,
// so that every thread of a block takes the same branch).
struct QueryInnerView {
    const QueryDesc* q;
    QueryRes* res;
    const uint32_t* q_of;
    const uint64_t* prefix;
    uint32_t nq;
    uint64_t nleaves;
};

RS_DEV ResolvedLeaf resolve_leaf(const QueryInnerView& V, uint64_t g) {
    const uint32_t i = owner_of(V.prefix, V.nq, g);
    const uint32_t qi = V.q_of[i];
    const QueryDesc& Q = V.q[qi];
    const uint64_t leaf = Q.i0 + 1 + (g - V.prefix[i]);
    ResolvedLeaf L;
    L.rec = Q.leaves[leaf];
    L.id = Q.first_id + leaf;
    L.seed = Q.seed;
    L.out = Q.out;
    L.status = &V.res[qi].status;
    if (!V.res[qi].go) L.rec.c = 0;   // over capacity or failed: write nothing
    else L.rec.off -= V.res[qi].base;
    return L;
}

}  // namespace rs
