// rs_group.h -- host planner of a group of device work: independent sampling
// requests (each its own split tree and leaves) and range queries on
// resident trees, issued as one fixed sequence of launches on one stream.
//
// A plan is built on the host, then bound to device memory in two parts:
// the upload image (request records, tree-level work items, leaf groups,
// query descriptors; written by the host and copied once) and the work area
// (node records, overflow lists, query scratch and results; device only).
// The batch API sizes both exactly; the server reuses fixed lanes.
#pragma once
#include <vector>

#include "rs_batch.cuh"
#include "rs_internal.h"

namespace rs {

// What a range query needs to know about its resident tree.
struct TreeInfo {
    const NodeRec* leaves;   // device, 2^D records
    uint64_t N, seed;
    int D, kind;
    bool wide;               // leaf size above 2^32: 64-bit keys
    uint64_t maxc;           // largest leaf count
    uint64_t maxk;           // largest leaf selection (count, or its complement)
};

struct GroupQuery {
    const TreeInfo* tree;
    uint64_t a, b;           // values in [a, b)
    uint64_t* out;           // device
    uint64_t cap;
};

// Leaf i of a tree of depth D over N positions that holds 0-based position
// `pos` (leaf ranges split at floor(S/2) and do not depend on the sample).
uint64_t leaf_of_position(uint64_t N, int D, uint64_t pos);

// Split-tree depth for n samples (the least D with n <= n0 2^D, lowered
// until 2^D <= N).
int plan_depth(uint64_t n, uint64_t N, uint32_t n0);

class GroupPlan {
public:
    // Plans requests (out_ptrs[r] non-null: request r writes there instead of
    // pool + out_off) and queries.  Requests with bad arguments get their
    // error in their status word at run time.  Queries must be valid.
    void build(const rs_request* reqs, uint64_t* const* out_ptrs, uint32_t R, const GroupQuery* qs, uint32_t Q);

    uint64_t upload_bytes() const { return up_bytes_; }
    uint64_t work_bytes() const { return work_bytes_; }
    uint64_t big_kmax() const { return big_kmax_; }
    uint32_t requests() const { return R_; }
    uint32_t queries() const { return Q_; }

    // Fixes device addresses (upload image at `up`, work area at `work`,
    // the general path's pool of big_pool_bytes(big_kmax()) at `big`), then
    // fills the upload image in host memory `img` (upload_bytes() bytes).
    void bind(unsigned char* up, unsigned char* work, void* big, unsigned char* img);

    // Device addresses of the query results (QueryRes[Q]) after bind().
    QueryRes* query_results() const { return qres_; }

    // Issues the group's device work on `st`: zeroing, roots, tree levels,
    // leaves of the requests; boundary leaves, locate, interior leaves of the
    // queries.  `status` holds R words (set by the run).
    int issue(const double* tab, int sms, uint64_t* pool, int* status, cudaStream_t st, uint64_t* launches);

    // Leaf-kernel blocks per SM for every leaf group (0 = occupancy limit).
    void set_blocks_per_sm(int per) { per_sm_ = per; }
    int blocks_per_sm() const { return per_sm_; }

    // Threads of the leaf kernels (256 or 512; 0 = the class's default: 256
    // for the small class, 512 for the large) of the small and the large
    // size class.  Output-invariant, like the blocks per SM.
    void set_leaf_threads(int small, int large) {
        threads_[0] = small;
        threads_[1] = large;
    }
    int leaf_threads(bool large) const { return threads_[large ? 1 : 0]; }
    // Whether the plan has request or query leaves of the size class.
    bool has_class(bool large) const;

    // Leaf groups: (H, WR) x (32-, 64-bit keys) x (small, large class), and
    // Algorithm B.
    static constexpr int kGroups = 11;

    // Leaf kernels with one block per leaf instead of a persistent grid, so
    // that their blocks retire often and kernels of other streams (a
    // server's other lanes) get SMs between them.
    void set_persistent(bool p) { persistent_ = p; }

    // Upper bounds of what one request or query adds to a group.
    static void request_cost(const rs_request& q, uint64_t* up, uint64_t* work);
    static void query_cost(const TreeInfo& t, uint64_t a, uint64_t b, uint64_t* up, uint64_t* work);
    static constexpr uint64_t kFixedCost = 64 * 256;   // alignment slack of one group

private:
    struct Sub {   // a leaf group (requests) or query subgroup, one kernel flavour
        int kind = 0;
        bool wide = false;
        bool large = false;
        bool compact = false;   // 64-bit keys, small means: the compact table (requests only)
        // requests: leaf descriptors; queries: bound items, then interior q_of/prefix
        std::vector<LeafDesc> desc;
        std::vector<uint32_t> a32, b32;
        std::vector<uint64_t> p64;
        uint64_t n1 = 0, n2 = 0;          // leaves (requests) | boundary items, interior leaves (queries)
        size_t o_desc = 0, o_a32 = 0, o_b32 = 0, o_p64 = 0;   // upload offsets
        size_t o_ovf1 = 0, o_ovf2 = 0;                        // work offsets
    };
    std::vector<BatchReq> reqs_;
    std::vector<std::vector<BatchTreeItem>> levels_;
    std::vector<QueryDesc> qdesc_;
    std::vector<uint64_t> qscratch_;   // scratch values per query
    Sub groups_[kGroups], qgroups_[kGroups];
    uint32_t R_ = 0, Q_ = 0;
    uint64_t nodes_ = 0, big_kmax_ = 0;
    // layout
    size_t o_reqs_ = 0, o_qdesc_ = 0;
    std::vector<size_t> o_levels_;
    size_t o_nodes_ = 0, o_zero_ = 0, zero_bytes_ = 0, o_qres_ = 0, o_qscr_ = 0;
    uint64_t up_bytes_ = 0, work_bytes_ = 0;
    // bound addresses
    unsigned char* up_ = nullptr;
    unsigned char* work_ = nullptr;
    void* big_ = nullptr;
    QueryRes* qres_ = nullptr;
    int per_sm_ = 0;
    bool persistent_ = true;
    int threads_[2] = {0, 0};
    int threads_of(const Sub& G) const {
        const int t = threads_[G.large ? 1 : 0];
        return t ? t : (G.large ? 512 : 256);
    }

    void layout();
};

}  // namespace rs
