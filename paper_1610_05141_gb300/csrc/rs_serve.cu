// rs_serve.cu -- serving: continuous batching of sampling jobs and range
// queries on resident trees.
//
// One worker thread owns the device side.  Jobs wait in a FIFO queue; a job
// is admitted when an in-flight slot is free and, if it writes into the
// server's output arena, when a first-fit allocation of its output succeeds.
// Whenever one of the lanes (a stream with its own workspace) is idle and
// jobs are waiting, the worker plans every admissible waiting job as one
// group (rs_group.h: one launch per tree level across all of the group's
// requests, one leaf kernel per leaf kind, the three steps of the queries),
// copies the plan in with one transfer, issues it and records an event.
// Groups on different lanes overlap on the device; jobs that arrive while
// groups run go out with the next idle lane.  Results (status, count, where
// the values are) come back through the poll call; arena memory stays
// reserved until the client releases the job.
//
// Lane 0 runs at the highest stream priority and takes only small jobs
// (queries, and samples of at most kSmallJob values) from anywhere in the
// queue; the other lanes take jobs in submission order whatever their size,
// so that large jobs cannot be passed over for ever.  Leaf kernels of the
// lanes use one block per leaf, so their blocks retire often and a small
// job's kernels do not wait for a large job's whole kernel.
//
// Every job's values equal those of its single call: a sample depends on
// its own (n, N, seed, n0) only (Sec. 4.5), a query on its tree's records.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "rs_group.h"

namespace rs {
int ctx_device(rs_ctx* ctx);
int ctx_sms(rs_ctx* ctx);
const double* ctx_tab(rs_ctx* ctx);
const TreeInfo* tree_info(const rs_tree* t);
int tree_device(const rs_tree* t);
uint64_t tree_samples(const rs_tree* t);
}  // namespace rs

namespace {

using Clock = std::chrono::steady_clock;

constexpr uint64_t kSmallJob = 1ull << 20;   // samples of a job lane 0 takes

int cuda_rc(cudaError_t e) {
    if (e == cudaSuccess) return RS_OK;
    return e == cudaErrorMemoryAllocation ? RS_ENOMEM : RS_ECUDA;
}

// First-fit allocator over [0, size) with coalescing of free blocks.
class Arena {
public:
    static constexpr uint64_t kGrain = 256;
    void reset(uint64_t size) {
        free_.clear();
        size_ = size & ~(kGrain - 1);
        if (size_) free_[0] = size_;
        used_ = 0;
    }
    uint64_t size() const { return size_; }
    uint64_t used() const { return used_; }
    static uint64_t round(uint64_t bytes) { return (std::max<uint64_t>(bytes, 1) + kGrain - 1) & ~(kGrain - 1); }
    bool alloc(uint64_t bytes, uint64_t* off) {
        const uint64_t need = round(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < need) continue;
            *off = it->first;
            const uint64_t rest = it->second - need;
            const uint64_t at = it->first + need;
            free_.erase(it);
            if (rest) free_[at] = rest;
            used_ += need;
            return true;
        }
        return false;
    }
    void release(uint64_t off, uint64_t bytes) {
        const uint64_t len = round(bytes);
        used_ -= len;
        auto next = free_.lower_bound(off);
        uint64_t start = off, end = off + len;
        if (next != free_.end() && next->first == end) {
            end += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == start) {
                start = prev->first;
                free_.erase(prev);
            }
        }
        free_[start] = end - start;
    }

private:
    std::map<uint64_t, uint64_t> free_;   // offset -> length
    uint64_t size_ = 0, used_ = 0;
};

struct Job {
    uint64_t ticket = 0;
    rs_job spec{};
    uint64_t* out = nullptr;
    uint64_t arena_off = ~0ull;   // arena block, if any
    uint64_t arena_bytes = 0;
    uint64_t cost_up = 0, cost_work = 0;
    double t_submit = 0, t_launch = 0, t_done = 0;
    int32_t status = RS_OK;
    uint64_t count = 0;
    bool done = false;
    bool small = false;           // lane 0 may take it out of order
};

struct Lane {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    unsigned char* up = nullptr;
    unsigned char* work = nullptr;
    void* big = nullptr;
    uint64_t up_cap = 0, work_cap = 0;
    unsigned char* img = nullptr;       // pinned, up_cap bytes
    int32_t* status_dev = nullptr;      // max_group words
    int32_t* status_host = nullptr;     // pinned
    rs::QueryRes* qres_host = nullptr;  // pinned, max_group entries
    std::vector<uint64_t> reqs, queries;   // tickets in plan order
    rs::GroupPlan plan;
    bool busy = false;
};

}  // namespace

struct rs_server {
    int device = 0;
    int sms = 0;
    const double* tab = nullptr;
    rs_server_config cfg{};
    unsigned char* arena_dev = nullptr;
    Arena arena;
    std::vector<Lane> lanes;
    Clock::time_point t0;

    std::mutex mu;
    std::condition_variable cv_work;   // the worker waits for submissions
    std::condition_variable cv_done;   // pollers wait for results
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, Job> jobs;   // not yet released
    std::deque<uint64_t> completed;            // not yet polled
    uint64_t next_ticket = 1;
    uint32_t inflight = 0;
    uint32_t fail_plans = 0;   // testing knob: plans that fail as if host memory ran out
    rs_server_stats stats{};
    bool stop = false;
    std::thread worker;

    double now_ms() const { return std::chrono::duration<double, std::milli>(Clock::now() - t0).count(); }
};

namespace {

// Marks a job finished (lock held).
void finish(rs_server* S, Job& j, int status, uint64_t count, double t) {
    j.status = status;
    j.count = count;
    j.t_done = t;
    j.done = true;
    S->completed.push_back(j.ticket);
    S->stats.completed++;
}

// Collects the results of lanes whose group has finished.
bool retire(rs_server* S) {
    bool any = false;
    for (Lane& L : S->lanes) {
        if (!L.busy) continue;
        const cudaError_t e = cudaEventQuery(L.ev);
        if (e == cudaErrorNotReady) continue;
        const int err = e == cudaSuccess ? RS_OK : RS_ECUDA;
        const double t = S->now_ms();
        std::lock_guard<std::mutex> lock(S->mu);
        for (size_t i = 0; i < L.reqs.size(); ++i) {
            Job& j = S->jobs[L.reqs[i]];
            finish(S, j, err ? err : L.status_host[i], err ? 0 : j.spec.n, t);
        }
        for (size_t i = 0; i < L.queries.size(); ++i) {
            Job& j = S->jobs[L.queries[i]];
            finish(S, j, err ? err : L.qres_host[i].status, err ? 0 : L.qres_host[i].count, t);
        }
        S->inflight -= (uint32_t)(L.reqs.size() + L.queries.size());
        L.reqs.clear();
        L.queries.clear();
        L.busy = false;
        any = true;
    }
    if (any) S->cv_done.notify_all();
    return any;
}

// Admits waiting jobs into an idle lane's group and issues it.  Lane 0
// (small_only) takes the small jobs in queue order and skips the others; the
// other lanes take the queue's head in order and stop at the first job that
// does not fit.
bool launch(rs_server* S, Lane& L, bool small_only) {
    std::vector<Job*> batch;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        uint64_t up = rs::GroupPlan::kFixedCost, work = rs::GroupPlan::kFixedCost;
        std::deque<uint64_t> skipped;
        while (!S->pending.empty() && S->inflight < S->cfg.max_inflight && batch.size() < S->cfg.max_group) {
            Job& j = S->jobs[S->pending.front()];
            if (small_only && !j.small) {
                if (skipped.size() >= S->cfg.max_group) break;   // bounded look-ahead
                skipped.push_back(S->pending.front());
                S->pending.pop_front();
                continue;
            }
            if (up + j.cost_up > L.up_cap || work + j.cost_work > L.work_cap) break;
            if (!j.spec.out_dev) {
                uint64_t off = 0;
                if (!S->arena.alloc(j.arena_bytes, &off)) break;   // wait for memory
                j.arena_off = off;
                j.out = reinterpret_cast<uint64_t*>(S->arena_dev + off);
                S->stats.peak_arena_bytes = std::max<uint64_t>(S->stats.peak_arena_bytes, S->arena.used());
            }
            up += j.cost_up;
            work += j.cost_work;
            S->pending.pop_front();
            S->inflight++;
            batch.push_back(&j);
        }
        // skipped jobs go back to the front, in their order
        while (!skipped.empty()) {
            S->pending.push_front(skipped.back());
            skipped.pop_back();
        }
        S->stats.peak_inflight = std::max<uint64_t>(S->stats.peak_inflight, S->inflight);
    }
    if (batch.empty()) return false;
    // plan: requests first, then queries (jobs map entries are stable while
    // admitted: only release erases, and only finished jobs)
    std::vector<rs_request> reqs;
    std::vector<uint64_t*> outs;
    std::vector<rs::GroupQuery> qs;
    L.reqs.clear();
    L.queries.clear();
    for (Job* j : batch) {
        if (j->spec.op == RS_OP_SAMPLE) {
            reqs.push_back(rs_request{j->spec.n, j->spec.N, j->spec.seed, 0, j->spec.n0, j->spec.kind});
            outs.push_back(j->out);
            L.reqs.push_back(j->ticket);
        } else {
            const rs::TreeInfo* t = rs::tree_info(j->spec.tree);
            const uint64_t lo = j->spec.a < 1 ? 1 : j->spec.a;
            const uint64_t hi = j->spec.b > t->N + 1 ? t->N + 1 : j->spec.b;
            qs.push_back(rs::GroupQuery{t, lo, hi, j->out, j->spec.cap});
            L.queries.push_back(j->ticket);
        }
    }
    const double t_launch = S->now_ms();
    int rc = RS_OK;
    bool inject = false;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        if (S->fail_plans) {
            S->fail_plans--;
            inject = true;
        }
    }
    try {
        if (inject) throw std::bad_alloc();
        L.plan.build(reqs.data(), outs.data(), (uint32_t)reqs.size(), qs.data(), (uint32_t)qs.size());
    } catch (const std::bad_alloc&) {
        rc = RS_ENOMEM;
    }
    if (!rc && (L.plan.upload_bytes() > L.up_cap || L.plan.work_bytes() > L.work_cap)) rc = RS_ECAPACITY;
    uint64_t nl = 0;
    if (!rc) {
        L.plan.set_persistent(false);
        L.plan.bind(L.up, L.work, L.big, L.img);
        rc = cuda_rc(cudaMemcpyAsync(L.up, L.img, L.plan.upload_bytes(), cudaMemcpyHostToDevice, L.st));
        if (!rc) rc = L.plan.issue(S->tab, S->sms, nullptr, L.status_dev, L.st, &nl);
        if (!rc && !reqs.empty())
            rc = cuda_rc(cudaMemcpyAsync(L.status_host, L.status_dev, reqs.size() * sizeof(int32_t),
                                         cudaMemcpyDeviceToHost, L.st));
        if (!rc && !qs.empty())
            rc = cuda_rc(cudaMemcpyAsync(L.qres_host, L.plan.query_results(), qs.size() * sizeof(rs::QueryRes),
                                         cudaMemcpyDeviceToHost, L.st));
        if (!rc) rc = cuda_rc(cudaEventRecord(L.ev, L.st));
    }
    std::lock_guard<std::mutex> lock(S->mu);
    for (Job* j : batch) j->t_launch = t_launch;
    S->stats.groups++;
    S->stats.launches += nl;
    S->stats.max_group_seen = std::max<uint64_t>(S->stats.max_group_seen, batch.size());
    if (rc) {
        // nothing of this group is in flight once the stream drains
        cudaStreamSynchronize(L.st);
        const double t = S->now_ms();
        for (Job* j : batch) finish(S, *j, rc, 0, t);
        S->inflight -= (uint32_t)batch.size();
        L.reqs.clear();
        L.queries.clear();
        S->cv_done.notify_all();
        return true;
    }
    L.busy = true;
    return true;
}

void worker_main(rs_server* S) {
    cudaSetDevice(S->device);
    for (;;) {
        {
            std::lock_guard<std::mutex> lock(S->mu);
            if (S->stop) break;
        }
        bool did = retire(S);
        bool busy = false;
        for (size_t li = 0; li < S->lanes.size(); ++li) {
            Lane& L = S->lanes[li];
            if (L.busy) {
                busy = true;
                continue;
            }
            if (launch(S, L, li == 0 && S->lanes.size() > 1)) {
                did = true;
                busy = true;
            }
        }
        if (did) continue;
        if (busy) {
            std::this_thread::yield();   // groups in flight: poll their events
            continue;
        }
        std::unique_lock<std::mutex> lock(S->mu);
        S->cv_work.wait_for(lock, std::chrono::milliseconds(2), [S] { return S->stop || !S->pending.empty(); });
    }
}

void free_lanes(rs_server* S) {
    for (Lane& L : S->lanes) {
        if (L.st) cudaStreamSynchronize(L.st);
        if (L.ev) cudaEventDestroy(L.ev);
        if (L.st) cudaStreamDestroy(L.st);
        cudaFree(L.up);
        cudaFree(L.work);
        cudaFree(L.big);
        cudaFree(L.status_dev);
        if (L.img) cudaFreeHost(L.img);
        if (L.status_host) cudaFreeHost(L.status_host);
        if (L.qres_host) cudaFreeHost(L.qres_host);
    }
    S->lanes.clear();
}

}  // namespace

extern "C" {

int rs_server_destroy(rs_server* S) {
    if (!S) return RS_OK;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    free_lanes(S);
    cudaFree(S->arena_dev);
    if (prev >= 0) cudaSetDevice(prev);
    delete S;
    return RS_OK;
}

int rs_server_create(rs_ctx* ctx, const rs_server_config* cfg, rs_server** out) {
    if (!ctx || !out) return RS_EINVAL;
    *out = nullptr;
    rs_server_config c{};
    c.arena_bytes = 1ull << 30;
    if (cfg) c = *cfg;
    if (c.max_inflight == 0) c.max_inflight = 4096;
    if (c.lanes == 0) c.lanes = 4;
    if (c.max_group == 0) c.max_group = 4096;
    if (c.lane_bytes == 0) c.lane_bytes = 256ull << 20;
    if (c.lanes > 64 || c.lane_bytes < (1ull << 20)) return RS_EINVAL;
    rs_server* S = new (std::nothrow) rs_server();
    if (!S) return RS_ENOMEM;
    S->device = rs::ctx_device(ctx);
    S->sms = rs::ctx_sms(ctx);
    S->tab = rs::ctx_tab(ctx);
    S->cfg = c;
    int prev = -1;
    cudaGetDevice(&prev);
    int rc = cuda_rc(cudaSetDevice(S->device));
    if (!rc && c.arena_bytes) rc = cuda_rc(cudaMalloc(&S->arena_dev, c.arena_bytes));
    S->arena.reset(c.arena_bytes);
    try {
        S->lanes.resize(c.lanes);
    } catch (const std::bad_alloc&) {
        rc = RS_ENOMEM;
    }
    const uint64_t big_bytes = rs::big_pool_bytes(rs::kBigLeafMax);
    for (Lane& L : S->lanes) {
        if (rc) break;
        L.up_cap = c.lane_bytes / 4;
        L.work_cap = c.lane_bytes - L.up_cap;
        int least = 0, greatest = 0;
        cudaDeviceGetStreamPriorityRange(&least, &greatest);
        const bool first = &L == &S->lanes[0];
        rc = cuda_rc(cudaStreamCreateWithPriority(&L.st, cudaStreamNonBlocking, first ? greatest : least));
        if (!rc) rc = cuda_rc(cudaEventCreateWithFlags(&L.ev, cudaEventDisableTiming));
        if (!rc) rc = cuda_rc(cudaMalloc(&L.up, L.up_cap));
        if (!rc) rc = cuda_rc(cudaMalloc(&L.work, L.work_cap));
        if (!rc) rc = cuda_rc(cudaMalloc(&L.big, big_bytes));
        if (!rc) rc = cuda_rc(cudaMalloc(&L.status_dev, c.max_group * sizeof(int32_t)));
        if (!rc) rc = cuda_rc(cudaMallocHost(&L.img, L.up_cap));
        if (!rc) rc = cuda_rc(cudaMallocHost(&L.status_host, c.max_group * sizeof(int32_t)));
        if (!rc) rc = cuda_rc(cudaMallocHost(&L.qres_host, c.max_group * sizeof(rs::QueryRes)));
    }
    if (prev >= 0) cudaSetDevice(prev);
    if (rc) {
        rs_server_destroy(S);
        return rc;
    }
    S->t0 = Clock::now();
    try {
        S->worker = std::thread(worker_main, S);
    } catch (...) {
        rs_server_destroy(S);
        return RS_ENOMEM;
    }
    *out = S;
    return RS_OK;
}

int rs_server_submit(rs_server* S, const rs_job* spec, uint64_t* ticket) {
    if (!S || !spec || !ticket) return RS_EINVAL;
    if (spec->op == RS_OP_QUERY && !spec->tree) return RS_EINVAL;
    if (spec->op != RS_OP_SAMPLE && spec->op != RS_OP_QUERY) return RS_EINVAL;
    Job j;
    j.spec = *spec;
    j.out = spec->out_dev;
    int immediate = -1;     // status of a job that completes at once
    uint64_t values = 0;    // output values the job needs room for
    if (spec->out_dev && ((uintptr_t)spec->out_dev & 7)) immediate = RS_EINVAL;
    if (immediate < 0 && spec->op == RS_OP_SAMPLE) {
        const bool wr = spec->kind == RS_KIND_WR;
        if (spec->kind > RS_KIND_B || spec->n0 == 0 || spec->N > (1ull << 62) || (spec->n > 0 && spec->N == 0) ||
            (!wr && spec->n > spec->N))
            immediate = RS_EINVAL;
        else if (rs::plan_depth(spec->n, spec->N, spec->n0) > rs::kMaxDepth)
            immediate = RS_ECAPACITY;
        else if (spec->n == 0)
            immediate = RS_OK;
        else {
            const rs_request q{spec->n, spec->N, spec->seed, 0, spec->n0, spec->kind};
            rs::GroupPlan::request_cost(q, &j.cost_up, &j.cost_work);
            values = spec->n;
            j.small = spec->n <= kSmallJob;
        }
    } else if (immediate < 0) {
        const rs::TreeInfo* t = rs::tree_info(spec->tree);
        const uint64_t lo = spec->a < 1 ? 1 : spec->a;
        const uint64_t hi = spec->b > t->N + 1 ? t->N + 1 : spec->b;
        if (rs::tree_device(spec->tree) != S->device) immediate = RS_EINVAL;
        else if (rs::tree_samples(spec->tree) == 0 || lo >= hi) immediate = RS_OK;
        else {
            rs::GroupPlan::query_cost(*t, lo, hi, &j.cost_up, &j.cost_work);
            values = spec->cap;
            j.small = true;
        }
    }
    if (immediate < 0 && !spec->out_dev) {
        j.arena_bytes = values * 8;
        if (Arena::round(j.arena_bytes) > S->arena.size()) immediate = RS_ECAPACITY;
    }
    if (immediate < 0) {
        const uint64_t up_cap = S->cfg.lane_bytes / 4, work_cap = S->cfg.lane_bytes - up_cap;
        if (j.cost_up + rs::GroupPlan::kFixedCost > up_cap || j.cost_work + rs::GroupPlan::kFixedCost > work_cap)
            immediate = RS_ECAPACITY;
    }
    {
        std::lock_guard<std::mutex> lock(S->mu);
        j.ticket = S->next_ticket++;
        j.t_submit = S->now_ms();
        *ticket = j.ticket;
        S->stats.submitted++;
        Job& slot = S->jobs[j.ticket] = j;
        if (immediate >= 0) {
            finish(S, slot, immediate, 0, slot.t_submit);
        } else {
            S->pending.push_back(j.ticket);
        }
    }
    if (immediate >= 0) S->cv_done.notify_all();
    else S->cv_work.notify_one();
    return RS_OK;
}

int rs_server_poll(rs_server* S, rs_result* results, uint32_t max, uint32_t* got, uint32_t wait_us) {
    if (!S || !got || (max > 0 && !results)) return RS_EINVAL;
    *got = 0;
    std::unique_lock<std::mutex> lock(S->mu);
    if (S->completed.empty() && wait_us > 0)
        S->cv_done.wait_for(lock, std::chrono::microseconds(wait_us), [S] { return !S->completed.empty(); });
    while (*got < max && !S->completed.empty()) {
        const Job& j = S->jobs[S->completed.front()];
        S->completed.pop_front();
        rs_result& r = results[(*got)++];
        r.ticket = j.ticket;
        r.status = j.status;
        r.reserved = 0;
        r.count = j.count;
        r.out_dev = j.out;
        r.submit_ms = j.t_submit;
        r.launch_ms = j.t_launch;
        r.done_ms = j.t_done;
    }
    return RS_OK;
}

int rs_server_release(rs_server* S, uint64_t ticket) {
    if (!S) return RS_EINVAL;
    bool freed = false;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        auto it = S->jobs.find(ticket);
        if (it == S->jobs.end() || !it->second.done) return RS_EINVAL;
        if (it->second.arena_off != ~0ull) {
            S->arena.release(it->second.arena_off, it->second.arena_bytes);
            freed = true;
        }
        S->jobs.erase(it);
    }
    if (freed) S->cv_work.notify_one();
    return RS_OK;
}

int rs_server_fail_next_plans(rs_server* S, uint32_t count) {
    if (!S) return RS_EINVAL;
    std::lock_guard<std::mutex> lock(S->mu);
    S->fail_plans = count;
    return RS_OK;
}

int rs_server_stats_get(rs_server* S, rs_server_stats* out) {
    if (!S || !out) return RS_EINVAL;
    std::lock_guard<std::mutex> lock(S->mu);
    *out = S->stats;
    out->arena_bytes_in_use = S->arena.used();
    return RS_OK;
}

}  // extern "C"
