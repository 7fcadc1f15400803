/*
 * rs.h -- C ABI of the GB300 divide-and-conquer random sampler.
 *
 * Sanders, Lamm, Huebschle-Schneider, Schrade, Dachsbacher, "Efficient
 * Parallel Random Sampling -- Vectorized, Cache-Efficient, and Online"
 * (ACM TOMS 44(3), 2018).
 *
 * The sampler draws n numbers from 1..N (Sec. 1-2).  The range is split
 * recursively at floor(S/2); a hypergeometric deviate (binomial when sampling
 * with replacement, Sec. 4.6) gives each half its share (Sec. 3.1 Algorithm
 * R).  Every tree node and every leaf draws from a Philox4x32-10 stream keyed
 * by the seed and the node id, so no node waits for another (Sec. 3.2
 * Algorithm P), and the result is a pure function of (n, N, seed, n0)
 * whatever the launch geometry (Sec. 4.5).  Leaves produce their share with
 * hash-style rejection (Sec. 2 Algorithm H, sorted as in Sec. 4.1) or with
 * Bernoulli skips plus a repair (Sec. 2 Algorithm B).
 *
 * Conventions for every call:
 *  - Device pointers ("_dev") are CUDA device memory owned by the caller
 *    (e.g. a torch tensor's data_ptr()); host pointers are plain host memory.
 *  - Output values are 1-based uint64 in 1..N.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Sampling calls are asynchronous on that stream; errors the device detects
 *    (an iteration cap, a leaf capacity) land in the context's status word and
 *    are returned by rs_sync.  Argument errors are returned immediately.
 *  - A context may be used from one host thread at a time; calls that share a
 *    context must be issued on one stream (they share its scratch memory).
 *  - Return codes are the RS_* values below.
 */
#ifndef RS_H
#define RS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    RS_OK = 0,
    RS_EINVAL = 1,     /* invalid argument                                    */
    RS_ECAPACITY = 2,  /* a result does not fit the caller's buffer or a limit */
    RS_ENOMEM = 3,     /* device or host allocation failed                    */
    RS_ECUDA = 4,      /* a CUDA runtime call failed                          */
    RS_ETIMEOUT = 5,   /* a bounded wait gave up                              */
    RS_EITER = 6       /* a rejection loop reached its iteration cap          */
};

/* Kinds of sample (also the `kind` field of rs_request). */
enum {
    RS_KIND_H = 0,   /* without replacement, hypergeometric splits, leaf H (Sec. 2, 3.1, 4.1) */
    RS_KIND_WR = 1,  /* with replacement, binomial splits (Sec. 4.6)                         */
    RS_KIND_B = 2    /* without replacement, Algorithm B as the base case (Sec. 2, 4.7)      */
};

typedef struct rs_ctx rs_ctx;
typedef struct rs_tree rs_tree;

/* Creates a context on CUDA device `device` (scratch memory, status word, the
 * ln x! table).  *ctx is owned by the caller and freed with rs_destroy.
 * Errors: RS_EINVAL (null ctx), RS_ECUDA (bad device), RS_ENOMEM. */
int rs_create(rs_ctx** ctx, int device);

/* Waits for the context's work, frees its memory.  Returns RS_OK or RS_ECUDA. */
int rs_destroy(rs_ctx* ctx);

/* Split-tree depth D for n samples (a1 plan): the least D >= 0 with
 * n <= n0 * 2^D, lowered until 2^D <= N.  The static depth replaces Algorithm
 * R's adaptive "n < n0" stop (Sec. 3.1) the way Algorithm P's fixed tree of
 * PEs does (Sec. 3.2, Sec. 4.5).  Host only.  Errors: RS_EINVAL (null out,
 * n0 = 0). */
int rs_plan(uint64_t n, uint64_t N, uint32_t n0, int* depth_out);

/* n distinct values from 1..N, strictly increasing, written to out_dev[0..n)
 * (Sec. 3.1 Algorithm R with Algorithm H leaves, sorted output Sec. 4.1).
 * out_dev: n uint64 slots of device memory, 8-byte aligned.
 * Errors: RS_EINVAL (n > N, n > 0 with N = 0, N > 2^62, n0 = 0, null out
 * with n > 0); device-side RS_EITER / RS_ECAPACITY via rs_sync.
 * n = 0 succeeds and writes nothing. */
int rs_sample(rs_ctx* ctx, uint64_t n, uint64_t N, uint64_t seed, uint32_t n0,
              uint64_t* out_dev, void* stream);

/* n values from 1..N drawn with replacement, non-decreasing (Sec. 4.6:
 * binomial splits).  n may exceed N.  Same buffers and errors as rs_sample
 * (except that n > N is allowed). */
int rs_sample_with_replacement(rs_ctx* ctx, uint64_t n, uint64_t N, uint64_t seed, uint32_t n0,
                               uint64_t* out_dev, void* stream);

/* Like rs_sample, with Algorithm B (Bernoulli sampling with a slightly larger
 * rate, then removal of the surplus) as the base case of the split tree
 * (Sec. 2, Sec. 4.7).  A uniform n-subset like rs_sample, but a different
 * one: the leaves draw from other streams. */
int rs_sample_b(rs_ctx* ctx, uint64_t n, uint64_t N, uint64_t seed, uint32_t n0,
                uint64_t* out_dev, void* stream);

/* rs_sample / rs_sample_with_replacement / rs_sample_b (by `kind`, an
 * RS_KIND_* value) with the sample also copied to host memory
 * out_host[0..n) while it is produced: once the split tree is done the
 * output is cut at eight leaf boundaries (a small read-back that waits for
 * the tree), and each piece goes to the host on a second stream as soon as
 * its leaves are written, while the next piece's leaves run.  out_dev: n
 * device slots (the sample, as with rs_sample); out_host: n slots of
 * page-locked host memory (cudaHostAlloc, torch's pin_memory) -- pageable
 * memory works but the copies then do not overlap.  Returns before the
 * copies finish; later work on `stream`, rs_sync and a synchronize of
 * `stream` wait for them.  The paper has no counterpart (its GPU timings
 * note that the transfer to the CPU dominated).  Errors: as rs_sample, and
 * RS_EINVAL for a bad kind or a null out_host with n > 0. */
int rs_sample_to_host(rs_ctx* ctx, int kind, uint64_t n, uint64_t N, uint64_t seed, uint32_t n0,
                      uint64_t* out_dev, uint64_t* out_host, void* stream);

/* Leaf records of the split tree of (n, N, seed, n0): recs_dev[4i..4i+3] =
 * (lo, s, n', offset) of leaf i (0-based, left to right): leaf i covers the
 * 0-based positions [lo, lo+s), holds n' samples and writes them at
 * out[offset..offset+n').  kind RS_KIND_WR uses binomial splits, the other
 * kinds hypergeometric splits (Sec. 3.1, 3.2, 4.6).  recs_dev: 4*2^D uint64
 * of device memory with 2^D <= max_leaves, else RS_ECAPACITY. */
int rs_split_tree(rs_ctx* ctx, uint64_t n, uint64_t N, uint64_t seed, uint32_t n0, int kind,
                  uint64_t* recs_dev, uint64_t max_leaves, void* stream);

/* Bernoulli(p) sample of the positions 0..N-1 by independent chunks with
 * geometric skips (Sec. 4.7, Sec. 2 Algorithm B), restricted to the window
 * [a, b) of 0-based positions.  Scratch: the chunk counts, and the staging
 * area of rs_set_bernoulli_staging.  Chunks have 2^c positions, c the least value
 * with 2^c p >= n0 (at most 62); a and b must be multiples of 2^c (b may also
 * equal N).  Writes the 1-based positions in increasing order to
 * out_dev[0..min(count, cap)) and the number in the window to *count_out
 * (host memory); this call synchronizes `stream` to read the count.
 * Errors: RS_EINVAL (p outside [0,1], n0 = 0, N > 2^62, bad window),
 * RS_ECAPACITY (count > cap; *count_out is still set, the first cap values
 * are written), RS_EITER. */
int rs_bernoulli(rs_ctx* ctx, double p, uint64_t N, uint64_t seed, uint32_t n0,
                 uint64_t a, uint64_t b, uint64_t* out_dev, uint64_t cap,
                 uint64_t* count_out, void* stream);

/* ---- Batches: many independent requests in one device run -------------
 * Each request is its own sample (own tree, own seed), exactly the output of
 * the corresponding single call (kind RS_KIND_H: rs_sample, RS_KIND_WR:
 * rs_sample_with_replacement, RS_KIND_B: rs_sample_b): the result depends on
 * the request alone (Sec. 4.5), and requests need no coordination (Sec.
 * 3.2).  Request r writes its n values at out_pool[out_off .. out_off + n);
 * the caller keeps the ranges disjoint. */
typedef struct {
    uint64_t n, N, seed, out_off;
    uint32_t n0, kind;
} rs_request;

typedef struct rs_batchplan rs_batchplan;

/* Plans a batch from host-resident requests: validates them (a request with
 * bad arguments gets RS_EINVAL in its status word at every run and does no
 * work), lays out the node records of all trees, the per-level work items and
 * the leaf groups, and allocates the plan's device memory.  The context must
 * outlive the plan.  Errors: RS_EINVAL, RS_ENOMEM, RS_ECUDA. */
int rs_batch_plan(rs_ctx* ctx, const rs_request* reqs_host, uint32_t R, rs_batchplan** plan);

/* Runs a plan on `stream` (asynchronous; device work only).  status_dev:
 * R int32 words of device memory, set by the run (RS_OK, RS_EINVAL,
 * RS_ECAPACITY, RS_EITER per request).  The first run issues plain launches;
 * later runs replay a CUDA graph captured for (out_pool_dev, status_dev)
 * (captured again if those pointers change). */
int rs_batch_run(rs_batchplan* plan, uint64_t* out_pool_dev, int32_t* status_dev, void* stream);

/* Picks, by timing whole runs, the leaf kernels' blocks per SM and then the
 * leaf block shape of each size class of leaves (output-invariant knobs:
 * the schedule of leaves over blocks and the block's shape never change a
 * value; Sec. 4.2 and 4.5).  Synchronizes `stream`. */
int rs_batch_tune(rs_batchplan* plan, uint64_t* out_pool_dev, int32_t* status_dev, void* stream);

/* Sets the leaf kernels' launch directly (what rs_batch_tune chooses):
 * the threads of the leaf blocks for the small and the large size class
 * (256 or 512; 0 = the class's default, 256 for leaves averaging up to
 * about 4,100 values and 512 above), and the leaf blocks per SM (0 = the
 * occupancy limit).  Output-invariant: no setting changes a value.  The
 * next run captures its graph again.  Errors: RS_EINVAL. */
int rs_batch_set_leaf_launch(rs_batchplan* plan, int small_threads, int large_threads, int blocks_per_sm);

/* Kernels one run launches. */
int rs_batch_launch_count(rs_batchplan* plan, uint64_t* per_run);

/* Waits for the device and frees the plan. */
int rs_batch_destroy(rs_batchplan* plan);

/* One-shot batch from device-resident requests: copies them to the host,
 * plans, runs, waits for `stream` and frees the plan. */
int rs_batch(rs_ctx* ctx, const rs_request* reqs_dev, uint32_t R, uint64_t* out_pool_dev,
             int32_t* status_dev, void* stream);

/* ---- Union of uneven segments (Sec. 4.3) -------------------------------
 * A universe made of p segments of sizes L[0..p) (the elements of segment i
 * are its positions 1..L[i]); the sample is a uniform n-subset of the union.
 * As with the paper's owners of uneven shares, the samples per segment come
 * first, from a binary tree of hypergeometric splits over the segments
 * (padded with empty segments to a power of two P; heap-numbered nodes, root
 * 1, segment i at node P + i): node v's c samples give HG(c, sum of its left
 * half's sizes, sum of its sizes) of stream (SPLIT, v), key seed, to the left
 * child and the rest to the right child.  Then each segment with samples
 * draws them alone (owner computes) as rs_sample(count_i, L[i],
 * rs_union_key(seed, i), n0).  L_host: p host words, sum at most 2^62;
 * p <= 2^24. */

/* Segment i's key: seed + (i + 1) * 0x9E3779B97F4A7C15 (mod 2^64). */
uint64_t rs_union_key(uint64_t seed, uint32_t i);

/* The count tree on the device; counts_host[0..p) (host memory) receives the
 * samples per segment.  Synchronizes `stream`.  Errors: RS_EINVAL (bad
 * sizes, n above their sum), RS_ENOMEM, RS_ECUDA, RS_EITER. */
int rs_union_counts(rs_ctx* ctx, const uint64_t* L_host, uint32_t p, uint64_t n, uint64_t seed,
                    uint64_t* counts_host, void* stream);

/* The union's sample: segment after segment, each segment's values as
 * increasing positions within it (1..L[i]), at out_dev[0..n) (device memory,
 * 8-byte aligned); counts_host[0..p) as rs_union_counts.  The segments' samples
 * run as one batch (rs_batch_plan / rs_batch_run of the segments with
 * samples).  Synchronizes `stream`.  Errors: as rs_union_counts and
 * rs_batch_plan, RS_EINVAL for n0 = 0, and a request's status error. */
int rs_union_sample(rs_ctx* ctx, const uint64_t* L_host, uint32_t p, uint64_t n, uint64_t seed, uint32_t n0,
                    uint64_t* out_dev, uint64_t* counts_host, void* stream);

/* ---- Online sorted sampling by peeling (Sec. 4.1) ----------------------
 * An iterator over a sample of n from 1..N in increasing order, in batches
 * of about n0 values, each made in O(n0) work (the paper's constant delay
 * per sample for constant n0).  With n_t samples left among the N_t
 * positions after the first lo_t (n_0 = n, N_0 = N, lo_0 = 0), batch t
 * (t = 0, 1, ...) splits off the next m_t = ceil(N_t n0 / n_t) positions and
 * takes c_t = HG(n_t, m_t, N_t) of the samples, the deviate of stream
 * (SPLIT, t + 1); once m_t >= N_t the batch is the rest (m_t = N_t,
 * c_t = n_t) and the last.  Batch t's values are the leaf H values of node
 * t + 1 over [lo_t, lo_t + m_t) with c_t samples (as in rs_sample's leaves).
 * A different sample from rs_sample's with the same arguments, with the
 * same distribution. */
typedef struct rs_peel rs_peel;

/* Creates the iterator (device state, room for max_batches batches per
 * call, 1 <= max_batches <= 2^20).  It uses the context's table and must be
 * destroyed before it.  Errors: RS_EINVAL (n > N, N > 2^62, n0 = 0, bad
 * max_batches), RS_ENOMEM, RS_ECUDA. */
int rs_peel_create(rs_ctx* ctx, uint64_t n, uint64_t N, uint64_t seed, uint32_t n0, uint32_t max_batches,
                   rs_peel** it);

/* Makes the next batches, as many as max_batches allows and whose values
 * all fit in cap, and writes their values in increasing order to
 * out_dev[0 .. *count_out) (device memory, 8-byte aligned); *batches_out =
 * the batches made (batches may be empty).  After the last batch it returns
 * RS_OK with 0 and 0.  Synchronizes `stream`.  Errors: RS_EINVAL,
 * RS_ECAPACITY (not even the next batch fits: *count_out = its size, the
 * state is unchanged), RS_ECUDA, RS_EITER; a device error stays with the
 * iterator. */
int rs_peel_next(rs_peel* it, uint64_t* out_dev, uint64_t cap, uint64_t* count_out, uint32_t* batches_out,
                 void* stream);

/* Samples and positions left and batches made so far.  Errors: RS_EINVAL. */
int rs_peel_state(rs_peel* it, uint64_t* n_left, uint64_t* N_left, uint64_t* batches_done);

/* Waits for the device and frees the iterator. */
int rs_peel_destroy(rs_peel* it);

/* ---- Sampling with replacement from a d-dimensional box (Sec. 4.6) -----
 * n points drawn uniformly and independently from the integer box
 * [0, E_0) x ... x [0, E_{d-1}) by bisection: the split tree of the
 * one-dimensional sampler with replacement (depth as rs_sample's with N =
 * the volume V), over boxes.  Node v (heap numbering, root 1 = the whole box
 * with n points) halves its largest extent e (lowest dimension on ties):
 * the lower half, extent floor(e/2), gets BIN(c, floor(e/2), e) of its c
 * points (stream (SPLIT, v)), the upper half the rest.  Leaf box i (node
 * 2^D + i) draws its points as row-major indices into itself (dimension 0
 * most significant), as the with-replacement leaf of node 2^D + i over
 * [0, its volume) (sorted), and writes their coordinates. */

/* out_dev: n * d uint64 (device memory, 8-byte aligned), point j's 0-based
 * coordinates at out_dev[j d .. j d + d); the points leaf after leaf, each
 * leaf's in row-major order.  1 <= d <= 4, every E_k >= 1, V <= 2^62.
 * Asynchronous after one wait for the tree (the leaves' largest volume and
 * count pick the leaf kernel); device errors as rs_sync.  Errors:
 * RS_EINVAL, RS_ECAPACITY (depth above the library's limit), RS_ENOMEM,
 * RS_ECUDA. */
int rs_points(rs_ctx* ctx, uint32_t d, const uint64_t* extents_host, uint64_t n, uint64_t seed, uint32_t n0,
              uint64_t* out_dev, void* stream);

/* ---- Resident trees and online sorted range queries -------------------
 * A resident tree holds, in device memory owned by the library, the leaf
 * records (range, count, output offset) of the split tree of one sample
 * (Sec. 3.1 Algorithm R; the records fix each leaf's share and output
 * position, Sec. 4.5).  A range query regenerates only the leaves whose
 * ranges overlap the queried values and returns the sample's values inside
 * them in increasing order (Sec. 4.1: sorted generation of a piece of the
 * sample without the rest).  The result equals the slice of the full
 * sample (rs_sample, rs_sample_with_replacement or rs_sample_b with the same
 * arguments) whose values lie in [a, b). */

/* Builds the split tree of (n, N, seed, n0) for sample kind `kind` (an
 * RS_KIND_* value) on `stream` and keeps its leaf records; waits for
 * `stream`.  The tree uses the context (its ln x! table and scratch) and
 * must be destroyed before it.  Device memory: 32 bytes per leaf plus the
 * query workspace.  Errors: RS_EINVAL (as rs_sample, or a bad kind),
 * RS_ECAPACITY (depth above the library's limit), RS_ENOMEM, RS_ECUDA, and
 * the device errors of the tree build (RS_EITER). */
int rs_tree_create(rs_ctx* ctx, uint64_t n, uint64_t N, uint64_t seed, uint32_t n0, int kind, void* stream,
                   rs_tree** tree);

/* Writes the sample's values v with a <= v < b, in increasing order (with
 * repeats for RS_KIND_WR), to out_dev[0..count) and count to *count_out
 * (host memory); synchronizes `stream`.  out_dev: device memory for `cap`
 * uint64 values, 8-byte aligned (may be NULL when cap = 0).  a and b are
 * clamped to 1..N+1; an empty range gives count 0.  Errors: RS_EINVAL,
 * RS_ECAPACITY (count > cap: *count_out is set, out_dev holds no useful
 * values), RS_ENOMEM, RS_ECUDA, RS_EITER.  Queries on one tree must be
 * issued from one host thread (they share the tree's workspace). */
int rs_tree_query(rs_tree* tree, uint64_t a, uint64_t b, uint64_t* out_dev, uint64_t cap, uint64_t* count_out,
                  void* stream);

/* Depth of the tree and its largest leaf count.  Errors: RS_EINVAL. */
int rs_tree_info(rs_tree* tree, int* depth, uint64_t* max_leaf_count);

/* Waits for the device and frees the tree. */
int rs_tree_destroy(rs_tree* tree);

/* ---- Serving: continuous batching of sampling jobs and range queries ----
 * A server owns a worker thread, an output arena in device memory and
 * `lanes` CUDA streams, each with a fixed workspace.  Jobs are admitted in
 * submission order when an in-flight slot is free and, for jobs that write
 * into the arena, when the arena has room for their output (admission by
 * memory).  Whenever a lane is idle and jobs are waiting, the worker issues
 * all admissible waiting jobs as one group on that lane (the batch
 * machinery above: one launch per tree level across the group's requests,
 * one leaf kernel per leaf kind, the three query steps), so jobs that arrive
 * while other groups are running are admitted as slots and memory free up
 * and run alongside them on the device.  Lane 0 runs at the highest stream
 * priority and takes only small jobs (queries, samples of at most 2^20
 * values) from anywhere in the queue; the other lanes take jobs in
 * submission order, so large jobs are never passed over for ever; the
 * lanes' leaf kernels use one block per leaf so that a small job's kernels
 * do not wait for a large job's whole kernel.  A job's result is exactly that of
 * the corresponding single call (rs_sample / rs_sample_with_replacement /
 * rs_sample_b / rs_tree_query): samples depend on their own arguments only
 * (Sec. 4.5).  The paper has no serving layer; this is the library's. */

typedef struct rs_server rs_server;

enum { RS_OP_SAMPLE = 0, RS_OP_QUERY = 1 };

typedef struct {
    uint32_t op;          /* RS_OP_SAMPLE or RS_OP_QUERY                          */
    uint32_t kind;        /* RS_OP_SAMPLE: an RS_KIND_* value                     */
    uint64_t n, N, seed;  /* RS_OP_SAMPLE: as rs_sample                           */
    uint32_t n0;          /* RS_OP_SAMPLE                                         */
    uint32_t reserved;
    rs_tree* tree;        /* RS_OP_QUERY: a tree on the server's device            */
    uint64_t a, b, cap;   /* RS_OP_QUERY: values in [a, b), room for cap of them   */
    uint64_t* out_dev;    /* output buffer (device, 8-byte aligned), or NULL: the
                             server's arena (n values, or cap values for a query) */
} rs_job;

typedef struct {
    uint64_t ticket;
    int32_t status;       /* RS_OK or the job's error                             */
    uint32_t reserved;
    uint64_t count;       /* values written                                       */
    uint64_t* out_dev;    /* where they are; arena memory stays reserved until
                             rs_server_release                                    */
    double submit_ms, launch_ms, done_ms;   /* since the server started; done_ms
                             is when the worker saw the job's group finish        */
} rs_result;

typedef struct {
    uint64_t arena_bytes;    /* output arena (0: no arena; jobs must bring out_dev)  */
    uint32_t max_inflight;   /* admitted jobs not yet completed (default 4096)       */
    uint32_t lanes;          /* streams, i.e. groups on the device at once (default 4) */
    uint32_t max_group;      /* jobs per group (default 4096)                        */
    uint32_t reserved;
    uint64_t lane_bytes;     /* device workspace per lane (default 256 MiB)          */
} rs_server_config;

typedef struct {
    uint64_t submitted, completed, groups, launches;
    uint64_t max_group_seen, peak_inflight, peak_arena_bytes, arena_bytes_in_use;
} rs_server_stats;

/* Creates a server on the context's device.  cfg may be NULL (defaults
 * above, arena 1 GiB).  The context must outlive the server and is not
 * otherwise used while the server runs.  Errors: RS_EINVAL, RS_ENOMEM,
 * RS_ECUDA. */
int rs_server_create(rs_ctx* ctx, const rs_server_config* cfg, rs_server** server);

/* Queues a job and returns its ticket (never blocks on the device).  A job
 * with bad arguments, or one that can never be admitted (its output larger
 * than the arena, its workspace larger than a lane), completes at once with
 * RS_EINVAL or RS_ECAPACITY in its result.  Errors of the call itself:
 * RS_EINVAL (null arguments, a query without a tree). */
int rs_server_submit(rs_server* server, const rs_job* job, uint64_t* ticket);

/* Moves up to `max` completed jobs' results into results[0..*got), waiting
 * up to wait_us microseconds for the first one.  Errors: RS_EINVAL. */
int rs_server_poll(rs_server* server, rs_result* results, uint32_t max, uint32_t* got, uint32_t wait_us);

/* Returns a completed job's arena memory to the server (no-op for jobs
 * with their own out_dev).  Errors: RS_EINVAL (unknown or unfinished
 * ticket). */
int rs_server_release(rs_server* server, uint64_t ticket);

/* Counters since creation.  Errors: RS_EINVAL. */
int rs_server_stats_get(rs_server* server, rs_server_stats* stats);

/* Testing knob: the next `count` groups the server plans fail as if the host
 * memory of their plan could not be allocated.  Their jobs finish with
 * RS_ENOMEM (their arena memory stays reserved until released, like any
 * finished job's); the server goes on with the jobs after them.
 * Errors: RS_EINVAL (null server). */
int rs_server_fail_next_plans(rs_server* server, uint32_t count);

/* Stops the worker (jobs still queued are dropped), waits for the device,
 * frees everything. */
int rs_server_destroy(rs_server* server);

/* Waits for `stream`, then returns and clears the context's device status
 * word (RS_OK, or the first device-side error since the last rs_sync). */
int rs_sync(rs_ctx* ctx, void* stream);

/* Static description of a return code.  Never NULL. */
const char* rs_strerror(int code);

/* Testing knob: leaves whose selection exceeds `cap` values take the
 * general (global-memory) path instead of the shared-memory one.  The output
 * does not change.  cap = 0 restores the default.  Errors: RS_EINVAL. */
int rs_set_leaf_capacity(rs_ctx* ctx, uint32_t cap);

/* Testing knob: on != 0 makes the split tree evaluate every ratio-of-uniforms
 * acceptance test 2 ln U <= T (Sec. 3.1, Sec. 4.6), and Bernoulli sampling
 * and Algorithm B leaves every geometric skip floor(ln U / ln(1 - p)) (Sec. 2
 * Algorithm B, Sec. 4.7), in FP64 as the definition states.  By default an
 * evaluation in single precision (and, for the skips, a fixed-point
 * logarithm) with a proven error bound decides the cases further from the
 * decision's boundary than the bound, and only the others are evaluated in
 * FP64; every outcome, and so the output, is the same either way.  Applies
 * to the context's later rs_sample*, rs_bernoulli* and rs_sample_b calls.
 * Errors: RS_EINVAL (null ctx). */
int rs_set_exact_deviates(rs_ctx* ctx, int on);

/* Testing knob: lowers the iteration caps of the method's loops on the
 * current device, for every context and call of the process: the
 * ratio-of-uniforms trials and the inversion restarts of one split deviate
 * (Sec. 3.1; defaults 2^20 and 64), the Philox blocks of one candidate or
 * skip stream (default 2^32: 2^34 32-bit candidates, 2^33 64-bit values),
 * and the attempts of one Algorithm B leaf (Sec. 2; default 64).  A value
 * at or above the default (UINT64_MAX, say) keeps the default; 0 allows no
 * trial, restart or attempt at all.  A loop that reaches its cap
 * ends with the device status RS_EITER (no trap; rs_sync, the batch's and
 * the server's statuses report it).  Errors: RS_ECUDA. */
int rs_set_iteration_caps(uint64_t rou_trials, uint64_t inv_restarts, uint64_t stream_blocks, uint64_t b_attempts);

/* Phase timing (tracing): while on, every sampling call records CUDA events
 * on its stream around its split-tree phase and its leaf phase (no host
 * synchronization).  Turning it on clears the totals.  rs_phase_totals waits
 * for the recorded calls and returns the summed durations in milliseconds
 * and the number of calls.  Errors: RS_EINVAL, RS_ECUDA, RS_ENOMEM. */
int rs_set_profiling(rs_ctx* ctx, int on);
int rs_phase_totals(rs_ctx* ctx, double* tree_ms, double* leaf_ms, uint64_t* calls);

/* Pipelining of deep split trees (depth >= log2_parts + 9): the subtrees
 * under level log2_parts are built one after another on a second,
 * highest-priority stream of the context, and the leaves of each run on the
 * caller's stream as soon as its subtree is done, beside the FP64 work of
 * the next subtrees, with at most leaf_blocks_per_sm leaf blocks per SM
 * (0 = as many as fit) so that tree blocks can run beside them.  The
 * output does not change.  log2_parts = 0 turns it off (the default: on
 * GB300 the leaves keep the issue slots busy and the tree blocks beside them
 * slow down more than the overlap gains).
 * Errors: RS_EINVAL (log2_parts outside 0..6, negative blocks). */
int rs_set_pipeline(rs_ctx* ctx, int log2_parts, int leaf_blocks_per_sm);

/* Bernoulli sampling by its size (Sec. 4.7, relation to Bernoulli sampling:
 * the number of chosen positions follows BIN(N, p); drawing it first and
 * then that many positions without replacement needs no logarithm per
 * position, which suits a GPU whose FP64 rate is low).  The size is the
 * binomial deviate of stream (SPLIT, 0) with p taken as K / 2^62,
 * K = floor(q 2^62 + 1/2), q = p for p <= 1/2 (else the size is N - BIN(N,
 * K'/2^62) with q = 1 - p); the positions are the rs_sample sample of that
 * size (kind H, the same seed, n0).  A different sample from rs_bernoulli's
 * (the same distribution).
 *
 * rs_bernoulli_size: the size to *count_out (host memory); synchronizes
 * `stream`.  Errors: RS_EINVAL (p outside [0, 1], N > 2^62), RS_ECUDA,
 * RS_EITER.
 *
 * rs_bernoulli_by_size: the 1-based positions in the window [a, b) of
 * 0-based positions (any ends), increasing, to out_dev[0..count); the window's
 * count to *count_out and the whole size to *total_out (host memory).  The
 * whole range (a = 0, b = N) runs rs_sample asynchronously on `stream` after
 * the size is read; other windows build the split tree and run a range query
 * (rs_tree_create / rs_tree_query, synchronous).  Errors: as rs_sample and
 * rs_tree_query, RS_EINVAL (bad window, n0 = 0), RS_ECAPACITY (count > cap;
 * the counts are still set). */
int rs_bernoulli_size(rs_ctx* ctx, double p, uint64_t N, uint64_t seed, uint64_t* count_out, void* stream);
int rs_bernoulli_by_size(rs_ctx* ctx, double p, uint64_t N, uint64_t seed, uint32_t n0, uint64_t a, uint64_t b,
                         uint64_t* out_dev, uint64_t cap, uint64_t* count_out, uint64_t* total_out, void* stream);

/* Largest staging area (bytes) rs_bernoulli may keep, and its slots per
 * chunk (0: mu + 8 sqrt(mu) + 64 for a chunk's expected count mu).  With
 * staging each chunk is walked once and its positions staged (about 1.1
 * times the output), then copied into place after the scan of the counts; a
 * chunk with more positions than slots is walked again for the copy.
 * Without (limit 0, an area above the limit, or an allocation that fails)
 * each chunk is walked twice, once to count and once to write.  The output
 * does not change.  Defaults: 16 GiB, 0.  Errors: RS_EINVAL. */
int rs_set_bernoulli_staging(rs_ctx* ctx, uint64_t max_bytes, uint64_t slots_per_chunk);

/* Number of kernels this context has launched since it was created. */
int rs_launch_count(rs_ctx* ctx, uint64_t* count);

/* rs_sample for callers that cannot allocate device memory while they run
 * (an allocator that owns the whole device, a host application that forbids
 * cudaMalloc after start-up, a loop that cannot take the device-wide stall of
 * cudaMalloc/cudaFree).  The paper has no counterpart: this is an interface
 * choice of this library.  It needs no context and allocates nothing: all
 * scratch memory is one static device array of about 6.6 MB that every GPU
 * using the library holds until the process exits.  Output is identical to
 * rs_sample with the same arguments.
 *  - Limits: split-tree depth <= 16 (n <= n0 * 2^16), else RS_ECAPACITY
 *    before any work; a leaf selecting more than 2^16 values ends with the
 *    device status RS_ECAPACITY.
 *  - Runs on the current CUDA device and `stream`, waits for `stream`, and
 *    returns the call's device status (RS_OK, RS_EITER, RS_ECAPACITY).
 *  - The first call on a device looks up the array's device address and
 *    builds its ln x! table: make that first call before any stream capture.
 *    Both are kept for the life of the process, so the entry point must not
 *    be called again after a cudaDeviceReset of that device.
 *  - Every call shares the array: calls that overlap on the GPU race. */
int rs_sample_static(uint64_t n, uint64_t N, uint64_t seed, uint32_t n0, uint64_t* out_dev, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RS_H */
