/*
 * bipart.h -- C ABI of the GB300 implementation of BiPart's deterministic multilevel hypergraph
 * bisection (Maleki, Agarwal, Burtscher, Pingali, PPoPP'21).
 *
 * Conventions for every entry point:
 *   - Hypergraphs are given as hyperedge -> pin CSR in int32: hedge_offsets[num_hedges + 1]
 *     (offsets[0] = 0, non-decreasing, offsets[E] = P) and hedge_pins[P] with every pin in
 *     [0, num_nodes).  Node weights and hyperedge weights are int32 >= 1; NULL means unit weights.
 *     The sum of node weights and the sum of hyperedge weights must each stay below 2^31.
 *   - "Host" pointers are ordinary CPU memory; "device" pointers are CUDA global memory of the
 *     current device.  The caller owns every array it passes and every output buffer; the
 *     library copies what it keeps.
 *   - Return codes: 0 = BIPART_OK, > 0 = warning (the result is valid), < 0 = error (outputs are
 *     unspecified).  bipart_last_error() describes the last error of the calling thread.
 *   - A handle is not thread-safe; distinct handles are independent.  All GPU work of a handle
 *     runs on its stream (bipart_set_stream); entry points that return host data synchronise it.
 *   - The result of every call is a deterministic function of its inputs: the same hypergraph and
 *     parameters always give the same partition, the same cut and the same coarse levels.
 */
#ifndef BIPART_H
#define BIPART_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BIPART_OK 0
#define BIPART_WARN_IMBALANCED 1      /* rebalancing could not reach the limit; result still valid */
#define BIPART_ERR_INVALID_ARG (-1)   /* bad k, epsilon, policy, levels, iters, level index, NULL */
#define BIPART_ERR_INVALID_CSR (-2)   /* malformed offsets, pin out of range, weight < 1, sums >= 2^31 */
#define BIPART_ERR_OOM (-3)           /* device allocation failed or a size limit was exceeded */
#define BIPART_ERR_CUDA (-4)          /* a CUDA runtime call failed (including: no usable GPU) */
#define BIPART_ERR_TIMEOUT (-5)       /* a bounded device-side wait expired */

/* Matching policies of Table 1 (Sec. 3.1.1): which hyperedges nodes prefer to merge along. */
#define BIPART_POLICY_LDH 0   /* lower degree first (the paper's default) */
#define BIPART_POLICY_HDH 1   /* higher degree first */
#define BIPART_POLICY_LWD 2   /* lower hyperedge weight first */
#define BIPART_POLICY_HWD 3   /* higher hyperedge weight first */
#define BIPART_POLICY_RAND 4  /* deterministic hash of the hyperedge id */

typedef struct bipart_graph *bipart_handle;

/* Optional device allocator used for every device buffer the library owns (for example the
 * caching allocator of a framework).  alloc returns NULL on failure; both receive the handle's
 * stream.  With no allocator set the library uses cudaMallocAsync / cudaFreeAsync on that stream.
 * Applies to allocations made after the call; pass NULLs to restore the default.  A buffer is
 * always freed by the allocator that made it.  The batch call, the server and nested k-way
 * allocate from several host threads at once: the functions must be thread-safe, and an
 * allocator that serialises its callers (a callback into an interpreter lock) serialises them. */
typedef void *(*bipart_alloc_fn)(void *ctx, size_t bytes, void *stream);
typedef void (*bipart_free_fn)(void *ctx, void *ptr, size_t bytes, void *stream);
int bipart_set_allocator(bipart_alloc_fn alloc, bipart_free_fn free_fn, void *ctx);

/* Creates a handle from host CSR arrays (Sec. 1.1 problem statement: nodes, hyperedges, optional
 * weights).  The arrays are copied to the device on `stream` (a cudaStream_t, NULL = the legacy
 * default stream; hedge_pins is read up to hedge_offsets[num_hedges] entries) and checked there by
 * a kernel whose loops are bounded by the sizes; no other kernel reads them before that check has
 * passed.  When it fails, or when no device work is possible, the CSR is validated on the host,
 * whose INVALID_CSR error (naming the first offending offset or pin, as a sequential pass would)
 * outranks any device error.  Then builds level 0 on the device: each hyperedge's pins sorted and
 * de-duplicated, hyperedges with fewer than 2 distinct pins dropped (they can never be cut), and
 * the node -> hyperedge incidence.  Errors: INVALID_ARG (NULL out, negative sizes),
 * INVALID_CSR, OOM, CUDA. */
int bipart_create(int32_t num_nodes, int32_t num_hedges, const int32_t *hedge_offsets,
                  const int32_t *hedge_pins, const int32_t *node_weights,
                  const int32_t *hedge_weights, void *stream, bipart_handle *out);

/* Same as bipart_create with the four arrays in device memory; validation runs on the device. */
int bipart_create_device(int32_t num_nodes, int32_t num_hedges, const int32_t *hedge_offsets,
                         const int32_t *hedge_pins, const int32_t *node_weights,
                         const int32_t *hedge_weights, void *stream, bipart_handle *out);

/* Changes the stream of a handle (a cudaStream_t; NULL = legacy default stream). */
int bipart_set_stream(bipart_handle h, void *stream);

/* Partitions the handle's hypergraph into k parts (Sec. 3; k-way by the nested recursive
 * bisection of Algorithm 6), writing part ids in [0, k) to out_parts[num_nodes] (HOST memory).
 *   k        number of parts, >= 1 (k = 1 gives all zeros).  A (sub)graph owning m parts is
 *            bisected with ceil(m/2) of them on side 0; for k a power of two every split is
 *            in halves, as in Algorithm 6 (other k: readings G1-G2, the paper is silent)
 *   epsilon  imbalance, 0 <= epsilon <= 1000: a side meant for ms of the m parts of a
 *            bisection of total node weight W stays at or below
 *            max(ceil(W ms / m), floor(W ms (1 + epsilon) / m)) (ms / m = 1/2 when halving)
 *   policy   BIPART_POLICY_* (Table 1)
 *   levels   maximum number of coarsening levels, >= 0 (the paper's default is 25, Sec. 3.4)
 *   refine_iters  refinement iterations per level, >= 0 (default 2, Sec. 3.4)
 * Returns OK, WARN_IMBALANCED, or an error. */
int bipart_partition(bipart_handle h, int32_t k, double epsilon, int32_t policy, int32_t levels,
                     int32_t refine_iters, int32_t *out_parts);

/* Same as bipart_partition with out_parts in DEVICE memory. */
int bipart_partition_device(bipart_handle h, int32_t k, double epsilon, int32_t policy,
                            int32_t levels, int32_t refine_iters, int32_t *d_out_parts);

/* Flags of bipart_params.  ADAPTIVE_EPS: every bisection of a k-way partition uses the largest
 * imbalance e' (in millionths) with (1 + e')^L <= 1 + epsilon, L = ceil(log2 k), so that the
 * nested allowances multiply to at most 1 + epsilon (reading G3; no effect for k <= 2). */
#define BIPART_FLAG_ADAPTIVE_EPS 1
/* MERGE_PARALLEL: when a level is contracted (Algorithm 2), coarse hyperedges with the same
 * sorted pin list are merged into the one with the smallest id, which carries the sum of their
 * weights (reading M1; the paper never merges, so this is off by default).  Every cut is
 * unchanged; coarse hyperedge weights then differ from 1, which gives the weight-based matching
 * policies (LWD, HWD, Table 1) something to order by.  The input level is not merged. */
#define BIPART_FLAG_MERGE_PARALLEL 2

/* Diagnostics: *active = 1 when the top-level bisection of the last partition call replayed a
 * captured CUDA graph (a handle captures one on the second call with the same parameters, or
 * on the third when its first call handed the coarse levels to the cluster tail), 0
 * when it ran eagerly. */
int bipart_plan_active(bipart_handle h, int32_t *active);

/* Levels of the hierarchy kept from the last k = 2 call (level 0 = the normalised input). */
int bipart_num_levels(bipart_handle h, int32_t *num_levels);

/* Copies level `level` of the kept hierarchy to host buffers (any buffer may be NULL):
 * sizes (N, E, P), hoff[E+1], pins[P] (ascending within each hyperedge), node weights[N],
 * hyperedge weights[E], cmap[N] (node -> node of level+1; -1 on the coarsest level) and the
 * matching of Algorithm 1 (hyperedge chosen by each node, -1 if none; -1 on the coarsest level). */
int bipart_get_level(bipart_handle h, int32_t level, int32_t *N, int32_t *E, int32_t *P,
                     int32_t *hoff, int32_t *pins, int32_t *node_weights,
                     int32_t *hedge_weights, int32_t *cmap, int32_t *match);

/* Cut of a partition given on the host (Sec. 1.1): sum over input hyperedges of
 * w_e * (lambda_e - 1), lambda_e = number of distinct parts among the pins of e.  Computed on
 * the device over the normalised level 0 (dropped hyperedges never contribute). */
int bipart_cut(bipart_handle h, const int32_t *parts, int64_t *cut);

/* Number of nodes / hyperedges / pins of the normalised level 0. */
int bipart_sizes(bipart_handle h, int32_t *N, int32_t *E, int32_t *P);

/* Waits for the handle's work on its stream, then releases every device buffer of the handle.
 * When all of them came from the library's own allocator, the release runs on a background
 * thread of the library (on a stream of its own, so the caller may destroy its stream at once)
 * and the memory returns to the library's pool shortly after the call returns; with an
 * allocator hook (bipart_set_allocator) the hook's free is called here.  NULL is ignored. */
void bipart_destroy(bipart_handle h);

/* Text of the last error on the calling thread ("" if none). */
const char *bipart_last_error(void);

/* Sec. 3.4 without the coarsening: re-runs the initial bisection (Algorithm 3) of the coarsest
 * level and the refinement and rebalancing (Algorithms 4-5) back to level 0 on the hierarchy the
 * handle's last partition built, with a new imbalance `epsilon` and `refine_iters` iterations;
 * the policy, levels and flags stay those of that call.  Requires that the last partition of the
 * handle had k = 2 (else BIPART_ERR_INVALID_ARG).  Coarsening depends on neither parameter, so
 * the result equals bipart_partition with the same k = 2, policy, levels and the new epsilon and
 * refine_iters.  out_parts: HOST, num_nodes entries.  Runs eagerly (no launch plan); the kept
 * hierarchy stays valid.  Used by design-space sweeps over refinement settings (Sec. 4.3). */
int bipart_refine_kept(bipart_handle h, double epsilon, int32_t refine_iters, int32_t *out_parts);

/* ---- Many independent hypergraphs on one GPU -------------------------------------------- */
/* One hypergraph in HOST memory (same conventions as bipart_create); the caller keeps the arrays
 * alive until the call that uses them has returned (batch) or been waited for (server). */
typedef struct {
    int32_t num_nodes, num_hedges;
    const int32_t *hedge_offsets, *hedge_pins, *node_weights, *hedge_weights;
} bipart_instance;

/* Parameters of one partition request (as in bipart_partition), plus BIPART_FLAG_* bits in
 * `flags` (unknown bits are rejected with INVALID_ARG). */
typedef struct {
    int32_t k;
    double epsilon;
    int32_t policy, levels, refine_iters;
    int32_t flags;
} bipart_params;

/* bipart_partition / bipart_partition_device with the parameters (and flags) in a struct. */
int bipart_partition_ex(bipart_handle h, const bipart_params *params, int32_t *out_parts);
int bipart_partition_device_ex(bipart_handle h, const bipart_params *params, int32_t *d_out_parts);

/* Partitions n independent hypergraphs concurrently on the current GPU (each as bipart_partition
 * would, Sec. 3 / Algorithm 6).  Instances of up to 2^18 nodes and 2^24 pins with k <= 1024 and
 * levels < 64 (no BIPART_FLAG_MERGE_PARALLEL) run in persistent launches, one thread block per
 * instance doing its whole partition, nested k-way included; they are grouped in size buckets by
 * pin count, each bucket launched with the block shape recorded for it by
 * bipart_batch_tune (or a default), all buckets in one CUDA graph that is replayed while the
 * batch keeps the same shape.  The other instances (and any whose level store outgrows its
 * block's arena) go to `workers` host threads (<= 0: min(16, n)), each owning a private workspace
 * and CUDA stream, largest first.  out_parts[i] (HOST, num_nodes entries) receives instance i's
 * parts, statuses[i] (may be NULL) its return code.  The result of every instance equals what
 * bipart_partition returns for it alone.  Staging buffers (pinned host and device), arenas, the
 * graph and the worker pool (whose workspaces keep their launch plans; a request goes preferably
 * to the worker that last ran one of the same sizes and parameters) are kept between calls;
 * bipart_batch_release frees them.  Each instance's sizes, pointers, hedge_offsets[0],
 * hedge_offsets[E] and parameters are checked on the host first; its CSR content is checked where it
 * is read: by its block, before the block reads the arrays through an index, or by its worker's
 * creation step.  A malformed instance gets INVALID_CSR with the host pass's message (the first
 * offending offset or pin) and leaves its out_parts untouched.  Returns OK when no instance
 * failed, else the first failing instance's error (see bipart_last_error). */
int bipart_partition_batch(int32_t n, const bipart_instance *instances, const bipart_params *params,
                           int32_t *const *out_parts, int32_t *statuses, int32_t workers);

/* Tunes the persistent batch launches on this batch: every candidate block shape (threads x
 * blocks per SM: 256x1, 256x2, 256x4, 512x1, 512x2, 1024x1) runs each size bucket's instances
 * alone (bucket
 * edges at 16Ki, 128Ki and 1Mi pins), timed by CUDA events (best of two), and the fastest is kept
 * for the bucket, in this process and in a JSON file keyed by the device name and SM count
 * ($BIPART_TUNE_CACHE, else $XDG_CACHE_HOME/bipart/batch_tune.json, else
 * $HOME/.cache/bipart/batch_tune.json; a file that cannot be written is skipped).  Only the
 * instances the persistent path takes are timed; results are discarded.  chosen (may be NULL;
 * 8 entries) receives per bucket its threads and blocks per SM, 0 0 for a bucket with no
 * instance.  Returns OK or the first error of the host checks (sizes, pointers, offsets[0] and
 * offsets[E], parameters); an instance whose CSR content is malformed is skipped by its block and
 * not timed. */
int bipart_batch_tune(int32_t n, const bipart_instance *instances, const bipart_params *params,
                      int32_t *chosen);

/* Frees the staging buffers, arenas, graph and worker pool the batch call keeps between calls,
 * then returns the unused memory of the library's device memory pool (where buffers freed by the
 * library stay reserved for its next allocations) to the driver. */
void bipart_batch_release(void);

/* Serving: a pool of `workers` threads (<= 0: 8) that partitions requests as they arrive, each
 * request's k-way subgraphs one after another on its worker's stream.  A request is admitted once
 * its estimated device working set fits, next to the running requests, in hbm_budget_bytes
 * (0 = unlimited); requests larger than the whole budget complete at once with BIPART_ERR_OOM.
 * Under a budget a worker frees its workspace after each request, so the device memory the
 * server's workspaces hold stays within the budget (the estimate bounds what a request
 * allocates); without one, workspaces keep their memory and launch plans, and a request goes
 * preferably to the worker that last ran one of the same sizes and parameters.  Results are
 * identical to bipart_partition on the same input. */
typedef struct bipart_server_s *bipart_server;
int bipart_server_create(size_t hbm_budget_bytes, int32_t workers, bipart_server *out);
/* Queues a request; the caller keeps instance arrays and out_parts (HOST) alive until waited.  A
 * request whose sizes, pointers, hedge_offsets[0], hedge_offsets[E] or parameters fail the host
 * checks completes at once with that error; its CSR content is checked where it is read (as in
 * bipart_partition_batch), a malformed one completing with INVALID_CSR. */
int bipart_server_submit(bipart_server server, const bipart_instance *instance,
                         const bipart_params *params, int32_t *out_parts, int64_t *ticket);
/* Waits for a request (timeout_ms < 0: forever; BIPART_ERR_TIMEOUT when it expires, the request
 * stays queued).  *status = the request's return code; queue_ms / run_ms = time from submit to
 * start and from start to completion (any may be NULL).  Each ticket can be waited for once. */
int bipart_server_wait(bipart_server server, int64_t ticket, int32_t timeout_ms, int32_t *status,
                       double *queue_ms, double *run_ms);
/* Micro-batches: once at least 8 waiting requests fit the persistent block path (see
 * bipart_partition_batch) and are small (pins x ceil(log2 k) <= 262,144: a batch completes as a
 * whole, so its longest member sets every member's latency), a free worker takes up to 1024 of
 * them, in queue order, as one batch (when its device memory fits the budget next to the running
 * requests); one batch runs at a time.  *batches / *batched_requests (may be NULL) = how many batches ran and the requests they
 * held so far. */
int bipart_server_stats(bipart_server server, int64_t *batches, int64_t *batched_requests);
/* Finishes all queued requests, then stops the workers. */
void bipart_server_destroy(bipart_server server);

/* Cut of a k-way partition computed without allocating any device memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot call cudaMalloc when they need
 * the cut -- a host application that gives all of HBM to its own memory pool up front (so an
 * allocation by a library fails or breaks the pool's accounting), or a latency-critical loop that
 * cannot afford the synchronisation an allocation may imply.
 *   All arrays are DEVICE memory owned by the caller: a valid hyperedge -> pin CSR
 *   (d_hedge_offsets[num_hedges + 1], d_hedge_pins), optional d_hedge_weights (NULL = unit;
 *   each weight >= 1, as bipart_create requires), d_parts[num_nodes] with values in [0, k), and
 *   the output d_cut (one int64).  Duplicate pins and single-pin hyperedges are allowed (they do
 *   not change the cut).
 *   Result: *d_cut = sum over hyperedges of w_e * (lambda_e - 1), written asynchronously on
 *   `stream`; -1 if a pin, a part or a hyperedge weight is out of range.
 *   Limits: num_hedges <= 4,194,304 and 1 <= k <= 64, else BIPART_ERR_INVALID_ARG before any GPU
 *   work.  Scratch is a fixed 16 MiB array inside the library's device image on every GPU that
 *   loads it (kept until exit).  The first call on each device looks up that array's address
 *   (make it before any stream capture).  All calls share the array: calls that overlap on the GPU
 *   race and must be serialised by the caller. */
int bipart_cut_noalloc(int32_t num_nodes, int32_t num_hedges, const int32_t *d_hedge_offsets,
                       const int32_t *d_hedge_pins, const int32_t *d_hedge_weights,
                       const int32_t *d_parts, int32_t k, int64_t *d_cut, void *stream);

/* ---- Diagnostics (not part of the paper's method) ---------------------------------------- */
/* Running total of kernels this library has launched in the process (all handles). */
int64_t bipart_kernel_launches(void);

/* Per-kernel timing: while enabled, the library brackets the launches of its main kernels with
 * CUDA events on the launching stream and accumulates, per kernel name, the number of launches,
 * their summed device time and their summed algorithmic bytes (the bytes the algorithm must move:
 * each array streamed once, gathers at element size).  on = 2 keeps the totals per kernel and
 * level instead ("name@cL" for the coarsening of level L, "name@rL" for the initial partition and
 * refinement at level L).  Enabling or disabling resets the totals. */
int bipart_profile_enable(int on);

/* Restricts per-kernel timing to the kernel named `kernel_name` (NULL or "" = all kernels), so
 * that timing one kernel perturbs the rest as little as possible.  Resets the totals. */
int bipart_profile_select(const char *kernel_name);

/* Reads entry `idx` of the per-kernel totals (finishes pending timing first).  Returns the number
 * of entries, or INVALID_ARG for an index out of range (idx = -1 only returns the count).
 * `name` receives at most name_len bytes including the terminating zero. */
int bipart_profile_read(int32_t idx, char *name, size_t name_len, int64_t *launches,
                        double *total_ms, double *total_bytes);

#ifdef __cplusplus
}
#endif
#endif /* BIPART_H */
