// Host-side structures of the sm_103a path: device buffers, the per-level store and the
// per-handle workspace.  Shared by the .cu translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <condition_variable>
#include <functional>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "bipart.h"
#include "common.cuh"

namespace bp {

// ---------------------------------------------------------------------------------- memory
// How a buffer was allocated: the free function and context in force at that time (null: the
// library's own cudaMallocAsync), so that a buffer is always returned to the allocator that
// made it, whatever bipart_set_allocator was called with in between.
struct AllocTag {
    bipart_free_fn free_fn = nullptr;
    void *ctx = nullptr;
};
void *dev_alloc(size_t bytes, cudaStream_t s, AllocTag *tag);
cudaMemPool_t lib_pool();  // the library's own memory pool on the current device (or null)
bool release_later(bipart_graph *g);  // hands a finished handle to the background releaser
void lib_pool_trim();      // returns the pool's unused memory to the driver
void dev_free(void *p, size_t bytes, cudaStream_t s, const AllocTag &tag);
void zero_fill(void *p, size_t bytes, cudaStream_t s);
uint32_t *pinned_take();            // a pinned 4 KB host block (pooled)
void pinned_release(uint32_t *p);
// Bumped whenever a buffer is (re)allocated: a captured graph is only valid while the buffers
// it points to are the ones it was captured with.
void note_realloc();

// A growable device buffer (capacity only grows; contents are not preserved on growth).
struct Buf {
    void *p = nullptr;
    size_t cap = 0;
    cudaStream_t s = nullptr;
    AllocTag tag;
    Buf() = default;
    Buf(const Buf &) = delete;
    Buf &operator=(const Buf &) = delete;
    ~Buf() { release(); }
    void release() {
        if (p) dev_free(p, cap, s, tag);
        p = nullptr;
        cap = 0;
    }
    void *ensure(size_t bytes, cudaStream_t stream) {
        if (bytes == 0) bytes = 16;
        if (bytes > cap) {
            release();
            s = stream;
            size_t c = bytes + bytes / 8 + 256;
            p = dev_alloc(c, stream, &tag);
            if (!p) throw Fail{BIPART_ERR_OOM, "device allocation of " + std::to_string(c) + " bytes failed"};
            cap = c;
            note_realloc();
        }
        return p;
    }
    // As ensure(), and a new allocation is zero-filled (for state that its users leave zero).
    void *ensure_zero(size_t bytes, cudaStream_t stream) {
        const void *old = p;
        void *q = ensure(bytes, stream);
        if (q != old) zero_fill(q, cap, stream);
        return q;
    }
    template <class T>
    T *as() const { return reinterpret_cast<T *>(p); }
};

// Tile states of the decoupled look-back scans issued on one stream, in two halves used in turn:
// a multi-tile scan runs on the clean half and clears the tile states that the previous
// multi-tile scan left in the other half, so no scan needs its last block to clean up after it.
// Each half's tile counter returns to zero by itself (a wrapping increment per tile).
struct ScanState {
    Buf buf;
    size_t half_words = 0;        // 64-bit words per half: [tile counter, unused, tile states...]
    int clean = 0;                // the half the next multi-tile scan runs on
    int64_t dirty[2] = {0, 0};    // tile states left set in each half
    // Both halves, for a scan of `tiles` tiles (a new, zeroed allocation when too small).
    unsigned long long *halves(int64_t tiles, cudaStream_t stream) {
        const size_t need = 2 + (size_t)tiles;
        if (need > half_words) {
            buf.ensure(16 * need, stream);  // more than the capacity: always a new allocation
            zero_fill(buf.p, buf.cap, stream);
            half_words = buf.cap / 16;
            clean = 0;
            dirty[0] = dirty[1] = 0;
        }
        return buf.as<unsigned long long>();
    }
    // Zeroes both halves (the start of a bisection, in case an earlier run stopped midway).
    void reset(cudaStream_t stream) {
        if (buf.p) BP_CUDA(cudaMemsetAsync(buf.p, 0, buf.cap, stream));
        clean = 0;
        dirty[0] = dirty[1] = 0;
    }
};

// One level of the multilevel hierarchy, resident in HBM.
//   hoff[E+1], pins[P]   hyperedge -> pins CSR, pins ascending within a hyperedge
//   hw[E]                hyperedge weights (nullptr: all 1)
//   nw[N]                node weights
//   noff[N+1], nadj[P]   node -> hyperedges CSR (order within a node unspecified)
//   cmap[N], match[N]    node -> node of the next level; Algorithm 1 matching (when coarser
//                        levels exist)
struct Level {
    int32_t N = 0, E = 0, P = 0;
    bool unit_hw = true;
    Buf b_hoff, b_pins, b_hw, b_nw, b_noff, b_nadj, b_cmap, b_match;
    Buf b_tsh, b_tsn;  // tile-start tables of the hyperedge and incidence CSRs
    // A level built by the cluster tail (tail.cu) is a view into the tail's arena: hoff, pins,
    // hw, nw, cmap, match (it has no incidence CSR and no tile-start tables).
    int32_t *view[6] = {};
    int32_t *tsh() const { return b_tsh.as<int32_t>(); }
    int32_t *tsn() const { return b_tsn.as<int32_t>(); }
    int32_t *hoff() const { return view[0] ? view[0] : b_hoff.as<int32_t>(); }
    int32_t *pins() const { return view[0] ? view[1] : b_pins.as<int32_t>(); }
    int32_t *hw() const { return unit_hw ? nullptr : (view[0] ? view[2] : b_hw.as<int32_t>()); }
    int32_t *nw() const { return view[0] ? view[3] : b_nw.as<int32_t>(); }
    int32_t *noff() const { return b_noff.as<int32_t>(); }
    int32_t *nadj() const { return b_nadj.as<int32_t>(); }
    int32_t *cmap() const { return view[0] ? view[4] : b_cmap.as<int32_t>(); }
    int32_t *match() const { return view[0] ? view[5] : b_match.as<int32_t>(); }
    bool is_view() const { return view[0] != nullptr; }
    void set_view(int32_t n, int32_t e, int32_t p, int32_t *hoff_, int32_t *pins_, int32_t *hw_,
                  int32_t *nw_, int32_t *cmap_, int32_t *match_) {
        N = n; E = e; P = p; unit_hw = hw_ == nullptr;
        view[0] = hoff_; view[1] = pins_; view[2] = hw_; view[3] = nw_; view[4] = cmap_; view[5] = match_;
    }
    void clear_view() {
        for (auto &v : view) v = nullptr;
    }
    void reserve(int32_t n, int32_t e, int32_t p, bool unit, cudaStream_t s) {
        clear_view();
        N = n; E = e; P = p; unit_hw = unit;
        b_hoff.ensure(sizeof(int32_t) * ((size_t)e + 1), s);
        b_pins.ensure(sizeof(int32_t) * (size_t)p, s);
        if (!unit) b_hw.ensure(sizeof(int32_t) * (size_t)e, s);
        b_nw.ensure(sizeof(int32_t) * (size_t)n, s);
        b_noff.ensure(sizeof(int32_t) * ((size_t)n + 1), s);
        b_nadj.ensure(sizeof(int32_t) * (size_t)p, s);
        b_cmap.ensure(sizeof(int32_t) * (size_t)n, s);
        b_match.ensure(sizeof(int32_t) * (size_t)n, s);
    }
};

// Scratch shared by all levels of one bisection, sized by the largest level seen.
struct Work {
    ScanState scan;  // decoupled look-back tile states
    Buf status;      // device error word (DevErr bits)
    Buf small;       // small device scalars (counters, totals, selection state)
    Buf e_a, e_b, e_c, e_d;  // per-hyperedge int32 scratch
    Buf e_key;       // per-hyperedge uint64 keys
    Buf n_a, n_b, n_c;       // per-node int32 scratch
    Buf n_key;       // per-node uint64 keys
    Buf p_a;         // per-pin int32 scratch
    Buf side_a, side_b;      // uint8 sides (ping-pong across levels)
    Buf gain;        // int32 gains
    Buf hc;          // int2 per-hyperedge gain contributions
    Buf n1;          // int32 per-hyperedge side-1 pin counts: two halves used by alternate passes
    int64_t n1_half = 0;
    int64_t gain_pass = 0;   // gain passes so far in this bisection
    int32_t n1_prev_E = 0;   // hyperedges counted by the previous pass (its half is dirty there)
    const void *n1_level = nullptr;  // the level whose counts the current half holds (else null)
    Buf moved;       // nodes moved since the counts were last brought up to date (int32)
    Buf e_best;      // per-hyperedge uint64 singleton-attach keys
    Buf m_fp, m_tkey, m_tmin, m_rep, m_wsum;  // parallel-net merging: fingerprints, table, groups
    Buf partial;     // per-block partial sums of grid-wide reductions
    Buf list;        // node list (rebalance candidates)
    Buf pinned;      // host-pinned mirror of `small`
    uint32_t *host_small = nullptr;
    // the cluster tail (tail.cu): arena of its coarse levels and its scratch
    Buf t_arena, t_e0, t_e1, t_e2, t_e3, t_e4, t_p, t_n, t_c, t_x, t_trace;
};

struct Params {
    int32_t k = 2;
    double eps = 0;
    int32_t policy = 0;
    int32_t levels = 0;
    int32_t iters = 0;
    int32_t flags = 0;      // BIPART_FLAG_*
    // derived: the imbalance every bisection uses (millionths, after the adaptive rule) and the
    // share of the bisection at hand (side 0 meant for m0 of m parts)
    int64_t e6 = 0;
    int32_t m0 = 1, m = 2;
};
// Checks the user parameters and fills the derived fields for the top-level bisection.
Params make_params(int32_t k, double eps, int32_t policy, int32_t levels, int32_t iters,
                   int32_t flags);

// Result of one bisection kept for parity queries.
struct Hierarchy {
    int32_t nlev = 0;
    bool valid = false;
    int32_t tail_from = -1;  // first level the cluster tail built (-1: none)
    Params params;           // the bisection that built it
};

// How the host driver executes: eagerly (reading sizes back, optionally recording them), or
// while capturing a CUDA graph (replaying the recorded sizes, which a device check verifies).
struct Exec {
    bool capturing = false;
    bool recording = false;
    std::vector<int32_t> sizes;
    size_t pos = 0;
    std::vector<uint8_t> flags;  // recorded control decisions, in order
    size_t flag_pos = 0;
    int flag_next = 0, flag_pending = -1;
    int64_t check_kernels = 0;   // size-check kernels per replay
    std::vector<std::pair<int, int32_t>> checks;  // deferred (slot index, recorded value)
    // the last eager top-level bisection, ready to be captured
    bool rec_valid = false;
    Params rec_params;
    uint64_t rec_gen = 0;
    int rec_nlev = 0;
    int64_t rec_kernels = 0;
    bool rec_tail = false;  // the recorded run used the cluster tail (not captured: see bisect_top)
};

struct Probe {
    std::string name;
    double bytes;
    cudaEvent_t a, b;
};

// A captured bisection of level 0 for fixed parameters.
struct Plan {
    bool valid = false;
    Params params;
    int nlev = 0;
    uint64_t gen = 0;
    int prof_epoch = -1;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t launches = 0;
    std::vector<Probe> probes;
    // the stream's scan state as the captured bisection leaves it: a replay runs no host code,
    // so the host copy is set to this after every launch (later scans on the stream, such as a
    // k-way split's, must see which half is clean)
    int scan_clean = 0;
    int64_t scan_dirty[2] = {0, 0};
    void reset();
};

}  // namespace bp

namespace bp {
// A few host threads that run fn(i) for i in [0, count) and return when all are done: the
// bisections of one recursion-tree level (each on the child workspace of its subgraph), and the
// host-side staging of a batch.
struct Lanes {
    explicit Lanes(int n) {
        BP_CUDA(cudaGetDevice(&device_));
        for (int i = 0; i < n; ++i) threads_.emplace_back([this]() { loop(); });
    }
    ~Lanes() {
        {
            std::lock_guard<std::mutex> lk(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        for (auto &t : threads_) t.join();
    }
    // fn(i) for i in [0, count), spread over the threads; returns when all are done
    void run(int count, const std::function<void(int)> &fn) {
        std::unique_lock<std::mutex> lk(mu_);
        fn_ = &fn;
        count_ = count;
        next_ = 0;
        done_ = 0;
        ++epoch_;
        cv_.notify_all();
        done_cv_.wait(lk, [&]() { return done_ == count_; });
        fn_ = nullptr;
    }

   private:
    void loop() {
        cudaSetDevice(device_);
        uint64_t seen = 0;
        std::unique_lock<std::mutex> lk(mu_);
        for (;;) {
            cv_.wait(lk, [&]() { return stop_ || (epoch_ != seen && next_ < count_); });
            if (stop_) return;
            while (next_ < count_) {
                const int i = next_++;
                const std::function<void(int)> *fn = fn_;
                lk.unlock();
                (*fn)(i);
                lk.lock();
                if (++done_ == count_) done_cv_.notify_all();
            }
            seen = epoch_;
        }
    }
    int device_ = 0;
    std::mutex mu_;
    std::condition_variable cv_, done_cv_;
    std::vector<std::thread> threads_;
    const std::function<void(int)> *fn_ = nullptr;
    int count_ = 0, next_ = 0, done_ = 0;
    uint64_t epoch_ = 0;
    bool stop_ = false;
};

// Deletes a child workspace, then its stream (the buffers are freed on that stream).
struct KidDel {
    void operator()(bipart_graph *g) const;
};
}  // namespace bp

struct bipart_graph {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool last_replayed = false;  // the last top-level bisection ran a captured plan
    cudaStream_t cap_stream = nullptr;  // private stream a plan is captured on (the legacy
                                        // default stream cannot be captured)
    bp::Level L0;                                  // normalised input
    std::vector<std::unique_ptr<bp::Level>> lev;   // coarse levels 1.. of the last bisection
    bp::Hierarchy hier;
    bp::Work w;
    // k-way: part vectors, node map of a subgraph (in a child: its own), bisection output
    bp::Buf part_a, part_b, l2g, side_out;
    bp::Buf in_hoff, in_pins, in_nw, in_hw;   // uploaded input (executor workspaces)
    int64_t total_node_weight = 0;
    bp::Exec ex;
    bp::Plan plan;
    uint64_t gen = 0;            // buffer (re)allocation count of this handle
    // k-way: one child workspace per subgraph of the recursion tree (own stream, level store and
    // launch plan), bisected concurrently by a few host threads; events order the streams
    std::vector<std::unique_ptr<bipart_graph, bp::KidDel>> kids;
    std::unique_ptr<bp::Lanes> lanes;
    cudaEvent_t kid_ready = nullptr, kid_done = nullptr;
    // in a child: the parent's parameters (k included) its subgraph and launch plan belong to; a
    // child's subgraph is the same for the same parent input and parameters, and only then may
    // its plan be replayed
    bp::Params kid_stamp;
    bool kid_stamp_valid = false;
    // host threads that bisect the subgraphs of a tree level (0: the default, 8 or
    // $BIPART_KWAY_LANES); with 1 the subgraphs are bisected one after another on this handle's
    // stream, which the children then share (workers of the batch and serving pools, whose
    // concurrency is across requests)
    int kid_lanes = 0;
    bool kid_own_stream = true;  // in a child: its stream was made for it
    // free what a request no longer needs as soon as it can (workers of a server under an HBM
    // budget): with one lane, the top bisection's coarse levels before the subgraphs'
    bool lean = false;
    bool ext_alloc = false;  // some buffer of this handle came from a bipart_set_allocator hook
    int32_t last_tail_from = -1;
    bool allow_tail = true;  // the next bisection may hand its coarse levels to the cluster tail  // tail start of the last bisection run on the host (eager or captured)
    ~bipart_graph();
};

namespace bp {

// ------------------------------------------------------------------- coarsening (coarsen.cu)
// Builds level 0 from a device CSR (already validated, P = its pin count): normalisation +
// incidence.
void build_level0(bipart_graph *g, Level &L, int32_t N, int32_t E, int32_t P, const int32_t *d_hoff,
                  const int32_t *d_pins, const int32_t *d_nw, const int32_t *d_hw);
// Algorithm 1 + 2 on `f`, producing `c` (sizes read back to the host).
// sizes: level_sizes() slots receiving {N', E', P'}.  init_done: f's key and reset pass already
// ran (with the previous level's incidence fill); more_levels: the level count allows another
// contraction after this one.  Returns whether c's own key and reset pass has been run.
// tail_new: contractions still allowed after c when the cluster tail may take over from c (-1:
// it may not).  When it does, *to_tail is set and c's node -> hyperedge incidence is not built:
// the caller must then run the tail from c (this is the one place that decides).
bool coarsen_level(bipart_graph *g, Level &f, Level &c, int policy, int32_t *sizes, bool merge,
                   bool init_done, bool more_levels, int tail_new = -1, int flags = 0,
                   bool *to_tail = nullptr);
// Node -> hyperedge incidence of a level whose hyperedge CSR is complete and whose node degrees
// were counted into degree_counters(g, N) while its pins were written.
void build_incidence(bipart_graph *g, Level &L);
int *degree_counters(bipart_graph *g, int32_t N);

// -------------------------------------------------------------------- refinement (refine.cu)
// Runs Algorithms 3, 5 (+ rebalance) over the hierarchy; writes side of level 0.  The status
// (1 = the level-0 rebalance ran out of candidates) is left in *bisect_status_word(g).
// Side 0 is meant for m0 of m parts: Algorithm 3 grows it to that share and limit[s] bounds
// side s (halving bisection: m0 / m = 1 / 2, equal limits).
// With tail_from >= 0 the levels from tail_from down were refined by the cluster tail, which left
// the side of level tail_from in the handle's first side buffer (side_a).
void uncoarsen(bipart_graph *g, std::vector<Level *> &levels, const int64_t limit[2], int m0,
               int m, int32_t iters, uint8_t *d_side0, int tail_from = -1);
const unsigned *bisect_status_word(bipart_graph *g);
// Bytes at the start of the small scratch holding counters and selection state that phases
// leave zero for the next one (cleared once at the start of every bisection).
size_t small_state_bytes();
void refine_init();  // once per process: kernel attributes (never during a capture)
void coarsen_init();  // same, for the coarsening kernels
// Weight limit of a side meant for ms of m parts of a (sub)graph of weight W, imbalance e6
// millionths: max(ceil(W ms / m), floor(W ms (10^6 + e6) / (m 10^6))) (reading C12; G2 for
// m != 2).
int64_t balance_limit(int64_t W, int32_t ms, int32_t m, int64_t e6);

// ------------------------------------------------------------------ cluster tail (tail.cu)
// Blocks per cluster of the tail kernel on this GPU (0: not available; the grid path runs every
// level).  BIPART_TAIL_NODES / BIPART_TAIL_PINS override the starting-level limits (0 disables).
int tail_cluster();
// Whether the rest of a bisection from level L (max_new more contractions allowed) can run as
// the cluster tail.
bool tail_eligible(const Level &L, int max_new, int flags);
// Runs the tail from levels.back(): appends the coarse levels it builds (arena views in g->lev),
// writes the bisection of the starting level to d_side and its rebalance status to the handle's
// refinement state.  Eager: one launch and one size read-back; while capturing: the recorded sizes.
void run_tail(bipart_graph *g, std::vector<Level *> &levels, const Params &p, const int64_t limit[2],
              uint8_t *d_side);
// Two device ints of the handle's size slots for the tail's level count and arena check.
int32_t *tail_info_slot(bipart_graph *g);
struct RState;
RState *refine_state(bipart_graph *g);

// ------------------------------------------------------------------------- diagnostics
// Brackets one kernel launch with CUDA events on `s` when profiling is on (see
// bipart_profile_enable); `bytes` is the launch's algorithmic traffic.
int prof_epoch();
void prof_collect(const std::vector<Probe> &probes);
// Tags the launches that follow with a phase ('c' coarsening, 'r' refinement, 0 none) and a level
// index; in profile mode 2 the totals are kept per kernel and tag.
void prof_level(char phase, int level);

struct ProfScope {
    int slot = -1;
    bool ended = false;
    ProfScope(const char *name, double bytes, cudaStream_t s);
    ~ProfScope() { end(); }
    // Records the end event now (right after the launch) instead of at destruction.
    void end();
    // Sets the algorithmic bytes when they are known only after the launch (its own read-back).
    void set_bytes(double bytes);
};

// ------------------------------------------------------------------------- block path (block.cu)
// One instance of a batch run by the persistent block kernel (device-side descriptor).
struct BInst {
    int N, E, P;
    int policy, levels, iters, k;
    long long e6;                        // imbalance of every bisection, millionths
    long long hoff, pins, nw, hw, out;  // offsets into the concatenated arrays (nw, hw < 0: unit)
    int status;                          // 0 ok, 1 imbalanced, 2 deferred (did not fit), 3 malformed
};
constexpr int kBlkDeferred = 2, kBlkMalformed = 3;
bool block_eligible(int64_t N, int64_t E, int64_t P, int k, int levels);
// Runs a batch with the persistent block kernels (instances in size buckets, each bucket with the
// block shape its tuning chose, all buckets in one CUDA graph); writes every instance's parts to
// outs[i] and its status to inst[i].status (2: did not fit a block's arena, the caller runs it;
// 3: its CSR failed the block's check, nothing was written, the caller reports it).
void run_block_batch(std::vector<BInst> &inst, const std::vector<const int32_t *> &hoff,
                     const std::vector<const int32_t *> &pins, const std::vector<const int32_t *> &nw,
                     const std::vector<const int32_t *> &hw, const std::vector<int32_t *> &outs);
// Times every candidate block shape on each size bucket of the batch and records the fastest
// (in this process and in the JSON tuning cache); chosen: 2 ints per bucket (threads, per SM).
void tune_block_batch(std::vector<BInst> &inst, const std::vector<const int32_t *> &hoff,
                      const std::vector<const int32_t *> &pins, const std::vector<const int32_t *> &nw,
                      const std::vector<const int32_t *> &hw, int32_t *chosen);
void release_block_batch();
// Device bytes the persistent path needs for these instances (nw / hw >= 0 marks weights), and
// the release of its device buffers (a server under a budget holds them only while a batch runs).
size_t block_batch_bytes(std::vector<BInst> inst);
void trim_block_batch();

// ------------------------------------------------------------------------- validation (api.cu)
void validate_params(int32_t k, double eps, int32_t policy, int32_t levels, int32_t iters);
// Returns the total node weight (N without node weights).
int64_t validate_host_csr(int32_t N, int32_t E, const int32_t *hoff, const int32_t *pins,
                          const int32_t *nw, const int32_t *hw);

// ------------------------------------------------------------------------- executor (api.cu)
bipart_graph *graph_new(cudaStream_t s);
void graph_load_host(bipart_graph *g, int32_t N, int32_t E, const int32_t *hoff,
                     const int32_t *pins, const int32_t *nw, const int32_t *hw);
int graph_partition_host(bipart_graph *g, const Params &p, int32_t *out);

// ------------------------------------------------------------------------- misc (api.cu)
uint32_t *dev_status(bipart_graph *g);
void check_status(bipart_graph *g);
void sync(bipart_graph *g);

// Scalar produced on the device that the host needs (a level size).  Eager: copied back (and
// recorded when recording).  Capturing: the recorded value is returned and a device check
// against the live value is added to the graph (a mismatch invalidates the plan): values in the
// per-level size slots are checked together by flush_checks() at the end of the capture, others
// at once.
int32_t read_i32(bipart_graph *g, const int32_t *d);
// Several such scalars with one host round trip (recorded and checked in order).
void read_i32s(bipart_graph *g, int n, const int32_t *const *d, int32_t *v);
// Reads a device flag in eager mode.
unsigned read_flag(bipart_graph *g, const unsigned *d);

// Three device ints {N', E', P'} for coarsening step `idx` of a bisection: distinct slots per
// level (so their checks can wait until the end of a captured bisection), or one shared slot past
// the slot capacity.
int32_t *level_sizes(bipart_graph *g, int idx);
// Adds the deferred size checks of a capture to the graph (one kernel).
void flush_checks(bipart_graph *g);

// Device-computed control decisions (loop continuation, the exact-select branch).  The
// computation is deterministic, so a captured bisection takes every decision the recorded eager
// run took, as straight-line kernels with no conditional node: flag_slot() gives the kernel that
// computes the next flag a slot to store it in (null outside a capture), device_flag() returns
// the flag (eager: read from the device and recorded; capturing: the recorded value) and, while
// capturing, adds the slot's check to the end-of-bisection verification.
unsigned *flag_slot(bipart_graph *g);
bool device_flag(bipart_graph *g, const unsigned *d_flag);

}  // namespace bp
