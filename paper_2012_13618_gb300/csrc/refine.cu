// Initial partitioning and refinement on sm_103a (Sec. 3.2-3.3): Algorithm 4 move gains from
// per-hyperedge side counts, Algorithm 3 growth of P0 by the top ceil(sqrt n) gains, Algorithm 5
// swaps of the gain >= 0 lists and the rebalancing pass.
//
// Node order is always (gain descending, node id ascending).  A top-K is found without sorting:
// one histogram pass over gains clamped to [-1024, 1023] fixes the threshold gain exactly unless
// it falls in one of the two clamped end buckets, in which case an exact radix select (up to
// three 11-bit passes over the order-preserving key gain ^ 0x80000000) narrows it down; the lowest
// ids among nodes whose gain equals the threshold are then taken by a scan over node ids (grid
// levels) or from a shared-memory bitmap of those nodes (one-block levels).  Only the
// rebalancing pass needs the chosen nodes in order; it sorts at most ceil(sqrt n) of them in one
// block.  The two data-dependent loops (Algorithm 3's rounds and the rebalancing rounds) are
// driven by a device-side flag; a captured bisection replays the recorded decisions as
// straight-line kernels and verifies every flag on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "lb.cuh"
#include "refine_dev.cuh"
#include "scan.cuh"

namespace bp {

namespace {

constexpr int kBlock = 256;

inline int grid_for(int64_t n, int per_block = kBlock, int cap = 152 * 16) {
    int64_t b = (n + per_block - 1) / per_block;
    if (b < 1) b = 1;
    return (int)std::min<int64_t>(b, cap);
}

// Selection passes over up to kSelOneBlock nodes run as one block of kSelOneThreads threads (the
// histogram, the threshold and the application in one launch).
constexpr int kSelOneThreads = 512;  // (512 was 9 us a bisection faster than 1024 in a same-box A/B)

// Threads of the one-block ordered rebalance move (512 was 4 us a bisection faster than 1024).
constexpr int kRebalThreads = 512;


// Blocks of a grid-wide sum (each block stores its partial; the last block adds them).
constexpr int kReduceBlocks = 608;

// Levels up to this many pins compute gains without the separate contribution pass.
constexpr int kDirectGainPins = 1'000'000;

// Levels whose nodes have at most this many incidences on average update the side-1 counts after
// a move (one warp per moved node) instead of recounting them; on coarser levels a moved node
// can carry a large share of all incidences.
constexpr int kDeltaMaxDegree = 64;

// Levels whose nodes average more incidences than this sum each warp's gain flushes per node
// before the atomic (many threads end on one node there); on the others it only costs time.
constexpr int kWarpSumDegree = 64;

}  // namespace

// Grid kernels: one launch per phase (device code in refine_dev.cuh).
// Side-1 pin counts of a level's first pass into n1, plus two clearing jobs: the other count
// buffer over the previous count's hyperedges (the two alternate from count to count), and the
// gains that the node-gain pass accumulates.
__global__ void __launch_bounds__(kLbBlock)
k_hedge_n1(int E, int P, const int *__restrict__ hoff, const int *__restrict__ pins,
           const uint8_t *__restrict__ side, int *__restrict__ n1, const int *__restrict__ ts,
           int *__restrict__ n1_prev, int E_prev, int *__restrict__ gain, int N) {
    d_hedge_n1(GridTeam(), E, P, hoff, pins, side, n1, ts);
    const int n = E_prev > N ? E_prev : N;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (i < E_prev) n1_prev[i] = 0;
        if (i < N) gain[i] = 0;
    }
}


// Gains from per-hyperedge contributions (large levels: one 8-byte gather per incidence) ...
__global__ void k_hedge_contrib(int E, const int *__restrict__ hoff, const int *__restrict__ hw,
                                int *__restrict__ n1, int2 *__restrict__ hc) {
    d_hedge_contrib(GridTeam(), E, hoff, hw, n1, hc, false);
}

__global__ void __launch_bounds__(kLbBlock)
k_node_gain(int N, int P, const int *__restrict__ noff, const int *__restrict__ nadj,
            const int2 *__restrict__ hc, const uint8_t *__restrict__ side, int *__restrict__ gain,
            const int *__restrict__ ts, bool warp_sum) {
    d_node_gain(GridTeam(), N, P, noff, nadj, hc, side, gain, ts, warp_sum);
}

// ... or formed on the spot (small levels, where the contribution pass costs more as a launch
// than its gathers save).
__global__ void __launch_bounds__(kLbBlock)
k_node_gain_direct(int N, int P, const int *__restrict__ noff, const int *__restrict__ nadj,
                   const int *__restrict__ hoff, const int *__restrict__ hw, const int *__restrict__ n1,
                   const uint8_t *__restrict__ side, int *__restrict__ gain, const int *__restrict__ ts,
                   bool warp_sum) {
    d_node_gain_direct(GridTeam(), N, P, noff, nadj, hoff, hw, n1, side, gain, ts, warp_sum);
}

// Side-1 counts brought up to date after a move instead of recounted (Algorithm 4's n1 is a
// plain count, so the result is the same): every moved node adds +1 (now on side 1) or -1 (now on
// side 0) to the count of each of its hyperedges, one warp per moved node over its incidences.
// The gains are cleared for the pass that follows.
__global__ void __launch_bounds__(kBlock)
k_n1_delta(int N, const int *__restrict__ noff, const int *__restrict__ nadj,
           const uint8_t *__restrict__ side, const int *__restrict__ moved, const RState *st,
           int *__restrict__ n1, int *__restrict__ gain) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    for (int v = tid; v < N; v += nt) gain[v] = 0;
    const int m = (int)st->moved_count;
    const int lane = threadIdx.x & 31;
    for (int k = tid >> 5; k < m; k += nt >> 5) {
        const int v = moved[k];
        const int d = side[v] ? 1 : -1;
        const int b = noff[v + 1];
        for (int j = noff[v] + lane; j < b; j += 32) atomicAdd(n1 + nadj[j], d);
    }
}

// Copies the grid's accumulated histogram into shared memory and clears it in global memory
// (the last block of a selection pass).
__device__ __forceinline__ void take_hist(RState *st, unsigned (*h)[kHistBins]) {
    unsigned *g = &st->hist[0][0];
    for (int i = threadIdx.x; i < 2 * kHistBins; i += blockDim.x) {
        (&h[0][0])[i] = __ldcg(g + i);
        g[i] = 0u;
    }
    __syncthreads();
}

// A loop condition evaluated by the last thread of the kernel that produced its inputs; in a
// captured bisection the flag is also stored in its check slot.
struct CondArgs {
    int kind;                    // COND_NONE, COND_INITIAL, COND_REBAL
    int first;                   // first evaluation of the loop (resets its counters)
    int m0, m;                   // Algorithm 3: side 0 grows to m0 / m of the weight
    long long limit0, limit1;    // rebalance: per-side limits
    long long max_rounds;
    unsigned *slot;              // flag_slot() of this evaluation (null outside a capture)
};
enum { COND_NONE = 0, COND_INITIAL = 1, COND_REBAL = 2 };

__device__ __forceinline__ void eval_cond(RState *st, const CondArgs &c, uint32_t *status) {
    if (c.kind == COND_INITIAL) d_initial_cond(st, c.max_rounds, status, c.first != 0, c.m0, c.m);
    else if (c.kind == COND_REBAL) d_rebal_cond(st, c.limit0, c.limit1, c.max_rounds, status, c.first != 0);
    else return;
    if (c.slot && threadIdx.x == 0) *c.slot = st->flag;
}

// Selection over a grid: clamped-gain histogram, then (last block) the per-group threshold; the
// rebalancing and moved lists are emptied for the application scan that follows.  st->slow is
// left for the exact passes (and stored in its check slot).
__global__ void __launch_bounds__(kBlock)
k_sel(int N, int kind, long long s, const int *__restrict__ gain, uint8_t *side,
      const int *__restrict__ nw, RState *st, unsigned *slow_slot) {
    __shared__ unsigned h[2][kHistBins];
    d_sel_hist(GridTeam(), N, kind, gain, side, nw, st, h);
    if (!last_block(&st->arrived)) return;
    take_hist(st, h);
    d_sel_find(kind, s, st, h);
    if (threadIdx.x == 0) {
        st->list_count = 0;
        st->moved_count = 0;
        if (slow_slot) *slow_slot = st->slow;
    }
}

// Selection of a level of at most kSelOneBlock nodes by one block (d_sel_small), then the loop
// condition that follows it.  Dynamic shared memory: 5 bytes per node.
__global__ void __launch_bounds__(kSelOneThreads, 1)
k_sel_small(int N, int kind, long long s, const int *__restrict__ gain, uint8_t *side,
            const int *__restrict__ nw, RState *st, uint32_t *status, int *list, int *moved,
            CondArgs cond, bool weights) {
    extern __shared__ int s_gain[];                                  // N gains
    signed char *s_grp = reinterpret_cast<signed char *>(s_gain + N);  // N groups (-1: none)
    __shared__ unsigned h[2][kHistBins];
    __shared__ unsigned long long red[33];
    d_sel_small(N, kind, s, gain, side, nw, st, status, list, moved, s_gain, s_grp, h);
    if (cond.kind == COND_NONE) return;
    // the loop condition that follows the selection, evaluated here instead of by a launch of
    // its own; with `weights` the side weights are summed afresh first (the initial partition
    // keeps them current as it moves nodes)
    __syncthreads();
    if (weights) {
        unsigned long long w0 = 0, w1 = 0;
        for (int v = threadIdx.x; v < N; v += blockDim.x) {
            const unsigned long long w = (unsigned long long)nw[v];
            if (side[v]) w1 += w;
            else w0 += w;
        }
        w0 = block_sum(w0, red);
        w1 = block_sum(w1, red);
        if (threadIdx.x == 0) {
            st->W[0] = w0;
            st->W[1] = w1;
        }
        __syncthreads();
    }
    eval_cond(st, cond, status);
}

// One digit of the exact radix select: histogram, then (last block) the narrowed range.
__global__ void __launch_bounds__(kBlock)
k_sel_exact(int N, int kind, const int *__restrict__ gain, const uint8_t *__restrict__ side,
            const int *__restrict__ nw, RState *st, uint32_t *status) {
    __shared__ unsigned h[2][kHistBins];
    const bool one = gridDim.x == 1;
    d_sel_hist_exact(GridTeam(), N, kind, gain, side, nw, st, h, !one);
    if (!one) {
        if (!last_block(&st->arrived)) return;
        take_hist(st, h);
    }
    d_sel_find_exact(st, status, h);
}

// W = side weights: one partial sum per block, added in block order by the last block, which
// then evaluates the loop condition that needs W (if any).
__global__ void __launch_bounds__(kBlock)
k_side_weights(int N, const uint8_t *__restrict__ side, const int *__restrict__ nw, RState *st,
               CondArgs cond, uint32_t *status, unsigned long long *__restrict__ partial) {
    __shared__ unsigned long long red[33];
    // per block: both sums reduced in the block and stored (no contended atomics); the last
    // block adds the partials in block order
    unsigned long long w0 = 0, w1 = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) {
        const unsigned long long w = (unsigned long long)nw[v];
        if (side[v]) w1 += w;
        else w0 += w;
    }
    w0 = block_sum(w0, red);
    w1 = block_sum(w1, red);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = w0;
        partial[2 * blockIdx.x + 1] = w1;
    }
    if (!last_block(&st->arrived)) return;
    unsigned long long s0 = 0, s1 = 0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        s0 += __ldcg(partial + 2 * b);
        s1 += __ldcg(partial + 2 * b + 1);
    }
    s0 = block_sum(s0, red);
    s1 = block_sum(s1, red);
    if (threadIdx.x == 0) {
        st->W[0] = s0;
        st->W[1] = s1;
    }
    __syncthreads();
    eval_cond(st, cond, status);
}

// Loop conditions evaluated alone (the Algorithm 3 loop body ends with one).
__global__ void k_initial_cond(RState *st, CondArgs cond, uint32_t *status) {
    eval_cond(st, cond, status);
}

// Ordered rebalance move, then (same block) the rebalance condition for the next round.
__global__ void __launch_bounds__(kRebalThreads)
k_rebal_move(const int *__restrict__ gain, uint8_t *__restrict__ side, const int *__restrict__ nw,
             const int *__restrict__ list, RState *st, long long s, CondArgs cond, uint32_t *status,
             int *__restrict__ moved) {
    extern __shared__ unsigned long long keys[];
    d_rebal_move(gain, side, nw, list, st, s, keys, moved);
    __syncthreads();
    eval_cond(st, cond, status);
}

__global__ void k_project(int N, const int *__restrict__ cmap, const uint8_t *__restrict__ coarse,
                          uint8_t *__restrict__ fine) {
    d_project(GridTeam(), N, cmap, coarse, fine);
}

__global__ void k_keep_status(RState *st) {
    if (threadIdx.x == 0) st->status0 = st->warn;
}

// ------------------------------------------------------------------------ host side
int64_t balance_limit(int64_t W, int32_t ms, int32_t m, int64_t e6) {
    const __int128 share = (__int128)W * ms;  // the side's share is share / m
    const int64_t a = (int64_t)((share + m - 1) / m);
    const int64_t b = (int64_t)(share * (1000000 + e6) / ((__int128)m * 1000000));
    return a > b ? a : b;
}

static int64_t ceil_sqrt64(int64_t n) {
    if (n <= 0) return 0;
    int64_t r = (int64_t)sqrt((double)n);
    while (r * r > n) r--;
    while ((r + 1) * (r + 1) <= n) r++;
    return r * r == n ? r : r + 1;
}

namespace {

RState *rstate(bipart_graph *g) {
    return reinterpret_cast<RState *>(g->w.small.as<char>() + 256);
}

int *count_n1(bipart_graph *g, Level &L, const uint8_t *side, int *gain);
void node_gains(bipart_graph *g, Level &L, const uint8_t *side, int *gain, int *n1);

// Algorithm 4: side-1 counts, then gains.  A level's first pass counts every hyperedge's side-1
// pins; later passes of the same level (on levels of moderate degree) bring the counts up to
// date from the nodes the selections moved since, which gives the same counts.

void compute_gains(bipart_graph *g, Level &L, const uint8_t *side, int *gain) {
    cudaStream_t s = g->stream;
    Work &w = g->w;
    int *n1;
    if (w.n1_level == &L && (int64_t)L.P <= kDeltaMaxDegree * (int64_t)L.N) {
        // the counts of this level are current up to the nodes moved since: update them
        n1 = w.n1.as<int>() + (size_t)((w.gain_pass - 1) & 1) * w.n1_half;
        ProfScope ps("n1_delta", 4.0 * L.N, s);
        k_n1_delta<<<std::min(grid_for(L.N), kReduceBlocks), kBlock, 0, s>>>(
            L.N, L.noff(), L.nadj(), side, w.moved.as<int>(), rstate(g), n1, gain);
        BP_LAUNCH();
    } else {
        n1 = count_n1(g, L, side, gain);
        w.n1_level = &L;
    }
    if (L.P == 0) return;
    node_gains(g, L, side, gain, n1);
}

// Full count of the side-1 pins of every hyperedge.  The counts alternate between two buffers
// from count to count: a count fills one while its k_hedge_n1 clears the other (dirty over the
// previous count's hyperedges) and the gains.
int *count_n1(bipart_graph *g, Level &L, const uint8_t *side, int *gain) {
    cudaStream_t s = g->stream;
    Work &w = g->w;
    const int cur = w.gain_pass & 1;
    int *n1 = w.n1.as<int>() + (size_t)cur * w.n1_half;
    int *n1_prev = w.n1.as<int>() + (size_t)(cur ^ 1) * w.n1_half;
    {
        // hoff, pins, one side byte per pin, one atomic per hyperedge run; clearing
        ProfScope ps("hedge_n1", 8.0 * L.E + 5.0 * L.P + 4.0 * w.n1_prev_E + 4.0 * L.N, s);
        const int64_t work = std::max<int64_t>({(int64_t)L.P, (int64_t)w.n1_prev_E, (int64_t)L.N});
        k_hedge_n1<<<lb_grid(work), kLbBlock, 0, s>>>(L.E, L.P, L.hoff(), L.pins(), side, n1, L.tsh(),
                                                       n1_prev, w.n1_prev_E, gain, L.N);
        BP_LAUNCH();
    }
    w.gain_pass++;
    w.n1_prev_E = L.E;
    return n1;
}

// gain[v] from the side-1 counts (the gains are zero on entry): on large levels k_node_gain
// gathers each hyperedge's contribution formed by k_hedge_contrib from its degree, count and
// weight; on smaller ones k_node_gain_direct forms it per incidence.
void node_gains(bipart_graph *g, Level &L, const uint8_t *side, int *gain, int *n1) {
    cudaStream_t s = g->stream;
    Work &w = g->w;
    const bool warp_sum = (int64_t)L.P > kWarpSumDegree * (int64_t)L.N;
    if (L.P > kDirectGainPins) {
        int2 *hc = w.hc.as<int2>();
        {
            ProfScope ps("hedge_contrib", 16.0 * L.E + (L.hw() ? 4.0 * L.E : 0.0), s);
            k_hedge_contrib<<<grid_for(L.E), kBlock, 0, s>>>(L.E, L.hoff(), L.hw(), n1, hc);
            BP_LAUNCH();
        }
        // noff, nadj, 8-byte contribution gather per incidence, side, gain
        ProfScope ps("node_gain", 9.0 * L.N + 12.0 * L.P, s);
        k_node_gain<<<lb_grid(L.P), kLbBlock, 0, s>>>(L.N, L.P, L.noff(), L.nadj(), hc, side, gain, L.tsn(),
                                                       warp_sum);
        BP_LAUNCH();
    } else {
        // noff, nadj, gathers of two offsets and a count (and a weight) per incidence, side, gain
        ProfScope ps("node_gain", 9.0 * L.N + 16.0 * L.P + (L.hw() ? 4.0 * L.P : 0.0), s);
        k_node_gain_direct<<<lb_grid(L.P), kLbBlock, 0, s>>>(L.N, L.P, L.noff(), L.nadj(), L.hoff(), L.hw(),
                                                             n1, side, gain, L.tsn(), warp_sum);
        BP_LAUNCH();
    }
}

// Top-K selection per `kind` and its application (flip, or collect for the ordered rebalance).
// With `cond`, a one-block selection also evaluates that loop condition (taking its check slot)
// and returns true; otherwise the caller launches the condition itself.
bool select_apply(bipart_graph *g, Level &L, int kind, long long sq, const int *gain,
                  uint8_t *side, int *list, CondArgs *cond = nullptr, bool weights = false) {
    int *moved = g->w.moved.as<int>();
    cudaStream_t s = g->stream;
    RState *st = rstate(g);
    if (L.N <= kSelOneBlock) {
        // one block: the selection, its exact passes if any, its application (and the condition)
        CondArgs c{COND_NONE, 0, 1, 2, 0, 0, 0, nullptr};
        if (cond) {
            cond->slot = flag_slot(g);
            c = *cond;
        }
        ProfScope ps("select_hist", 9.0 * L.N, s);
        k_sel_small<<<1, kSelOneThreads, 5 * (size_t)std::max(L.N, 1), s>>>(
            L.N, kind, sq, gain, side, L.nw(), st, dev_status(g), list, moved, c, weights);
        BP_LAUNCH();
        return cond != nullptr;
    }
    unsigned *slot = flag_slot(g);
    {
        ProfScope ps("select_hist", 9.0 * L.N, s);
        k_sel<<<std::min(grid_for(L.N), 608), kBlock, 0, s>>>(L.N, kind, sq, gain, side, L.nw(), st, slot);
        BP_LAUNCH();
    }
    if (device_flag(g, &st->slow)) {
        ProfScope ps("select_exact", 3 * 9.0 * L.N, s);
        for (int pass = 0; pass < 3; ++pass) {
            k_sel_exact<<<std::min(grid_for(L.N), 608), kBlock, 0, s>>>(L.N, kind, gain, side, L.nw(), st,
                                                                         dev_status(g));
            BP_LAUNCH();
        }
    }
    ProfScope ps("select_apply", 10.0 * L.N, s);
    scan(L.N, TieIn{kind, gain, side, L.nw(), st}, ApplyOut{kind, gain, side, L.nw(), st, list, moved},
         g->w.scan, dev_status(g), s);
    return false;
}

void side_weights(bipart_graph *g, Level &L, const uint8_t *side, const CondArgs &cond) {
    cudaStream_t s = g->stream;
    RState *st = rstate(g);
    const int grid = std::min(grid_for(L.N), kReduceBlocks);
    auto *partial = (unsigned long long *)g->w.partial.as<void>();
    ProfScope ps("side_weights", 5.0 * L.N, s);
    k_side_weights<<<grid, kBlock, 0, s>>>(L.N, side, L.nw(), st, cond, dev_status(g), partial);
    BP_LAUNCH();
}

// Algorithm 3 on the coarsest level (side 0 grown to its share m0 / m).
void initial_partition(bipart_graph *g, Level &L, uint8_t *side, int *gain, int m0, int m) {
    cudaStream_t s = g->stream;
    if (L.N == 0) return;
    RState *st = rstate(g);
    const long long sq = ceil_sqrt64(L.N);
    BP_CUDA(cudaMemsetAsync(side, 1, (size_t)L.N, s));
    CondArgs c{COND_INITIAL, 1, m0, m, 0, 0, (long long)L.N + 1, flag_slot(g)};
    side_weights(g, L, side, c);
    c.first = 0;
    for (int64_t it = 0; device_flag(g, &st->flag); ++it) {
        if (it > (int64_t)L.N + 2) throw Fail{BIPART_ERR_TIMEOUT, "Algorithm 3 made no progress"};
        compute_gains(g, L, side, gain);
        if (select_apply(g, L, SEL_INITIAL, sq, gain, side, nullptr, &c)) continue;
        c.slot = flag_slot(g);
        ProfScope ps("loop_cond", 0.0, s);
        k_initial_cond<<<1, 32, 0, s>>>(st, c, dev_status(g));
        BP_LAUNCH();
    }
}

// One refinement iteration; with `cond` (the rebalance's first condition, after the last
// iteration) returns whether the selection kernel evaluated it.
bool refine_iter(bipart_graph *g, Level &L, uint8_t *side, int *gain, CondArgs *cond = nullptr) {
    if (L.N == 0) return false;
    compute_gains(g, L, side, gain);
    return select_apply(g, L, SEL_REFINE, 0, gain, side, nullptr, cond, true);
}

CondArgs rebal_cond_args(Level &L, const int64_t limit[2], int first) {
    return CondArgs{COND_REBAL, first, 1, 2, (long long)limit[0], (long long)limit[1], (long long)L.N + 1,
                    nullptr};
}

// Rebalance of reading C13 with a limit per side; leaves warn = 1 when it ran out of candidates.
// `cond_done`: the first condition was evaluated by the last refinement iteration's selection.
void rebalance(bipart_graph *g, Level &L, uint8_t *side, int *gain, const int64_t limit[2],
               bool cond_done) {
    cudaStream_t s = g->stream;
    RState *st = rstate(g);
    const int64_t sq = ceil_sqrt64(L.N);
    if (sq > kRebalMax) throw Fail{BIPART_ERR_OOM, "level too large for the ordered rebalance"};
    int *list = (int *)g->w.list.ensure(sizeof(int) * (size_t)std::max<int64_t>(sq, 1), s);
    int S = 1;
    while (S < sq) S <<= 1;
    const size_t smem = sizeof(unsigned long long) * (size_t)S;
    CondArgs c = rebal_cond_args(L, limit, 1);
    if (!cond_done) {
        c.slot = flag_slot(g);
        side_weights(g, L, side, c);
    }
    c.first = 0;
    for (int64_t it = 0; device_flag(g, &st->flag); ++it) {
        if (it > (int64_t)L.N + 2) throw Fail{BIPART_ERR_TIMEOUT, "rebalance made no progress"};
        compute_gains(g, L, side, gain);
        select_apply(g, L, SEL_REBAL, sq, gain, side, list);
        c.slot = flag_slot(g);
        ProfScope ps("rebal_move", 0.0, s);
        k_rebal_move<<<1, kRebalThreads, smem, s>>>(gain, side, L.nw(), list, st, sq, c, dev_status(g),
                                           g->w.moved.as<int>());
        BP_LAUNCH();
    }
}

}  // namespace

RState *refine_state(bipart_graph *g) { return rstate(g); }

void uncoarsen(bipart_graph *g, std::vector<Level *> &levels, const int64_t limit[2], int m0,
               int m, int32_t iters, uint8_t *d_side0, int tail_from) {
    cudaStream_t s = g->stream;
    const int Lc = (int)levels.size() - 1;
    int64_t nmax = 1, emax = 1;
    for (Level *L : levels) {
        nmax = std::max<int64_t>(nmax, L->N);
        emax = std::max<int64_t>(emax, L->E);
    }
    uint8_t *sa = (uint8_t *)g->w.side_a.ensure((size_t)nmax, s);
    uint8_t *sb = (uint8_t *)g->w.side_b.ensure((size_t)nmax, s);
    int *gain = (int *)g->w.gain.ensure(sizeof(int) * (size_t)nmax, s);
    g->w.hc.ensure(sizeof(int2) * (size_t)emax, s);
    g->w.partial.ensure(sizeof(unsigned long long) * 2 * kReduceBlocks, s);
    // two halves of emax counts, both zero at the start of a bisection (cleared here once in case
    // an earlier run stopped midway)
    g->w.n1_half = emax;
    void *n1 = g->w.n1.ensure(sizeof(int) * 2 * (size_t)emax, s);
    BP_CUDA(cudaMemsetAsync(n1, 0, sizeof(int) * 2 * (size_t)emax, s));
    g->w.gain_pass = 0;
    g->w.n1_prev_E = 0;
    g->w.n1_level = nullptr;
    g->w.moved.ensure(sizeof(int) * (size_t)nmax, s);

    uint8_t *cur = sa, *other = sb;
    // with the tail, the levels from tail_from down are done and sa holds level tail_from's side
    const int top = tail_from >= 0 ? tail_from : Lc;
    if (tail_from < 0) {
        prof_level('r', Lc);
        initial_partition(g, *levels[Lc], cur, gain, m0, m);
    }
    for (int l = top; l >= 0; --l) {
        if (tail_from >= 0 && l == top) continue;
        Level *L = levels[l];
        s = g->stream;
        prof_level('r', l);
        if (l < top) {
            if (L->N > 0) {
                ProfScope ps("project", 6.0 * L->N, s);
                k_project<<<grid_for(L->N), kBlock, 0, s>>>(L->N, L->cmap(), cur, other);
                BP_LAUNCH();
            }
            std::swap(cur, other);
            g->w.n1_level = nullptr;  // a new level: its counts are recounted
        }
        bool cond_done = false;
        for (int it = 0; it < iters; ++it) {
            CondArgs first = rebal_cond_args(*L, limit, 1);
            cond_done = refine_iter(g, *L, cur, gain, it + 1 == iters ? &first : nullptr);
        }
        if (L->N > 0) rebalance(g, *L, cur, gain, limit, cond_done);
        else BP_CUDA(cudaMemsetAsync(&rstate(g)->warn, 0, sizeof(unsigned), g->stream));
    }
    s = g->stream;
    ProfScope ps("loop_cond", 0.0, s);
    k_keep_status<<<1, 32, 0, s>>>(rstate(g));
    BP_LAUNCH();
    if (levels[0]->N > 0)
        BP_CUDA(cudaMemcpyAsync(d_side0, cur, (size_t)levels[0]->N, cudaMemcpyDeviceToDevice, s));
}

const unsigned *bisect_status_word(bipart_graph *g) { return &rstate(g)->status0; }

size_t small_state_bytes() { return 256 + sizeof(RState); }

void refine_init() {
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, []() {
        err = cudaFuncSetAttribute(k_rebal_move, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(sizeof(unsigned long long) * kRebalMax));
        if (err == cudaSuccess)
            err = cudaFuncSetAttribute(k_sel_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       5 * kSelOneBlock);
    });
    BP_CUDA(err);
}

}  // namespace bp
