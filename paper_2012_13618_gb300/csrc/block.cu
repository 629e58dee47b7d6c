// Batched partitioning in persistent launches: every thread block takes whole instances from a
// queue (largest first) and runs the complete partition of an instance on its own -- level-0
// normalisation, coarsening (Algorithms 1-2), the initial partition (Algorithm 3), refinement
// and rebalancing (Algorithms 4-5), and for k > 2 the nested bisections of Algorithm 6 with net
// splitting -- with the phases separated by __syncthreads() instead of kernel boundaries.  The
// phase code is the device code the grid kernels run (coarsen_dev.cuh, refine_dev.cuh)
// instantiated for a one-block team, so an instance's result is identical to the single-instance
// path.
//
// Instances go into size buckets by pin count; each bucket runs as its own persistent launch with
// the block shape (threads, blocks per SM) its tuning chose, and the launches of all buckets,
// with the copies in and out, form one CUDA graph whose branches run at the same time (a bucket
// that runs out of instances frees its SMs for the others).  The graph is kept and replayed while
// the batches keep the same shape.  The tuner times every candidate shape on each bucket of a
// given batch and keeps the winners in a JSON file per device.
//
// Each block owns an arena in HBM (sized by the host for the largest instance of its bucket) from
// which it carves the level store and scratch of its current instance with a bump pointer.  An
// instance whose hierarchy does not fit is marked deferred and the host runs it through the
// single-instance path instead.
#include <cuda_runtime.h>
#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "coarsen_dev.cuh"
#include "common.cuh"
#include "internal.h"
#include "refine_dev.cuh"
#include "scan.cuh"

namespace bp {

namespace {

constexpr int kMaxLev = 64;               // levels a block keeps (instances asking more: grid path)
constexpr int kMaxStack = 64;             // pending part ranges of the nested k-way recursion
constexpr int kBlockMaxK = 1024;          // largest k run inside a block
constexpr size_t kSmemBytes = 32 * 1024;  // union: bitmap window / gain histogram / sort keys

}  // namespace

struct BArgs {
    BInst *inst;
    const int *order;  // this bucket's instances, largest first
    int n;
    int *next;         // this bucket's queue head
    const int *hoff, *pins, *nw, *hw;
    int *parts;
    char *arena;
    size_t arena_bytes;
    uint32_t *status;
};

struct DLevel {
    int N, E, P;
    int *hoff, *pins, *hw, *nw, *noff, *nadj, *cmap, *match;
};

namespace {

// Bump allocator over the block's arena; every thread computes the same pointers.
struct Arena {
    char *base;
    size_t cap, top;
    bool overflow;
    template <class T>
    __device__ T *take(size_t count) {
        size_t bytes = (sizeof(T) * (count ? count : 1) + 255) & ~size_t(255);
        if (top + bytes > cap) {
            overflow = true;
            return reinterpret_cast<T *>(base);  // never dereferenced: the instance is abandoned
        }
        T *p = reinterpret_cast<T *>(base + top);
        top += bytes;
        return p;
    }
};

template <class T>
__device__ void blk_fill(T *a, size_t n, T v) {
    for (size_t i = threadIdx.x; i < n; i += blockDim.x) a[i] = v;
}

struct Ctx {
    CtaTeam t;
    Arena ar;
    char *smem;
    uint32_t *status;
    // scratch (sized by the input instance)
    int *e_a, *e_b, *e_c, *e_d, *n_a, *n_b, *n_c, *p_a, *gain, *list, *cnt4;
    unsigned long long *e_key, *n_key;
    int2 *hc;
    uint8_t *side_a, *side_b;
    signed char *grp;
    RState *st;
    // nested k-way: the part vector and the node maps of the current subgraph
    int *parts, *loc, *l2g, *snw;
};

// Sorted-unique pins of every hyperedge (mapped through map, or as is) into p_a at the
// hyperedge's offset, their counts into e_a.
template <bool MAP>
__device__ __noinline__ void blk_dedup(Ctx &x, int E, const int *hoff, const int *pins, const int *map) {
    int *counters = x.cnt4;
    if (threadIdx.x == 0) { counters[0] = 0; counters[1] = 0; counters[2] = 0; counters[3] = 0; }
    __syncthreads();
    d_seg_small<MAP>(x.t, E, hoff, pins, map, x.p_a, x.e_a, x.e_c, x.e_d, counters);
    __syncthreads();
    d_seg_mid<MAP>(x.t, hoff, pins, map, x.p_a, x.e_a, x.e_c, counters);
    __syncthreads();
    d_seg_big<MAP>(x.t, hoff, pins, map, x.p_a, x.e_a, x.e_d, counters, reinterpret_cast<uint32_t *>(x.smem));
    __syncthreads();
}

// The compacted hyperedge CSR of `c` (hyperedges whose e_a count is >= 2, their pins from p_a,
// weights carried) with the degrees of c's c.N nodes counted into n_a.  False on arena overflow.
__device__ __noinline__ bool blk_compact(Ctx &x, int E, int P, const int *hoff, const int *hw, DLevel &c) {
    int *cnt = x.e_a, *emap = x.e_b, *counters = x.cnt4;
    c.hoff = x.ar.take<int>((size_t)E + 1);
    c.hw = hw ? x.ar.take<int>((size_t)E) : nullptr;
    if (x.ar.overflow) return false;
    if (E > 0) {
        block_scan_items(E, CompactIn{cnt}, CompactOut{E, hw, c.hoff, c.hw, emap, counters + 2, nullptr});
    } else if (threadIdx.x == 0) {
        c.hoff[0] = 0;
        counters[2] = counters[3] = 0;
    }
    __syncthreads();
    c.E = counters[2];
    c.P = counters[3];
    c.pins = x.ar.take<int>((size_t)c.P);
    if (x.ar.overflow) return false;
    blk_fill(x.n_a, (size_t)c.N, 0);  // degree counters of the compacted level
    __syncthreads();
    if (P > 0) d_seg_copy(x.t, E, P, hoff, x.p_a, cnt, emap, c.hoff, c.pins, x.n_a);
    __syncthreads();
    return true;
}

// Node -> hyperedge incidence of `c` from the degrees in n_a.
__device__ __noinline__ bool blk_incidence(Ctx &x, DLevel &c) {
    c.noff = x.ar.take<int>((size_t)c.N + 1);
    c.nadj = x.ar.take<int>((size_t)c.P);
    c.cmap = x.ar.take<int>((size_t)c.N);
    c.match = x.ar.take<int>((size_t)c.N);
    if (x.ar.overflow) return false;
    if (c.N > 0) block_scan_items(c.N, DegIn{x.n_a}, DegOut{c.N, c.noff, x.n_b, nullptr});
    else if (threadIdx.x == 0) c.noff[0] = 0;
    __syncthreads();
    if (c.P > 0) d_fill_adj(x.t, c.E, c.P, c.hoff, c.pins, x.n_b, c.nadj);
    __syncthreads();
    return true;
}

// Algorithms 1 and 2 on level f into c.  Returns false on arena overflow.
__device__ __noinline__ bool blk_coarsen(Ctx &x, const DLevel &f, DLevel &c, int policy) {
    const int N = f.N, E = f.E;
    unsigned long long *hkey = x.e_key;
    int *ssize = x.e_a, *sweight = x.e_b, *gcid = x.e_d, *grp = x.n_c;
    unsigned *rep = reinterpret_cast<unsigned *>(x.e_c);
    d_hedge_key(x.t, E, policy, f.hoff, f.hw, hkey);
    blk_fill(ssize, (size_t)E, 0);
    blk_fill(sweight, (size_t)E, 0);
    blk_fill(rep, (size_t)E, 0xffffffffu);
    blk_fill(x.n_key, (size_t)N, ~0ull);
    __syncthreads();
    if (f.P > 0) d_match_min(x.t, N, f.P, f.noff, f.nadj, hkey, x.n_key);
    __syncthreads();
    d_match_set(x.t, N, x.n_key, f.nw, f.match, ssize, sweight);
    __syncthreads();
    unsigned long long *best = hkey;  // the hyperedge keys are no longer needed
    blk_fill(best, (size_t)E, ~0ull);
    __syncthreads();
    if (f.P > 0) d_single_best(x.t, E, f.P, f.hoff, f.pins, f.match, ssize, sweight, best);
    __syncthreads();
    d_group(x.t, N, f.match, ssize, best, grp, rep);
    __syncthreads();
    if (N > 0) block_scan_items(N, RenumIn{grp, rep}, RenumOut{N, grp, f.cmap, gcid, x.cnt4 + 2});
    __syncthreads();
    c.N = N > 0 ? x.cnt4[2] : 0;
    __syncthreads();
    c.nw = x.ar.take<int>((size_t)c.N);
    if (x.ar.overflow) return false;
    blk_fill(c.nw, (size_t)c.N, 0);
    __syncthreads();
    d_cmap(x.t, N, grp, gcid, f.nw, f.cmap, c.nw);
    __syncthreads();
    blk_dedup<true>(x, E, f.hoff, f.pins, f.cmap);
    if (!blk_compact(x, E, f.P, f.hoff, f.hw, c)) return false;
    return blk_incidence(x, c);
}

// ----------------------------------------------------------------- refinement (block versions)
__device__ __noinline__ void blk_gains(Ctx &x, const DLevel &L, const uint8_t *side) {
    int *n1 = x.e_d;
    blk_fill(n1, (size_t)L.E, 0);
    blk_fill(x.gain, (size_t)L.N, 0);
    __syncthreads();
    if (L.P > 0) d_hedge_n1(x.t, L.E, L.P, L.hoff, L.pins, side, n1);
    __syncthreads();
    d_hedge_contrib(x.t, L.E, L.hoff, L.hw, n1, x.hc);
    __syncthreads();
    if (L.P > 0) d_node_gain(x.t, L.N, L.P, L.noff, L.nadj, x.hc, side, x.gain);
    __syncthreads();
}

// Selection and application of one pass of Algorithm 3 / 5 or of the rebalance.  Levels whose
// nodes fit one tie bitmap word per thread take the shared-memory selection in one sweep.
__device__ __noinline__ void blk_select_apply(Ctx &x, const DLevel &L, int kind, long long sq, uint8_t *side) {
    RState *st = x.st;
    unsigned(*h)[kHistBins] = reinterpret_cast<unsigned(*)[kHistBins]>(x.smem);
    if (L.N <= kSelOneBlock && L.N <= 32 * (int)blockDim.x) {
        d_sel_small(L.N, kind, sq, x.gain, side, L.nw, st, x.status, x.list, nullptr, x.gain, x.grp, h);
        __syncthreads();
        return;
    }
    blk_fill(&st->hist[0][0], (size_t)2 * kHistBins, 0u);
    if (threadIdx.x == 0) st->list_count = 0;
    __syncthreads();
    d_sel_hist(x.t, L.N, kind, x.gain, side, L.nw, st, h);
    __syncthreads();
    d_sel_find(kind, sq, st, st->hist);
    __syncthreads();
    if (st->slow) {
        for (int pass = 0; pass < 3; ++pass) {
            blk_fill(&st->hist[0][0], (size_t)2 * kHistBins, 0u);
            __syncthreads();
            d_sel_hist_exact(x.t, L.N, kind, x.gain, side, L.nw, st, h);
            __syncthreads();
            d_sel_find_exact(st, x.status, st->hist);
            __syncthreads();
        }
    }
    block_scan_items(L.N, TieIn{kind, x.gain, side, L.nw, st}, ApplyOut{kind, x.gain, side, L.nw, st, x.list});
    __syncthreads();
}

__device__ void blk_side_weights(Ctx &x, const DLevel &L, const uint8_t *side) {
    if (threadIdx.x == 0) { x.st->W[0] = 0; x.st->W[1] = 0; }
    __syncthreads();
    d_side_weights(x.t, L.N, side, L.nw, x.st->W);
    __syncthreads();
}

__device__ long long blk_ceil_sqrt(long long n) {
    long long s = (long long)ceilf(sqrtf((float)n));
    while (s * s < n) ++s;
    while (s > 1 && (s - 1) * (s - 1) >= n) --s;
    return s;
}

// Algorithm 3 with side 0 grown to its share m0 / m of the weight (reading G2).
__device__ __noinline__ void blk_initial(Ctx &x, const DLevel &L, uint8_t *side, int m0, int m) {
    if (L.N == 0) return;
    RState *st = x.st;
    const long long s = blk_ceil_sqrt(L.N);
    blk_fill(side, (size_t)L.N, (uint8_t)1);
    if (threadIdx.x == 0) st->rounds = 0;
    __syncthreads();
    blk_side_weights(x, L, side);
    if (threadIdx.x == 0) d_initial_cond(st, (long long)L.N + 1, x.status, true, m0, m);
    __syncthreads();
    while (st->flag) {
        blk_gains(x, L, side);
        blk_select_apply(x, L, SEL_INITIAL, s, side);
        if (threadIdx.x == 0) d_initial_cond(st, (long long)L.N + 1, x.status, false, m0, m);
        __syncthreads();
    }
}

// Rebalance of reading C13 with a limit per side.
__device__ __noinline__ void blk_rebalance(Ctx &x, const DLevel &L, uint8_t *side, long long limit0, long long limit1) {
    RState *st = x.st;
    const long long s = blk_ceil_sqrt(L.N);
    blk_side_weights(x, L, side);
    if (threadIdx.x == 0) d_rebal_cond(st, limit0, limit1, (long long)L.N + 1, x.status, true);
    __syncthreads();
    while (st->flag) {
        blk_gains(x, L, side);
        blk_select_apply(x, L, SEL_REBAL, s, side);
        d_rebal_move(x.gain, side, L.nw, x.list, st, s, reinterpret_cast<unsigned long long *>(x.smem));
        __syncthreads();
        if (threadIdx.x == 0) d_rebal_cond(st, limit0, limit1, (long long)L.N + 1, x.status, false);
        __syncthreads();
    }
}

// Total node weight of a level.
__device__ unsigned long long blk_weight(int N, const int *nw) {
    __shared__ unsigned long long s_w;
    if (threadIdx.x == 0) s_w = 0;
    __syncthreads();
    unsigned long long w = 0;
    for (int v = threadIdx.x; v < N; v += blockDim.x) w += (unsigned long long)nw[v];
    w = warp_sum(w);
    if ((threadIdx.x & 31) == 0 && w) atomicAdd(&s_w, w);
    __syncthreads();
    const unsigned long long r = s_w;
    __syncthreads();
    return r;
}

// The most a side meant for ms of m parts may weigh: max(ceil(W ms / m), floor(W ms (1 + e) / m))
// with e = e6 / 10^6, in exact integer arithmetic.  Within a block W < 2^49 (2^18 nodes of
// int32 weights), m <= 1024 and e6 <= 10^9, so every product below stays under 2^60.
__device__ long long blk_limit(unsigned long long W, int ms, int m, long long e6) {
    const unsigned long long share = W * (unsigned long long)ms;
    const unsigned long long a = (share + (unsigned long long)m - 1) / (unsigned long long)m;
    const unsigned long long D = (unsigned long long)m * 1000000ull, F = 1000000ull + (unsigned long long)e6;
    const unsigned long long b = (share / D) * F + (share % D) * F / D;
    return (long long)(a > b ? a : b);
}

// Sec. 3.4 on the level in lev[0] (incidence built): coarsen until `levels` levels exist or the
// node count stops changing (reading C11), Algorithm 3 on the coarsest level, then refinement and
// rebalancing back to level 0.  *result points at level 0's sides.  Returns the level-0
// rebalance's imbalance flag, or 2 on arena overflow.
__device__ __noinline__ int blk_bisect(Ctx &x, DLevel *lev, const BInst &I, unsigned long long W, int m0, int m,
                          uint8_t **result) {
    const long long lim0 = blk_limit(W, m0, m, I.e6), lim1 = blk_limit(W, m - m0, m, I.e6);
    int nl = 1;
    while (nl - 1 < I.levels && lev[nl - 1].E > 0) {
        const size_t mark = x.ar.top;
        if (!blk_coarsen(x, lev[nl - 1], lev[nl], I.policy)) return 2;
        if (lev[nl].N == lev[nl - 1].N) {
            x.ar.top = mark;
            break;
        }
        ++nl;
    }
    uint8_t *cur = x.side_a, *other = x.side_b;
    blk_initial(x, lev[nl - 1], cur, m0, m);
    for (int l = nl - 1; l >= 0; --l) {
        const DLevel &L = lev[l];
        if (l < nl - 1) {
            d_project(x.t, L.N, L.cmap, cur, other);
            __syncthreads();
            uint8_t *tmp = cur;
            cur = other;
            other = tmp;
        }
        for (int it = 0; it < I.iters; ++it) {
            if (L.N == 0) break;
            blk_gains(x, L, cur);
            blk_select_apply(x, L, SEL_REFINE, 0, cur);
        }
        if (L.N > 0) blk_rebalance(x, L, cur, lim0, lim1);
        else if (threadIdx.x == 0) x.st->warn = 0;
        __syncthreads();
    }
    *result = cur;
    return x.st->warn ? 1 : 0;
}

// Nodes of part `lo` renumbered in ascending id (reading C16): loc (global -> local, -1 outside),
// l2g and the subgraph's node weights; the count goes to *count.
struct SubIn {
    const int *part;
    int lo;
    __device__ uint64_t operator()(int64_t v) const { return part[v] == lo ? 1ull : 0ull; }
};
struct SubOut {
    int64_t n;
    const int *nw;
    int *loc, *l2g, *snw, *count;
    __device__ void operator()(int64_t v, uint64_t pre, uint64_t val) const {
        if (val) {
            loc[v] = (int)pre;
            l2g[pre] = (int)v;
            snw[pre] = nw[v];
        } else {
            loc[v] = -1;
        }
        if (v == n - 1) *count = (int)(pre + val);
    }
};

// Net splitting: every hyperedge of G restricted to the subgraph's nodes (local ids, in G's
// order, which is ascending) into p_a at the hyperedge's offset, the kept counts into e_a.
// Hyperedges of up to 32 pins take one thread, larger ones a warp.
__device__ __noinline__ void blk_split_nets(Ctx &x, const DLevel &G) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
    for (int e0 = warp * 32; e0 < G.E; e0 += warps * 32) {
        const int e = e0 + lane;
        int a = 0, d = 0;
        if (e < G.E) {
            a = G.hoff[e];
            d = G.hoff[e + 1] - a;
        }
        const bool small = e < G.E && d <= 32;
        if (small) {
            int c = 0;
            for (int i = 0; i < d; ++i) {
                const int l = x.loc[G.pins[a + i]];
                if (l >= 0) x.p_a[a + c++] = l;
            }
            x.e_a[e] = c;
        }
        unsigned big = __ballot_sync(0xffffffffu, e < G.E && !small);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const int eb = e0 + src, ab = G.hoff[eb], db = G.hoff[eb + 1] - ab;
            int c = 0;
            for (int i0 = 0; i0 < db; i0 += 32) {
                const int l = i0 + lane < db ? x.loc[G.pins[ab + i0 + lane]] : -1;
                const unsigned keep = __ballot_sync(0xffffffffu, l >= 0);
                if (l >= 0) x.p_a[ab + c + __popc(keep & ((1u << lane) - 1u))] = l;
                c += __popc(keep);
            }
            if (lane == 0) x.e_a[eb] = c;
        }
    }
    __syncthreads();
}

// One whole instance: its parts go to a.parts + I.out.  Returns its status (0 ok, 1 imbalanced,
// 2 deferred).
__device__ int blk_solve(Ctx &x, const BArgs &a, const BInst &I, DLevel *lev, int2 *stack) {
    const int N = I.N, E = I.E, P = I.P;
    int *out = a.parts + I.out;
    // scratch sized by the input (every subgraph is smaller)
    x.e_a = x.ar.take<int>(E);
    x.e_b = x.ar.take<int>(E);
    x.e_c = x.ar.take<int>(E);
    x.e_d = x.ar.take<int>(E);
    x.e_key = x.ar.take<unsigned long long>(E);
    x.hc = x.ar.take<int2>(E);
    x.n_a = x.ar.take<int>(N);
    x.n_b = x.ar.take<int>(N);
    x.n_c = x.ar.take<int>(N);
    x.n_key = x.ar.take<unsigned long long>(N);
    x.gain = x.ar.take<int>(N);
    x.side_a = x.ar.take<uint8_t>(N);
    x.side_b = x.ar.take<uint8_t>(N);
    x.grp = x.ar.take<signed char>(N);
    x.p_a = x.ar.take<int>(P);
    x.list = x.ar.take<int>((size_t)blk_ceil_sqrt(N > 0 ? N : 1) + 2);
    x.cnt4 = x.ar.take<int>(8);
    x.st = x.ar.take<RState>(1);
    if (I.k > 2) {
        x.parts = x.ar.take<int>(N);
        x.loc = x.ar.take<int>(N);
        x.l2g = x.ar.take<int>(N);
        x.snw = x.ar.take<int>(N);
    }
    if (x.ar.overflow) return 2;
    blk_fill(reinterpret_cast<unsigned *>(x.st), sizeof(RState) / sizeof(unsigned), 0u);
    if (I.k == 1) {
        blk_fill(out, (size_t)N, 0);
        __syncthreads();
        return 0;
    }
    // level 0: the normalised input
    const int *hoff = a.hoff + I.hoff, *pins = a.pins + I.pins;
    const int *hw = I.hw >= 0 ? a.hw + I.hw : nullptr;
    DLevel G;
    G.N = N;
    blk_dedup<false>(x, E, hoff, pins, nullptr);
    if (!blk_compact(x, E, P, hoff, hw, G)) return 2;
    G.nw = x.ar.take<int>(N);
    if (x.ar.overflow) return 2;
    for (int v = threadIdx.x; v < N; v += blockDim.x) G.nw[v] = I.nw >= 0 ? a.nw[I.nw + v] : 1;
    __syncthreads();
    if (!blk_incidence(x, G)) return 2;
    lev[0] = G;
    // the top bisection: side 0 meant for ceil(k / 2) of the k parts
    const int m0 = (I.k + 1) / 2;
    uint8_t *side = nullptr;
    int warn = blk_bisect(x, lev, I, blk_weight(N, G.nw), m0, I.k, &side);
    if (warn == 2) return 2;
    int *parts = I.k == 2 ? out : x.parts;
    for (int v = threadIdx.x; v < N; v += blockDim.x) parts[v] = side[v] ? m0 : 0;
    __syncthreads();
    if (I.k == 2) return warn;
    // Algorithm 6: the subgraph holding parts [lo, lo + m) is bisected with side 0 meant for
    // ceil(m / 2) of them until every range holds one part.  Ranges own disjoint part values, so
    // they are taken in any order, each extracted from level 0 by the part vector.
    const size_t mark = x.ar.top;
    int sp = 2;
    if (threadIdx.x == 0) {
        stack[0] = make_int2(m0, I.k - m0);
        stack[1] = make_int2(0, m0);
    }
    __syncthreads();
    while (sp > 0) {
        const int2 r = stack[--sp];
        if (r.y < 2) continue;
        block_scan_items(N, SubIn{parts, r.x}, SubOut{N, G.nw, x.loc, x.l2g, x.snw, x.cnt4 + 4});
        __syncthreads();
        DLevel S;
        S.N = x.cnt4[4];
        __syncthreads();
        if (S.N == 0) continue;
        S.nw = x.snw;
        blk_split_nets(x, G);
        if (!blk_compact(x, G.E, G.P, G.hoff, G.hw, S)) return 2;
        if (!blk_incidence(x, S)) return 2;
        lev[0] = S;
        const int q0 = (r.y + 1) / 2;
        const int w = blk_bisect(x, lev, I, blk_weight(S.N, S.nw), q0, r.y, &side);
        if (w == 2) return 2;
        warn |= w;
        for (int i = threadIdx.x; i < S.N; i += blockDim.x) parts[x.l2g[i]] = side[i] ? r.x + q0 : r.x;
        if (threadIdx.x == 0) {
            stack[sp] = make_int2(r.x + q0, r.y - q0);
            stack[sp + 1] = make_int2(r.x, q0);
        }
        sp += 2;
        x.ar.top = mark;
        __syncthreads();
    }
    for (int v = threadIdx.x; v < N; v += blockDim.x) out[v] = parts[v];
    __syncthreads();
    return warn;
}

}  // namespace

template <int BT, int MINB>
__global__ void __launch_bounds__(BT, MINB) k_batch(BArgs a) {
    extern __shared__ __align__(16) char smem[];
    __shared__ DLevel lev[kMaxLev];
    __shared__ int2 stack[kMaxStack];
    __shared__ int s_inst;
    for (;;) {
        if (threadIdx.x == 0) s_inst = atomicAdd(a.next, 1);
        __syncthreads();
        const int q = s_inst;
        __syncthreads();
        if (q >= a.n) break;
        const int i = a.order[q];
        Ctx x;
        x.ar.base = a.arena + (size_t)blockIdx.x * a.arena_bytes;
        x.ar.cap = a.arena_bytes;
        x.ar.top = 0;
        // a misaligned arena would fault on its 8-byte arrays: defer instead of touching it
        x.ar.overflow = ((uintptr_t)x.ar.base & 255) != 0;
        x.smem = smem;
        x.status = a.status;
        const BInst I = a.inst[i];
        const int st = blk_solve(x, a, I, lev, stack);
        if (threadIdx.x == 0) a.inst[i].status = st;
        __syncthreads();
    }
}

// ------------------------------------------------------------------ host side
namespace {

// Candidate block shapes (threads, blocks per SM asked of the compiler's register budget).  The
// selection of Algorithms 3 and 5 needs at least 256 threads.
struct Shape {
    int threads, per_sm;
    const void *fn;
};
const Shape kShapes[] = {
    {256, 1, (const void *)k_batch<256, 1>},
    {256, 2, (const void *)k_batch<256, 2>},
    {512, 1, (const void *)k_batch<512, 1>},
    {1024, 1, (const void *)k_batch<1024, 1>},
};
constexpr int kNumShapes = (int)(sizeof(kShapes) / sizeof(kShapes[0]));

// Size buckets by pin count: [0, 16K), [16K, 128K), [128K, 1M), [1M, ...).
constexpr int kBuckets = 4;
const int64_t kBucketEdge[kBuckets - 1] = {16 << 10, 128 << 10, 1 << 20};
// Shapes used before a bucket is tuned on this device.
const int kDefaultShape[kBuckets] = {1, 2, 2, 2};

int bucket_of(int64_t P) {
    int b = 0;
    while (b < kBuckets - 1 && P >= kBucketEdge[b]) ++b;
    return b;
}

// Upper bound of the arena bytes an instance may need (level store over all levels, scratch and,
// for k > 2, the part vector, node maps and one subgraph's level store); instances above the
// arena given to their bucket are deferred by the device.
size_t arena_estimate(int64_t N, int64_t E, int64_t P, int k) {
    const int64_t level0 = 4 * (E + 1) + 4 * E + 4 * P + 4 * N + 4 * (N + 1) + 4 * P + 8 * N;
    const int64_t scratch = E * (4 * 4 + 8 + 8) + N * (4 * 3 + 8 + 4 + 3) + 4 * P + 64 * 1024;
    const int64_t kway = k > 2 ? 16 * N + level0 : 0;
    return (size_t)(scratch + 5 * level0 + kway + (4 << 20));
}

// ---------------------------------------------------------------- tuning table (JSON cache)
// {"version": 1, "devices": {"<name> / <SMs> SMs": {"<bucket>": [threads, per_sm], ...}, ...}}
// A minimal reader for exactly this layout (objects, arrays, strings, integers).
struct JVal {
    enum Kind { NUL, NUM, STR, ARR, OBJ } kind = NUL;
    long long num = 0;
    std::string str;
    std::vector<JVal> arr;
    std::vector<std::pair<std::string, JVal>> obj;
};

struct JParse {
    const char *p, *end;
    bool ok = true;
    void ws() {
        while (p < end && (*p == ' ' || *p == '\n' || *p == '\r' || *p == '\t')) ++p;
    }
    bool lit(char c) {
        ws();
        if (p < end && *p == c) {
            ++p;
            return true;
        }
        return false;
    }
    std::string string() {
        std::string s;
        if (!lit('"')) {
            ok = false;
            return s;
        }
        while (p < end && *p != '"') {
            if (*p == '\\' && p + 1 < end) ++p;
            s.push_back(*p++);
        }
        if (p < end) ++p;
        else ok = false;
        return s;
    }
    JVal value(int depth = 0) {
        JVal v;
        ws();
        if (!ok || p >= end || depth > 8) {
            ok = false;
            return v;
        }
        if (*p == '{') {
            ++p;
            v.kind = JVal::OBJ;
            if (lit('}')) return v;
            do {
                std::string k = string();
                if (!lit(':')) ok = false;
                if (!ok) return v;
                v.obj.emplace_back(k, value(depth + 1));
            } while (ok && lit(','));
            if (!lit('}')) ok = false;
        } else if (*p == '[') {
            ++p;
            v.kind = JVal::ARR;
            if (lit(']')) return v;
            do v.arr.push_back(value(depth + 1));
            while (ok && lit(','));
            if (!lit(']')) ok = false;
        } else if (*p == '"') {
            v.kind = JVal::STR;
            v.str = string();
        } else {
            char *q = nullptr;
            v.num = std::strtoll(p, &q, 10);
            if (q == p) ok = false;
            else {
                v.kind = JVal::NUM;
                p = q;
            }
        }
        return v;
    }
};

std::string tune_path() {
    if (const char *e = std::getenv("BIPART_TUNE_CACHE")) return e;
    std::string dir;
    if (const char *x = std::getenv("XDG_CACHE_HOME")) dir = x;
    else if (const char *h = std::getenv("HOME")) dir = std::string(h) + "/.cache";
    else dir = "/tmp";
    return dir + "/bipart/batch_tune.json";
}

void mkdirs_for(const std::string &path) {
    for (size_t i = 1; i < path.size(); ++i)
        if (path[i] == '/') ::mkdir(path.substr(0, i).c_str(), 0755);
}

// device key -> bucket -> shape index
using TuneTable = std::map<std::string, std::map<int, int>>;

TuneTable read_table(const std::string &path) {
    TuneTable t;
    FILE *f = std::fopen(path.c_str(), "rb");
    if (!f) return t;
    std::string text;
    char buf[4096];
    size_t r;
    while ((r = std::fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, r);
    std::fclose(f);
    JParse jp{text.data(), text.data() + text.size()};
    JVal root = jp.value();
    if (!jp.ok || root.kind != JVal::OBJ) return t;
    for (auto &kv : root.obj) {
        if (kv.first != "devices" || kv.second.kind != JVal::OBJ) continue;
        for (auto &dev : kv.second.obj) {
            if (dev.second.kind != JVal::OBJ) continue;
            for (auto &b : dev.second.obj) {
                const int bucket = std::atoi(b.first.c_str());
                if (bucket < 0 || bucket >= kBuckets || b.second.kind != JVal::ARR || b.second.arr.size() != 2) continue;
                for (int s = 0; s < kNumShapes; ++s)
                    if (kShapes[s].threads == b.second.arr[0].num && kShapes[s].per_sm == b.second.arr[1].num)
                        t[dev.first][bucket] = s;
            }
        }
    }
    return t;
}

void write_table(const std::string &path, const TuneTable &t) {
    mkdirs_for(path);
    const std::string tmp = path + ".tmp" + std::to_string((long long)::getpid());
    FILE *f = std::fopen(tmp.c_str(), "wb");
    if (!f) return;  // a cache that cannot be written only costs a re-tune
    std::fprintf(f, "{\"version\": 1, \"devices\": {");
    bool first_dev = true;
    for (auto &dev : t) {
        std::string name;
        for (char c : dev.first) name += (c == '"' || c == '\\') ? '_' : c;
        std::fprintf(f, "%s\n  \"%s\": {", first_dev ? "" : ",", name.c_str());
        bool first = true;
        for (auto &b : dev.second) {
            std::fprintf(f, "%s\"%d\": [%d, %d]", first ? "" : ", ", b.first, kShapes[b.second].threads,
                         kShapes[b.second].per_sm);
            first = false;
        }
        std::fprintf(f, "}");
        first_dev = false;
    }
    std::fprintf(f, "\n}}\n");
    std::fclose(f);
    std::rename(tmp.c_str(), path.c_str());
}

// ---------------------------------------------------------------- the batch context
// Pinned host memory that only grows.
struct Pinned {
    void *p = nullptr;
    size_t cap = 0;
    void *ensure(size_t bytes) {
        if (bytes == 0) bytes = 16;
        if (bytes > cap) {
            if (p) cudaFreeHost(p);
            p = nullptr;
            cap = 0;
            const size_t c = bytes + bytes / 8 + 4096;
            if (cudaHostAlloc(&p, c, cudaHostAllocDefault) != cudaSuccess) {
                cudaGetLastError();
                p = nullptr;
                throw Fail{BIPART_ERR_OOM, "pinned host allocation of " + std::to_string(c) + " bytes failed"};
            }
            cap = c;
        }
        return p;
    }
    void release() {
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
    }
};

// Byte offsets of the batch's arrays in the staging buffers (host and device alike).
struct Layout {
    size_t inst, order, hoff, pins, nw, hw, in_end;  // inputs
    size_t parts, out_end;                           // outputs (after the inputs)
};

struct BucketRun {
    int shape = 0, blocks = 0, count = 0, first = 0;  // instances order[first, first + count)
    size_t arena = 0, arena_off = 0;
};

struct BatchCtx {
    std::mutex mu;
    int device = -1, sms = 0;
    std::string dev_key;
    cudaStream_t stream = nullptr;
    cudaStream_t branch[kBuckets] = {};
    cudaEvent_t fork = nullptr, join[kBuckets] = {};
    Pinned host;                 // inputs then outputs
    Buf dev, arena, misc;
    std::unique_ptr<Lanes> lanes;
    bool attrs = false;
    int occ[kNumShapes] = {};
    // the table: loaded once, updated by the tuner
    bool table_loaded = false;
    TuneTable table;
    // the last graph and the batch shape it was captured for
    cudaGraphExec_t exec = nullptr;
    std::vector<long long> key;

    void init() {
        int dev_now = 0;
        BP_CUDA(cudaGetDevice(&dev_now));
        if (device == dev_now) return;
        if (device >= 0) throw Fail{BIPART_ERR_INVALID_ARG, "the batch path serves one device per process"};
        device = dev_now;
        BP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
        cudaDeviceProp prop;
        BP_CUDA(cudaGetDeviceProperties(&prop, device));
        dev_key = std::string(prop.name) + " / " + std::to_string(sms) + " SMs";
        BP_CUDA(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
        BP_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        for (int b = 0; b < kBuckets; ++b) {
            BP_CUDA(cudaStreamCreateWithFlags(&branch[b], cudaStreamNonBlocking));
            BP_CUDA(cudaEventCreateWithFlags(&join[b], cudaEventDisableTiming));
        }
        for (int s = 0; s < kNumShapes; ++s) {
            BP_CUDA(cudaFuncSetAttribute(kShapes[s].fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes));
            int per = 0;
            BP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kShapes[s].fn, kShapes[s].threads, kSmemBytes));
            occ[s] = std::max(1, std::min(per, kShapes[s].per_sm));
        }
        lanes.reset(new Lanes(16));
    }
    int shape_for(int bucket) {
        if (!table_loaded) {
            table = read_table(tune_path());
            table_loaded = true;
        }
        auto it = table.find(dev_key);
        if (it != table.end()) {
            auto jt = it->second.find(bucket);
            if (jt != it->second.end()) return jt->second;
        }
        return kDefaultShape[bucket];
    }
    void drop_graph() {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        key.clear();
    }
};

BatchCtx &ctx() {
    static BatchCtx *c = new BatchCtx;  // never destroyed: process exit tears the context down
    return *c;
}

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

// Everything a batch call prepares on the host before the device work.
struct Prepared {
    std::vector<int> order;  // instances by bucket, largest first within a bucket
    BucketRun run[kBuckets];
    Layout lay;
    size_t arena_total = 0;
    std::vector<long long> key;
};

Prepared prepare(BatchCtx &c, std::vector<BInst> &inst, const std::vector<const int32_t *> &nw,
                 const std::vector<const int32_t *> &hw, const int *force_shape) {
    const int n = (int)inst.size();
    Prepared pr;
    int64_t sh = 0, sp = 0, sn = 0, sw = 0, so = 0;
    for (int i = 0; i < n; ++i) {
        BInst &I = inst[i];
        I.hoff = sh;
        I.pins = sp;
        I.nw = nw[i] ? sn : -1;
        I.hw = hw[i] ? sw : -1;
        I.out = so;
        I.status = 0;
        sh += I.E + 1;
        sp += I.P;
        if (nw[i]) sn += I.N;
        if (hw[i]) sw += I.E;
        so += I.N;
    }
    std::vector<std::vector<int>> by(kBuckets);
    for (int i = 0; i < n; ++i) by[bucket_of(inst[i].P)].push_back(i);
    // optional override (tests of the deferral path): arena bytes per block in MiB
    size_t arena_cap = 0;
    if (const char *env = std::getenv("BIPART_BLOCK_ARENA_MB")) {
        long long mb = std::atoll(env);
        if (mb > 0) arena_cap = (size_t)mb << 20;
    }
    for (int b = kBuckets - 1; b >= 0; --b) {
        std::vector<int> &v = by[b];
        std::stable_sort(v.begin(), v.end(), [&](int x, int y) { return inst[x].P > inst[y].P; });
        BucketRun &r = pr.run[b];
        r.first = (int)pr.order.size();
        r.count = (int)v.size();
        pr.order.insert(pr.order.end(), v.begin(), v.end());
        if (v.empty()) continue;
        r.shape = force_shape ? force_shape[b] : c.shape_for(b);
        r.blocks = std::min(r.count, c.sms * c.occ[r.shape]);
        size_t a = 0;
        for (int i : v) a = std::max(a, arena_estimate(inst[i].N, inst[i].E, inst[i].P, inst[i].k));
        if (arena_cap) a = std::min(a, arena_cap);
        r.arena = al256(a);
        r.arena_off = pr.arena_total;
        pr.arena_total += r.arena * (size_t)r.blocks;
    }
    Layout &L = pr.lay;
    L.inst = 0;
    L.order = al256(L.inst + sizeof(BInst) * (size_t)n);
    L.hoff = al256(L.order + sizeof(int) * (size_t)n);
    L.pins = al256(L.hoff + sizeof(int) * (size_t)sh);
    L.nw = al256(L.pins + sizeof(int) * (size_t)sp);
    L.hw = al256(L.nw + sizeof(int) * (size_t)sn);
    L.in_end = al256(L.hw + sizeof(int) * (size_t)sw);
    L.parts = L.in_end;
    L.out_end = al256(L.parts + sizeof(int) * (size_t)so);
    // the graph depends on the sizes, the parameters, the bucket shapes and the buffers
    std::vector<long long> &k = pr.key;
    k.reserve((size_t)n * 9 + 4 * kBuckets + 4);
    k.push_back(n);
    for (const BInst &I : inst) {
        k.push_back(I.N);
        k.push_back(I.E);
        k.push_back(I.P);
        k.push_back(I.k);
        k.push_back(I.policy);
        k.push_back(I.levels);
        k.push_back(I.iters);
        k.push_back(I.e6);
        k.push_back((I.nw >= 0) | ((I.hw >= 0) << 1));
    }
    for (int b = 0; b < kBuckets; ++b) {
        k.push_back(pr.run[b].shape);
        k.push_back(pr.run[b].blocks);
        k.push_back((long long)pr.run[b].arena);
    }
    return pr;
}

// Copies the batch's inputs into the pinned staging buffer on the context's host threads.
void stage_inputs(BatchCtx &c, const Prepared &pr, const std::vector<BInst> &inst,
                  const std::vector<const int32_t *> &hoff, const std::vector<const int32_t *> &pins,
                  const std::vector<const int32_t *> &nw, const std::vector<const int32_t *> &hw) {
    char *h = (char *)c.host.p;
    const Layout &L = pr.lay;
    std::memcpy(h + L.inst, inst.data(), sizeof(BInst) * inst.size());
    std::memcpy(h + L.order, pr.order.data(), sizeof(int) * pr.order.size());
    struct Piece {
        void *dst;
        const void *src;
        size_t bytes;
    };
    std::vector<Piece> pieces;
    const size_t kPiece = 4 << 20;
    auto add = [&](size_t off, const int32_t *src, int64_t count) {
        const size_t bytes = sizeof(int32_t) * (size_t)count;
        for (size_t o = 0; o < bytes; o += kPiece)
            pieces.push_back({h + off + o, (const char *)src + o, std::min(kPiece, bytes - o)});
    };
    for (size_t i = 0; i < inst.size(); ++i) {
        const BInst &I = inst[i];
        add(L.hoff + sizeof(int) * (size_t)I.hoff, hoff[i], I.E + 1);
        if (I.P > 0) add(L.pins + sizeof(int) * (size_t)I.pins, pins[i], I.P);
        if (I.nw >= 0) add(L.nw + sizeof(int) * (size_t)I.nw, nw[i], I.N);
        if (I.hw >= 0 && I.E > 0) add(L.hw + sizeof(int) * (size_t)I.hw, hw[i], I.E);
    }
    // pieces grouped into about 64 tasks of similar size
    const size_t tasks = std::min<size_t>(pieces.size(), 64);
    if (tasks == 0) return;
    c.lanes->run((int)tasks, [&](int t) {
        for (size_t j = (size_t)t; j < pieces.size(); j += tasks) std::memcpy(pieces[j].dst, pieces[j].src, pieces[j].bytes);
    });
}

// Records the batch's device work on c.stream: inputs in, one persistent launch per bucket on its
// own branch, outputs back.  Run eagerly or under capture.
void record(BatchCtx &c, const Prepared &pr, int n) {
    char *h = (char *)c.host.p, *d = (char *)c.dev.p;
    const Layout &L = pr.lay;
    cudaStream_t s = c.stream;
    BP_CUDA(cudaMemcpyAsync(d, h, L.in_end, cudaMemcpyHostToDevice, s));
    int *heads = c.misc.as<int>();
    uint32_t *status = reinterpret_cast<uint32_t *>(heads + 16);
    BP_CUDA(cudaMemsetAsync(heads, 0, 256, s));
    BP_CUDA(cudaEventRecord(c.fork, s));
    for (int b = kBuckets - 1; b >= 0; --b) {
        const BucketRun &r = pr.run[b];
        if (r.count == 0) continue;
        cudaStream_t bs = c.branch[b];
        BP_CUDA(cudaStreamWaitEvent(bs, c.fork, 0));
        BArgs a;
        a.inst = reinterpret_cast<BInst *>(d + L.inst);
        a.order = reinterpret_cast<const int *>(d + L.order) + r.first;
        a.n = r.count;
        a.next = heads + b;
        a.hoff = reinterpret_cast<const int *>(d + L.hoff);
        a.pins = reinterpret_cast<const int *>(d + L.pins);
        a.nw = reinterpret_cast<const int *>(d + L.nw);
        a.hw = reinterpret_cast<const int *>(d + L.hw);
        a.parts = reinterpret_cast<int *>(d + L.parts);
        a.arena = c.arena.as<char>() + r.arena_off;
        a.arena_bytes = r.arena;
        a.status = status;
        void *args[] = {&a};
        BP_CUDA(cudaLaunchKernel(kShapes[r.shape].fn, dim3(r.blocks), dim3(kShapes[r.shape].threads), args,
                                 kSmemBytes, bs));
        BP_LAUNCH();
        BP_CUDA(cudaEventRecord(c.join[b], bs));
        BP_CUDA(cudaStreamWaitEvent(s, c.join[b], 0));
    }
    BP_CUDA(cudaMemcpyAsync(h + L.inst, d + L.inst, sizeof(BInst) * (size_t)n, cudaMemcpyDeviceToHost, s));
    BP_CUDA(cudaMemcpyAsync(h + L.parts, d + L.parts, L.out_end - L.parts, cudaMemcpyDeviceToHost, s));
    BP_CUDA(cudaMemcpyAsync(h + L.out_end, status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
}

// Ensures the context's buffers for a prepared batch (dropping the graph when one moves).
void ensure_buffers(BatchCtx &c, const Prepared &pr) {
    const void *h0 = c.host.p, *d0 = c.dev.p, *a0 = c.arena.p, *m0 = c.misc.p;
    c.host.ensure(pr.lay.out_end + 256);
    c.dev.ensure(pr.lay.out_end, c.stream);
    c.arena.ensure(std::max<size_t>(pr.arena_total, 256), c.stream);
    c.misc.ensure(256, c.stream);
    if (c.host.p != h0 || c.dev.p != d0 || c.arena.p != a0 || c.misc.p != m0) c.drop_graph();
}

// Runs a prepared and staged batch (graph replay when the shape repeats); returns kernel ms when
// timed.
float launch(BatchCtx &c, const Prepared &pr, int n, bool use_graph, bool timed) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (timed) {
        BP_CUDA(cudaEventCreate(&e0));
        BP_CUDA(cudaEventCreate(&e1));
        BP_CUDA(cudaEventRecord(e0, c.stream));
    }
    if (use_graph) {
        if (!c.exec || c.key != pr.key) {
            c.drop_graph();
            cudaGraph_t g = nullptr;
            BP_CUDA(cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal));
            try {
                record(c, pr, n);
            } catch (...) {
                cudaStreamEndCapture(c.stream, &g);
                if (g) cudaGraphDestroy(g);
                cudaGetLastError();
                throw;
            }
            BP_CUDA(cudaStreamEndCapture(c.stream, &g));
            const cudaError_t e = cudaGraphInstantiate(&c.exec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                c.exec = nullptr;
                BP_CUDA(e);
            }
            c.key = pr.key;
        }
        BP_CUDA(cudaGraphLaunch(c.exec, c.stream));
    } else {
        record(c, pr, n);
    }
    float ms = 0.f;
    if (timed) BP_CUDA(cudaEventRecord(e1, c.stream));
    BP_CUDA(cudaStreamSynchronize(c.stream));
    if (timed) {
        cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    uint32_t dst = 0;
    std::memcpy(&dst, (char *)c.host.p + pr.lay.out_end, sizeof(dst));
    if (dst & DEV_TIMEOUT) throw Fail{BIPART_ERR_TIMEOUT, "a bounded device loop expired in the batch kernel"};
    return ms;
}

}  // namespace

bool block_eligible(int64_t N, int64_t E, int64_t P, int k, int levels) {
    (void)E;
    return k >= 1 && k <= kBlockMaxK && levels < kMaxLev && N <= (1 << 18) && P <= (1 << 24);
}

void run_block_batch(std::vector<BInst> &inst, const std::vector<const int32_t *> &hoff,
                     const std::vector<const int32_t *> &pins, const std::vector<const int32_t *> &nw,
                     const std::vector<const int32_t *> &hw, const std::vector<int32_t *> &outs) {
    const int n = (int)inst.size();
    if (n == 0) return;
    BatchCtx &c = ctx();
    std::lock_guard<std::mutex> lk(c.mu);
    c.init();
    const bool timing = std::getenv("BIPART_TIMING") != nullptr;
    auto t0 = std::chrono::steady_clock::now();
    Prepared pr = prepare(c, inst, nw, hw, nullptr);
    ensure_buffers(c, pr);
    auto t1 = std::chrono::steady_clock::now();
    stage_inputs(c, pr, inst, hoff, pins, nw, hw);
    auto t2 = std::chrono::steady_clock::now();
    const bool replay = c.exec && c.key == pr.key;
    const float ms = launch(c, pr, n, true, timing);
    auto t3 = std::chrono::steady_clock::now();
    const char *h = (const char *)c.host.p;
    std::memcpy(inst.data(), h + pr.lay.inst, sizeof(BInst) * (size_t)n);
    const int32_t *parts = reinterpret_cast<const int32_t *>(h + pr.lay.parts);
    const int tasks = std::min(n, 64);
    c.lanes->run(tasks, [&](int t) {
        for (int i = t; i < n; i += tasks)
            if (inst[i].status != 2) std::memcpy(outs[i], parts + inst[i].out, sizeof(int32_t) * (size_t)inst[i].N);
    });
    if (timing) {
        auto t4 = std::chrono::steady_clock::now();
        auto dms = [](auto a, auto b) { return std::chrono::duration<double, std::milli>(b - a).count(); };
        std::fprintf(stderr, "[bipart] block batch: %d instances, graph %s, prepare %.2f ms, staging %.2f ms "
                     "(%.1f MiB), device %.2f ms (events %.2f), copy-out %.2f ms\n", n,
                     replay ? "replayed" : "captured", dms(t0, t1), dms(t1, t2), pr.lay.in_end / 1048576.0,
                     dms(t2, t3), ms, dms(t3, t4));
        for (int b = 0; b < kBuckets; ++b)
            if (pr.run[b].count)
                std::fprintf(stderr, "[bipart]   bucket %d: %d instances, %d blocks x %d threads, arena %.1f MiB/block\n",
                             b, pr.run[b].count, pr.run[b].blocks, kShapes[pr.run[b].shape].threads,
                             pr.run[b].arena / 1048576.0);
    }
}

// Times every candidate shape on each bucket of the batch (kernel time by CUDA events, the best
// of two runs) and records the fastest per bucket, in this process and in the JSON cache.
// chosen[2 b], chosen[2 b + 1] receive bucket b's threads and blocks per SM (0 when the batch has
// no instance in it).
void tune_block_batch(std::vector<BInst> &inst, const std::vector<const int32_t *> &hoff,
                      const std::vector<const int32_t *> &pins, const std::vector<const int32_t *> &nw,
                      const std::vector<const int32_t *> &hw, int32_t *chosen) {
    const int n = (int)inst.size();
    BatchCtx &c = ctx();
    std::lock_guard<std::mutex> lk(c.mu);
    c.init();
    if (!c.table_loaded) {
        c.table = read_table(tune_path());
        c.table_loaded = true;
    }
    std::vector<int> counts(kBuckets, 0);
    for (const BInst &I : inst) counts[bucket_of(I.P)]++;
    const bool verbose = std::getenv("BIPART_TIMING") != nullptr;
    for (int b = 0; b < kBuckets; ++b) {
        if (chosen) chosen[2 * b] = chosen[2 * b + 1] = 0;
        if (counts[b] == 0) continue;
        // this bucket's instances alone
        std::vector<BInst> sub;
        std::vector<const int32_t *> sh, sp, sn, sw;
        for (int i = 0; i < n; ++i)
            if (bucket_of(inst[i].P) == b) {
                sub.push_back(inst[i]);
                sh.push_back(hoff[i]);
                sp.push_back(pins[i]);
                sn.push_back(nw[i]);
                sw.push_back(hw[i]);
            }
        int best = -1;
        float best_ms = 0.f;
        for (int s = 0; s < kNumShapes; ++s) {
            int force[kBuckets];
            for (int q = 0; q < kBuckets; ++q) force[q] = s;
            Prepared pr = prepare(c, sub, sn, sw, force);
            ensure_buffers(c, pr);
            stage_inputs(c, pr, sub, sh, sp, sn, sw);
            float ms = 0.f;
            for (int rep = 0; rep < 2; ++rep) {
                const float t = launch(c, pr, (int)sub.size(), false, true);
                ms = rep == 0 ? t : std::min(ms, t);
            }
            int deferred = 0;
            const BInst *out = reinterpret_cast<const BInst *>((const char *)c.host.p + pr.lay.inst);
            for (size_t i = 0; i < sub.size(); ++i) deferred += out[i].status == 2;
            if (verbose)
                std::fprintf(stderr, "[bipart] tune bucket %d (%zu instances): %d x %d per SM: %.2f ms%s\n", b,
                             sub.size(), kShapes[s].threads, kShapes[s].per_sm, ms,
                             deferred ? " (some deferred: not eligible)" : "");
            if (deferred) continue;
            if (best < 0 || ms < best_ms) {
                best = s;
                best_ms = ms;
            }
        }
        if (best < 0) continue;
        c.table[c.dev_key][b] = best;
        if (chosen) {
            chosen[2 * b] = kShapes[best].threads;
            chosen[2 * b + 1] = kShapes[best].per_sm;
        }
    }
    c.drop_graph();
    write_table(tune_path(), c.table);
}

// Frees the batch context's buffers and graph (they are kept between calls otherwise).
void release_block_batch() {
    BatchCtx &c = ctx();
    std::lock_guard<std::mutex> lk(c.mu);
    if (c.device < 0) return;
    if (c.stream) cudaStreamSynchronize(c.stream);
    c.drop_graph();
    c.host.release();
    c.dev.release();
    c.arena.release();
    c.misc.release();
}

}  // namespace bp
