// Device side of the batched form (see block.cu): the one-block bisection and nested k-way of an
// instance, and the persistent kernel template that block_shapes_*.cu instantiate for each block
// shape.  Everything here is per translation unit except the argument structures.
#pragma once

#include <cuda_runtime.h>

#include "coarsen_dev.cuh"
#include "common.cuh"
#include "internal.h"
#include "refine_dev.cuh"
#include "scan.cuh"

namespace bp {

constexpr int kMaxLev = 64;               // levels a block keeps (instances asking more: grid path)
constexpr int kMaxStack = 64;             // pending part ranges of the nested k-way recursion
constexpr int kBlockMaxK = 1024;          // largest k run inside a block
constexpr size_t kSmemBytes = 32 * 1024;  // union: bitmap window / gain histogram / sort keys /
                                          // a small level's degree counters or fill cursors
constexpr int kPrivNodes = (int)(kSmemBytes / sizeof(int));

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
    int *tsh, *tsn;  // tile-start tables of the hyperedge and incidence CSRs (lb.cuh)
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
    int *dw;  // weighted degree of the level being refined
    unsigned long long *e_key, *n_key;
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
// weights carried, its tile-start table written on the way) with the degrees of c's c.N nodes
// counted into n_a.  ts: the tile starts of the input CSR (null for a raw input).  False on arena
// overflow.
__device__ __noinline__ bool blk_compact(Ctx &x, int E, int P, const int *hoff, const int *hw, DLevel &c,
                                         const int *ts) {
    int *cnt = x.e_a, *emap = x.e_b, *counters = x.cnt4;
    c.hoff = x.ar.take<int>((size_t)E + 1);
    c.hw = hw ? x.ar.take<int>((size_t)E) : nullptr;
    c.tsh = x.ar.take<int>((size_t)P / kTsGran + 2);  // the compacted level has at most P pins
    if (x.ar.overflow) return false;
    if (E > 0) {
        block_scan_items(E, CompactIn{cnt}, CompactOut{E, hw, c.hoff, c.hw, emap, counters + 2, c.tsh});
    } else if (threadIdx.x == 0) {
        c.hoff[0] = 0;
        counters[2] = counters[3] = 0;
    }
    __syncthreads();
    c.E = counters[2];
    c.P = counters[3];
    c.pins = x.ar.take<int>((size_t)c.P);
    if (x.ar.overflow) return false;
    // degree counters of the compacted level: in shared memory when its nodes fit (few nodes
    // means many pins a node, whose atomics would queue on the same global words)
    const bool priv = c.N <= kPrivNodes;
    int *deg = priv ? reinterpret_cast<int *>(x.smem) : x.n_a;
    blk_fill(deg, (size_t)c.N, 0);
    __syncthreads();
    if (P > 0) d_seg_copy(x.t, E, P, hoff, x.p_a, cnt, emap, c.hoff, c.pins, deg, ts);
    __syncthreads();
    if (priv) {
        for (int v = threadIdx.x; v < c.N; v += blockDim.x) x.n_a[v] = deg[v];
        __syncthreads();
    }
    return true;
}

// Node -> hyperedge incidence of `c` from the degrees in n_a.
__device__ __noinline__ bool blk_incidence(Ctx &x, DLevel &c) {
    c.noff = x.ar.take<int>((size_t)c.N + 1);
    c.nadj = x.ar.take<int>((size_t)c.P);
    c.cmap = x.ar.take<int>((size_t)c.N);
    c.match = x.ar.take<int>((size_t)c.N);
    c.tsn = x.ar.take<int>((size_t)c.P / kTsGran + 2);
    if (x.ar.overflow) return false;
    // the fill's cursors in shared memory when the nodes fit (as the degree counters)
    int *cursor = c.N <= kPrivNodes ? reinterpret_cast<int *>(x.smem) : x.n_b;
    if (c.N > 0) block_scan_items(c.N, DegIn{x.n_a}, DegOut{c.N, c.noff, cursor, c.tsn});
    else if (threadIdx.x == 0) c.noff[0] = 0;
    __syncthreads();
    if (c.P > 0) d_fill_adj(x.t, c.E, c.P, c.hoff, c.pins, cursor, c.nadj, c.tsh);
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
    if (f.P > 0) d_match_min(x.t, N, f.P, f.noff, f.nadj, hkey, x.n_key, f.tsn);
    __syncthreads();
    d_match_set(x.t, N, x.n_key, f.nw, f.match, ssize, sweight);
    __syncthreads();
    unsigned long long *best = hkey;  // the hyperedge keys are no longer needed
    blk_fill(best, (size_t)E, ~0ull);
    __syncthreads();
    if (f.P > 0) d_single_best(x.t, E, f.P, f.hoff, f.pins, f.match, ssize, sweight, best, f.tsh);
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
    if (!blk_compact(x, E, f.P, f.hoff, f.hw, c, f.tsh)) return false;
    return blk_incidence(x, c);
}

// ----------------------------------------------------------------- refinement (block versions)
// Weighted degree D[v] = sum of w_e over v's hyperedges, once per level (load-balanced over the
// incidence, one atomic per run).
__device__ __noinline__ void blk_wdeg(Ctx &x, const DLevel &L) {
    blk_fill(x.dw, (size_t)L.N, 0);
    __syncthreads();
    if (L.P > 0) {
        const int *hw = L.hw;
        lb_for_each_items<int>(
            L.noff, L.N, L.P, L.nadj, 0, [&](int, int e, int acc) { return acc + (hw ? hw[e] : 1); },
            [&](int v, int acc) {
                if (acc) atomicAdd(x.dw + v, acc);
            },
            x.t, L.tsn);
    }
    __syncthreads();
}

// Algorithm 4's gains regrouped: an uncut hyperedge gives -w_e to each of its pins and a cut one
// gives +w_e to a pin alone on its side and 0 to the others, so gain[v] = -D[v] + sum over v's
// cut hyperedges of w_e (1 + [v alone on its side]) -- the same integers, with only the cut
// hyperedges touching the gains.  Hyperedges of up to 32 pins take one thread (counting, then
// scattering), larger ones a warp.
__device__ __noinline__ void blk_gains_cut(Ctx &x, const DLevel &L, const uint8_t *side) {
    for (int v = threadIdx.x; v < L.N; v += blockDim.x) x.gain[v] = -x.dw[v];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
    for (int e0 = warp * 32; e0 < L.E; e0 += warps * 32) {
        const int e = e0 + lane;
        int a = 0, d = 0;
        if (e < L.E) {
            a = L.hoff[e];
            d = L.hoff[e + 1] - a;
        }
        const bool small = e < L.E && d <= 32;
        if (small) {
            int n1 = 0;
            for (int i = 0; i < d; ++i) n1 += side[L.pins[a + i]];
            if (n1 > 0 && n1 < d) {
                const int w = L.hw ? L.hw[e] : 1;
                for (int i = 0; i < d; ++i) {
                    const int v = L.pins[a + i];
                    const int mine = side[v] ? n1 : d - n1;
                    atomicAdd(x.gain + v, mine == 1 ? 2 * w : w);
                }
            }
        }
        unsigned big = __ballot_sync(0xffffffffu, e < L.E && !small);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const int eb = e0 + src, ab = L.hoff[eb], db = L.hoff[eb + 1] - ab;
            int n1 = 0;
            for (int i = lane; i < db; i += 32) n1 += side[L.pins[ab + i]];
            n1 = __reduce_add_sync(0xffffffffu, n1);
            if (n1 > 0 && n1 < db) {
                const int w = L.hw ? L.hw[eb] : 1;
                for (int i = lane; i < db; i += 32) {
                    const int v = L.pins[ab + i];
                    const int mine = side[v] ? n1 : db - n1;
                    atomicAdd(x.gain + v, mine == 1 ? 2 * w : w);
                }
            }
        }
    }
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
        blk_gains_cut(x, L, side);
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
        blk_gains_cut(x, L, side);
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
    if (lev[nl - 1].N > 0) blk_wdeg(x, lev[nl - 1]);
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
        if (L.N > 0 && l < nl - 1) blk_wdeg(x, L);  // the coarsest level's came with Algorithm 3
        for (int it = 0; it < I.iters; ++it) {
            if (L.N == 0) break;
            blk_gains_cut(x, L, cur);
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
    x.n_a = x.ar.take<int>(N);
    x.n_b = x.ar.take<int>(N);
    x.n_c = x.ar.take<int>(N);
    x.n_key = x.ar.take<unsigned long long>(N);
    x.gain = x.ar.take<int>(N);
    x.dw = x.ar.take<int>(N);
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
    if (!blk_compact(x, E, P, hoff, hw, G, nullptr)) return 2;
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
        if (!blk_compact(x, G.E, G.P, G.hoff, G.hw, S, G.tsh)) return 2;
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

// Streams v[0, n) through the block, kU independent loads in flight per thread (one load at a time
// would leave a block at a few GB/s); f(i, v[i]) sees every element once.
template <class F>
__device__ __forceinline__ void blk_stream(const int *v, int n, F f) {
    constexpr int kU = 8;
    for (int i0 = threadIdx.x; i0 < n; i0 += kU * blockDim.x) {
        int x[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int i = i0 + u * blockDim.x;
            x[u] = i < n ? v[i] : 0;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i < n) f(i, x[u]);
        }
    }
}

// Whether the instance's staged CSR is well formed: offsets non-decreasing from 0 to P, pins in
// [0, N), weights at least 1 with sums below 2^31 (the handle path's checks).  The whole block runs
// it before anything reads the arrays through an index; every load is bounded by N, E and P.
__device__ bool blk_csr_ok(const BArgs &a, const BInst &I, unsigned long long *s_sum, int *s_bad) {
    if (threadIdx.x == 0) {
        s_sum[0] = s_sum[1] = 0;
        *s_bad = 0;
    }
    __syncthreads();
    const int *hoff = a.hoff + I.hoff;
    bool bad = threadIdx.x == 0 && (hoff[0] != 0 || hoff[I.E] != I.P);
    // offsets: each element against its successor (hoff[e + 1] read through the same stream)
    blk_stream(hoff + 1, I.E, [&](int e, int next) { bad |= next < hoff[e]; });
    const unsigned N = (unsigned)I.N;
    blk_stream(a.pins + I.pins, I.P, [&](int, int v) { bad |= (unsigned)v >= N; });
    unsigned long long sn = 0, se = 0;
    if (I.nw >= 0)
        blk_stream(a.nw + I.nw, I.N, [&](int, int w) {
            bad |= w < 1;
            sn += (unsigned)max(w, 0);
        });
    if (I.hw >= 0)
        blk_stream(a.hw + I.hw, I.E, [&](int, int w) {
            bad |= w < 1;
            se += (unsigned)max(w, 0);
        });
    sn = warp_sum(sn);
    se = warp_sum(se);
    if ((threadIdx.x & 31) == 0) {
        if (sn) atomicAdd(&s_sum[0], sn);
        if (se) atomicAdd(&s_sum[1], se);
    }
    if (bad) atomicOr(s_bad, 1);
    __syncthreads();
    const bool ok = *s_bad == 0 && s_sum[0] < (1ull << 31) && s_sum[1] < (1ull << 31);
    __syncthreads();
    return ok;
}

}  // namespace

template <int BT, int MINB>
__global__ void __launch_bounds__(BT, MINB) k_batch(BArgs a) {
    extern __shared__ __align__(16) char smem[];
    __shared__ DLevel lev[kMaxLev];
    __shared__ int2 stack[kMaxStack];
    __shared__ int s_inst, s_bad;
    __shared__ unsigned long long s_sum[2];
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
        const int st = blk_csr_ok(a, I, s_sum, &s_bad) ? blk_solve(x, a, I, lev, stack) : kBlkMalformed;
        if (threadIdx.x == 0) a.inst[i].status = st;
        __syncthreads();
    }
}

}  // namespace bp
