// The coarse tail of a multilevel bisection in one thread-block-cluster launch (Sec. 3.4 from the
// first level of at most kTailNodes nodes down): the remaining coarsening levels (Algorithms 1 and
// 2), the initial partition of the coarsest level (Algorithm 3), and refinement and rebalancing of
// every tail level back up to the level the tail started from (Algorithms 4 and 5).
//
// Why a cluster: small coarse levels still carry 10^4 - 10^5 pins, too many for one block, while
// the grid path spends ~25 dependent launches per level whose cost is latency, not bandwidth (and,
// in an eager call, host round trips for sizes and loop decisions).  A cluster of C blocks
// (C = 16 where the GPU allows it) on C SMs keeps every node-indexed array in each block's shared
// memory, separates phases with cluster barriers (far cheaper than a kernel boundary) and
// combines per-block partial results through distributed shared memory.
//
// Work split: a level's hyperedges are cut into chunks at fixed pin positions (every kTailChunk
// pins, a table per level); block r of C owns the chunks [K r / C, K (r + 1) / C).  A block streams
// its chunks through shared memory -- the next chunk's hyperedge offsets and pins are copied in
// with asynchronous 16-byte copies while the current one is processed -- and every per-hyperedge pass
// (matching keys, weighted degrees, side counts and gains, contraction) scatters into shared-memory
// node arrays.  Node-indexed results are combined by a reduce-scatter (block r owns node slice r)
// and, where every block needs them, an all-gather.  Decisions that follow (the selections of
// Algorithms 3 / 5, the rebalance move, the loop conditions, the renumbering) are computed by every
// block on identical data and come out identical in every block: no block waits on another except
// at a cluster barrier, and every block runs the same sequence of barriers.
//
// Gains use the weighted degree D[v] = sum of w_e over v's hyperedges, computed once per level:
// gain[v] = -D[v] + sum over v's CUT hyperedges of w_e (1 + [v alone on its side]), which is
// Algorithm 4's sum regrouped (an uncut hyperedge contributes -w_e to every pin, a cut one +w_e to
// a pin alone on its side); only cut hyperedges then touch the node arrays.
//
// Results are the same integers as the grid path's: minima and sums are order-independent, ties
// are broken by ids, and the coarse numbering, the contraction order and the selection follow the
// same readings of the paper (C1-C15).  The coarse levels are written to an arena in global memory
// (layout tail_layout(), shared with the host) so the hierarchy stays queryable.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstdlib>
#include <mutex>

#include <cooperative_groups.h>

#include "coarsen_dev.cuh"
#include "common.cuh"
#include "internal.h"
#include "refine_dev.cuh"
#include "tail.h"

namespace bp {

namespace cg = cooperative_groups;

namespace {

constexpr int kTT = kTailThreads;
constexpr int kNT = kTailNodes;
constexpr int kQ = kTailChunk;
constexpr int kThreadDeg = 16;  // hyperedges up to this degree: one thread; above: one warp
constexpr int kWarpDeg = 256;   // contraction: above this, the whole block (bitmap)

// A chunk window in shared memory: the offsets hoff[ha .. e1] and the pins [pa, p1), both from a
// 16-byte aligned start (ha = e0 & ~3, pa = p0 & ~3).  A chunk has at most kQ / 2 + 1 hyperedges
// (every hyperedge has >= 2 pins and starts inside the chunk's kQ pin positions) and, unless one
// of its hyperedges is wider than kQ, fewer than 2 kQ pins; wider chunks are processed from
// global memory.
constexpr int kStageHoff = ((kQ / 2 + 2 + 3 + 3) / 4) * 4;  // hoff[e0 .. e1] from e0 & ~3
constexpr int kStagePins = 2 * kQ + 4;                       // pins[p0 .. p1) from p0 & ~3
constexpr size_t kStageBytes = 4 * (size_t)(kStageHoff + kStagePins);
constexpr int kChunkHedges = kQ / 2 + 1;

// Dynamic shared memory: two chunk stages at the start, then one of two views.
// Coarsening: R0 = 8 kNT bytes (matching keys; later two int arrays), R1 = 4 kNT (matched
// hyperedges; later coarse ids), BM = kNT bits, SW = kNT / 32 word prefixes, then the
// contraction's per-chunk counts and lists.  Refinement: partial and final gains, the block's
// slice of the weighted degrees, two side arrays, the selection groups, the selection state, the
// rebalance's sort keys and candidate list, and the passes' list of wide hyperedges.
constexpr size_t kSTG = 0;
constexpr size_t kV = kSTG + 2 * kStageBytes;

constexpr size_t kR0 = kV;
constexpr size_t kR1 = kR0 + 8 * (size_t)kNT;
constexpr size_t kBM = kR1 + 4 * (size_t)kNT;
constexpr size_t kSW = kBM + (size_t)kNT / 8;
constexpr size_t kCC = kSW + (size_t)kNT / 8;                   // chunk: distinct counts
constexpr size_t kCL = kCC + 4 * (size_t)(kChunkHedges + 3);    // chunk: tier / copy lists
constexpr int kCListMax = 3 * (kQ / 9 + 8);                     // >= 3 ints per hyperedge of degree > 8
constexpr size_t kCoarsenEnd = kCL + 4 * (size_t)kCListMax;

constexpr int kSliceMax = kNT / 4 + 8;                          // a slice has <= ceil(N / 4) nodes
constexpr size_t kGP = kV;                                      // partial gains
constexpr size_t kGF = kGP + 4 * (size_t)kNT;                   // final gains
constexpr size_t kDS = kGF + 4 * (size_t)kNT;                   // weighted degrees of the slice
constexpr size_t kSA = kDS + 4 * (size_t)kSliceMax;
constexpr size_t kSB = kSA + (size_t)kNT;
constexpr size_t kGR = kSB + (size_t)kNT;
constexpr size_t kST = kGR + (size_t)kNT;
constexpr size_t kKY = kST + ((sizeof(RState) + 255) & ~size_t(255));
constexpr int kRebalKeys = 256;  // >= the next power of two of ceil(sqrt(kNT))
constexpr size_t kLS = kKY + 8 * (size_t)kRebalKeys;
constexpr size_t kWL = kLS + 4 * (size_t)kRebalKeys;           // wide hyperedges of a chunk
constexpr size_t kRefineEnd = kWL + 4 * (size_t)(kChunkHedges + 3);

constexpr size_t kSmemBytes = kCoarsenEnd > kRefineEnd ? kCoarsenEnd : kRefineEnd;

__device__ __forceinline__ void csync() { cg::this_cluster().sync(); }

template <class T>
__device__ __forceinline__ T *remote(T *p, int rank) {
    return cg::this_cluster().map_shared_rank(p, rank);
}

// Diagnostics: block 0's thread 0 stamps (tag, nanoseconds) pairs after a count in trace[0];
// tag = level << 8 | phase.
__device__ __forceinline__ void trace(const TailArgs &a, int level, int phase) {
    if (!a.trace || threadIdx.x != 0 || cg::this_cluster().block_rank() != 0) return;
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    const unsigned long long i = a.trace[0]++;
    if (i < (unsigned long long)kTailTraceMax) {
        a.trace[1 + 2 * i] = ((unsigned long long)level << 8) | (unsigned)phase;
        a.trace[2 + 2 * i] = t;
    }
}

// ceil(sqrt(n)) in integers (reading C14).
__device__ __forceinline__ long long d_ceil_sqrt(long long n) {
    if (n <= 0) return 0;
    long long r = (long long)sqrt((double)n);
    while (r * r > n) --r;
    while ((r + 1) * (r + 1) <= n) ++r;
    return r * r == n ? r : r + 1;
}

struct TLev {
    int N, E, P, K;
    const int *hoff, *pins, *hw, *nw;
    int *cmap, *match;
    int *ce, *cp;  // chunk table: chunk c = hyperedges [ce[c], ce[c + 1]), pins [cp[c], cp[c + 1])
};

// Slice of [0, n) owned by block r of C.
__device__ __forceinline__ int slice_lo(int n, int r, int C) { return (int)((long long)n * r / C); }

// The block whose slice holds node v.
__device__ __forceinline__ int slice_of(int n, int v, int C) {
    int q = (int)((long long)v * C / n);
    while (q > 0 && v < slice_lo(n, q, C)) --q;
    while (q + 1 < C && v >= slice_lo(n, q + 1, C)) ++q;
    return q;
}

// Chunk table entries of hyperedge e (first pin o, k pins): every boundary c * kQ in (o, o + k]
// starts its chunk at hyperedge e + 1 (pin o + k).
__device__ __forceinline__ void mark_chunks(int *ce, int *cp, int e, int o, int k) {
    for (int c = o / kQ + 1; (long long)c * kQ <= (long long)o + k; ++c) {
        ce[c] = e + 1;
        cp[c] = o + k;
    }
}

// ------------------------------------------------------------------------ chunk streaming
// The block's chunks of a level, their table in shared memory (entries c_lo .. c_hi).
struct Chunks {
    int c_lo, c_hi;
    const int *ce, *cp;
};

__device__ void load_chunks(const TLev &L, int r, int C, Chunks &ch, int *s_ce, int *s_cp) {
    ch.c_lo = (int)((long long)L.K * r / C);
    ch.c_hi = (int)((long long)L.K * (r + 1) / C);
    ch.ce = s_ce;
    ch.cp = s_cp;
    __syncthreads();  // the previous table may still be read
    for (int i = threadIdx.x; i <= ch.c_hi - ch.c_lo; i += kTT) {
        s_ce[i] = __ldcg(L.ce + ch.c_lo + i);
        s_cp[i] = __ldcg(L.cp + ch.c_lo + i);
    }
    __syncthreads();
}

// A chunk window; H and P address hyperedge offsets and pins by their global indices, from the
// shared copy (generic pointers into shared memory) or, for a wide chunk, from global memory.
struct Win {
    int e0, e1, p0, p1, ha, pa;
    bool wide;
    const int *H, *P;
};

__device__ __forceinline__ Win make_win(const TLev &L, const Chunks &ch, int c) {
    Win w;
    w.e0 = ch.ce[c - ch.c_lo];
    w.e1 = ch.ce[c - ch.c_lo + 1];
    w.p0 = ch.cp[c - ch.c_lo];
    w.p1 = ch.cp[c - ch.c_lo + 1];
    w.ha = w.e0 & ~3;
    w.pa = w.p0 & ~3;
    w.wide = w.p1 - w.pa > kStagePins;
    w.H = L.hoff;
    w.P = L.pins;
    return w;
}

// 16-byte asynchronous copies global -> shared (no registers held while they fly).
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Issues the copies of window w into `stage` and points w at it (16-byte pieces from 16-byte
// aligned starts; the arrays carry slack after their ends for the last piece).
__device__ __forceinline__ void win_issue(const TLev &L, Win &w, int *stage) {
    int *sh = stage, *sp = stage + kStageHoff;
    const int nh = (w.e1 + 1 - w.ha + 3) >> 2;
    for (int i = threadIdx.x; i < nh; i += kTT) cp_async16(sh + 4 * i, L.hoff + w.ha + 4 * i);
    w.H = sh - w.ha;
    if (!w.wide) {
        const int np = (w.p1 - w.pa + 3) >> 2;
        for (int i = threadIdx.x; i < np; i += kTT) cp_async16(sp + 4 * i, L.pins + w.pa + 4 * i);
        w.P = sp - w.pa;
    }
    cp_async_commit();
}

// Streams the block's chunks: fn(w) for every chunk window once it is in shared memory, the next
// chunk's copies in flight meanwhile.  fn may use __syncthreads (every thread calls it).
template <class Fn>
__device__ __forceinline__ void stream(const TLev &L, const Chunks &ch, char *smem, Fn fn) {
    if (ch.c_lo >= ch.c_hi) return;
    int *stages[2] = {reinterpret_cast<int *>(smem + kSTG), reinterpret_cast<int *>(smem + kSTG + kStageBytes)};
    Win w = make_win(L, ch, ch.c_lo);
    win_issue(L, w, stages[0]);
    for (int c = ch.c_lo; c < ch.c_hi; ++c) {
        cp_async_wait_all();
        __syncthreads();  // chunk c is in place, and everyone is done with the other stage
        const Win cur = w;
        if (c + 1 < ch.c_hi) {
            w = make_win(L, ch, c + 1);
            win_issue(L, w, stages[(c + 1 - ch.c_lo) & 1]);
        }
        fn(cur);
    }
    __syncthreads();
}

// Per-hyperedge pass over a window: one(e, a, d) by a thread for degrees <= kThreadDeg, then
// wide(e, a, d) by a whole warp for the others; `list` holds kChunkHedges entries, `cnt` is a
// shared counter.
template <class One, class Wide>
__device__ __forceinline__ void win_hedges(const Win &w, int *list, int *cnt, One one, Wide wide) {
    if (threadIdx.x == 0) *cnt = 0;
    __syncthreads();
    for (int e = w.e0 + (int)threadIdx.x; e < w.e1; e += kTT) {
        const int a = w.H[e], d = w.H[e + 1] - a;
        if (d > kThreadDeg) list[atomicAdd(cnt, 1)] = e;
        else one(e, a, d);
    }
    __syncthreads();
    const int n = *cnt;
    for (int i = threadIdx.x >> 5; i < n; i += kTT / 32) {
        const int e = list[i];
        const int a = w.H[e], d = w.H[e + 1] - a;
        wide(e, a, d);
    }
}

// The chunk table of a level whose hyperedges are split among the blocks by count (the starting
// level; coarse levels get theirs from the contraction).
__device__ void build_chunks(const TLev &L, int r, int C) {
    const int e_lo = slice_lo(L.E, r, C), e_hi = slice_lo(L.E, r + 1, C);
    for (int e0 = e_lo + 8 * (int)threadIdx.x; e0 < e_hi; e0 += 8 * kTT) {
        int o[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) o[k] = e0 + k <= e_hi ? __ldg(L.hoff + e0 + k) : 0;
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (e0 + k < e_hi) mark_chunks(L.ce, L.cp, e0 + k, o[k], o[k + 1] - o[k]);
    }
    if (r == 0 && threadIdx.x == 0) {
        L.ce[0] = 0;
        L.cp[0] = 0;
        L.ce[L.K] = L.E;
        L.cp[L.K] = L.P;
    }
}

// ------------------------------------------------------------------------------ coarsening
// Algorithms 1 and 2 on level f into level c, written at arena offset *top.  Returns false (in
// every block) when the arena is too small; *need then holds the bytes that would have been
// needed.
__device__ bool tail_coarsen(const TailArgs &a, const TLev &f, TLev &c, size_t *top, size_t *need,
                             int lv, char *smem, int *s_ce, int *s_cp) {
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks(), r = (int)cl.block_rank();
    const int N = f.N;
    unsigned long long *s_key = reinterpret_cast<unsigned long long *>(smem + kR0);
    int *s_match = reinterpret_cast<int *>(smem + kR1);
    int *clist = reinterpret_cast<int *>(smem + kCL);
    __shared__ int s_cnt[4];
    __shared__ unsigned long long s_red[33];
    trace(a, lv, 1);
    Chunks ch;
    load_chunks(f, r, C, ch, s_ce, s_cp);
    const int ea = ch.ce[0], eb = ch.ce[ch.c_hi - ch.c_lo];
    const int pa_r = ch.cp[0];
    // matching keys of this block's copy; the per-hyperedge accumulators of this block's range
    for (int v = threadIdx.x; v < N; v += kTT) s_key[v] = ~0ull;
    for (int e = ea + (int)threadIdx.x; e < eb; e += kTT) {
        a.e_ssize[e] = 0;
        a.e_sweight[e] = 0;
        a.e_rep[e] = 0xffffffffu;
    }
    // Algorithm 1: every node keeps the smallest (priority, hash) key of its hyperedges (the
    // hash is a bijection of the id, so the key names the hyperedge); shared-memory minima, read
    // first so that most pins need no atomic
    auto hkey = [&](int e, int d) -> unsigned long long {
        const uint32_t h = mix32((uint32_t)e);
        const uint32_t w = f.hw ? (uint32_t)__ldg(f.hw + e) : 1u;
        return ((unsigned long long)policy_priority(a.policy, (uint32_t)d, w, h) << 32) | h;
    };
    stream(f, ch, smem, [&](const Win &w) {
        win_hedges(w, clist, &s_cnt[0],
                   [&](int e, int b0, int d) {
                       const unsigned long long k = hkey(e, d);
                       for (int i = 0; i < d; ++i) {
                           const int u = w.P[b0 + i];
                           if (k < s_key[u]) atomicMin(&s_key[u], k);
                       }
                   },
                   [&](int e, int b0, int d) {
                       const unsigned long long k = hkey(e, d);
                       for (int i = threadIdx.x & 31; i < d; i += 32) {
                           const int u = w.P[b0 + i];
                           if (k < s_key[u]) atomicMin(&s_key[u], k);
                       }
                   });
    });
    trace(a, lv, 2);
    csync();
    // reduce-scatter of the minima: this block owns nodes [nlo, nhi); match and the sizes and
    // weights of the matched sets S(e) (global integer atomics)
    const int nlo = slice_lo(N, r, C), nhi = slice_lo(N, r + 1, C);
    for (int v = nlo + (int)threadIdx.x; v < nhi; v += kTT) {
        unsigned long long k = s_key[v];
        for (int q = 0; q < C; ++q) {
            if (q == r) continue;
            const unsigned long long x = remote(s_key, q)[v];
            k = x < k ? x : k;
        }
        const int m = k == ~0ull ? -1 : (int)unmix32((uint32_t)k);
        f.match[v] = m;
        if (m >= 0) {
            atomicAdd(&a.e_ssize[m], 1);
            atomicAdd(&a.e_sweight[m], __ldg(f.nw + v));
        }
    }
    csync();
    trace(a, lv, 3);
    // every block: the matching of all nodes, and for each node the weight of its step-1 merged
    // set (-1 when it is not in one): Algorithm 2's first loop
    int *s_mw = reinterpret_cast<int *>(smem + kR0);  // keys are dead now
    for (int v0 = threadIdx.x; v0 < N; v0 += 4 * kTT) {
        int m[4], sz[4], wt[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int v = v0 + u * kTT;
            m[u] = v < N ? __ldcg(f.match + v) : -1;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            sz[u] = m[u] >= 0 ? __ldcg(a.e_ssize + m[u]) : 0;
            wt[u] = m[u] >= 0 ? __ldcg(a.e_sweight + m[u]) : 0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int v = v0 + u * kTT;
            if (v < N) {
                s_match[v] = m[u];
                s_mw[v] = sz[u] >= 2 ? wt[u] : -1;
            }
        }
    }
    __syncthreads();
    // Algorithm 2's second loop (reading C7) for this block's node slice: a singleton set {u}
    // joins the lightest step-1 merged node among the pins of its hyperedge (ties: smaller set
    // id); grp = the matched hyperedge of the final group, -1 alone; rep = smallest member
    {
        const int lane = threadIdx.x & 31;
        for (int v0 = nlo + (int)(threadIdx.x & ~31); v0 < nhi; v0 += kTT) {
            const int v = v0 + lane;
            int g = -1, wide = 0, b0 = 0, d = 0;
            if (v < nhi) {
                const int m = s_match[v];
                if (m >= 0) {
                    if (s_mw[v] >= 0) {
                        g = m;
                    } else {
                        b0 = __ldg(f.hoff + m);
                        d = __ldg(f.hoff + m + 1) - b0;
                        if (d <= 32) {
                            unsigned long long best = ~0ull;
                            for (int i = 0; i < d; ++i) {
                                const int u = __ldg(f.pins + b0 + i);
                                const int w = s_mw[u];
                                if (w >= 0) {
                                    const unsigned long long k = ((unsigned long long)(unsigned)w << 32) | (unsigned)s_match[u];
                                    best = k < best ? k : best;
                                }
                            }
                            g = best == ~0ull ? -1 : (int)(best & 0xffffffffu);
                        } else {
                            wide = 1;
                        }
                    }
                }
            }
            // singletons of hyperedges wider than a warp: the whole warp scans the pins
            unsigned todo = __ballot_sync(0xffffffffu, wide);
            while (todo) {
                const int src = __ffs(todo) - 1;
                todo &= todo - 1;
                const int bb = __shfl_sync(0xffffffffu, b0, src), dd = __shfl_sync(0xffffffffu, d, src);
                unsigned long long best = ~0ull;
                for (int i = lane; i < dd; i += 32) {
                    const int u = __ldg(f.pins + bb + i);
                    const int w = s_mw[u];
                    if (w >= 0) {
                        const unsigned long long k = ((unsigned long long)(unsigned)w << 32) | (unsigned)s_match[u];
                        best = k < best ? k : best;
                    }
                }
                best = warp_min(best);
                if (lane == src) g = best == ~0ull ? -1 : (int)(best & 0xffffffffu);
            }
            if (v < nhi) {
                a.n_grp[v] = g;
                if (g >= 0) atomicMin(&a.e_rep[g], (unsigned)v);
            }
        }
    }
    csync();
    trace(a, lv, 4);
    // every block: coarse ids ascending by smallest member (reading C8), coarse node weights
    int *s_rv = reinterpret_cast<int *>(smem + kR0 + 4 * (size_t)kNT);  // representative
    int *s_cw = reinterpret_cast<int *>(smem + kR0);                     // coarse weights
    unsigned *bm = reinterpret_cast<unsigned *>(smem + kBM);
    int *sw = reinterpret_cast<int *>(smem + kSW);
    int *s_cmap = s_match;                                               // matches are dead now
    const int words = (N + 31) >> 5;
    for (int i = threadIdx.x; i < words; i += kTT) bm[i] = 0;
    __syncthreads();
    for (int v0 = threadIdx.x; v0 < N; v0 += 4 * kTT) {
        int gg[4], rv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int v = v0 + u * kTT;
            gg[u] = v < N ? __ldcg(a.n_grp + v) : -1;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) rv[u] = gg[u] < 0 ? v0 + u * kTT : (int)__ldcg(a.e_rep + gg[u]);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int v = v0 + u * kTT;
            if (v < N) {
                s_rv[v] = rv[u];
                if (rv[u] == v) atomicOr(&bm[v >> 5], 1u << (v & 31));
            }
        }
    }
    __syncthreads();
    int Nc;
    {
        // exclusive prefix of the representative bits per word (words <= kNT / 32 <= kTT)
        const int t = threadIdx.x;
        const unsigned long long cw = t < words ? (unsigned long long)__popc(bm[t]) : 0ull;
        unsigned long long tot;
        const unsigned long long ex = block_exclusive_scan<unsigned long long>(cw, s_red, &tot);
        if (t < words) sw[t] = (int)ex;
        Nc = (int)tot;
    }
    __syncthreads();
    for (int v = threadIdx.x; v < N; v += kTT) {
        const int rv = s_rv[v];
        s_cmap[v] = sw[rv >> 5] + __popc(bm[rv >> 5] & ((1u << (rv & 31)) - 1u));
    }
    for (int x = threadIdx.x; x < Nc; x += kTT) s_cw[x] = 0;
    __syncthreads();
    for (int v = threadIdx.x; v < N; v += kTT) {
        atomicAdd(&s_cw[s_cmap[v]], __ldg(f.nw + v));
        if (v >= nlo && v < nhi) f.cmap[v] = s_cmap[v];
    }
    __syncthreads();
    trace(a, lv, 5);
    // contraction (Algorithm 2, reading C9), chunk by chunk in ascending hyperedge order: every
    // hyperedge's pins mapped to coarse ids, sorted and de-duplicated; the kept ones (>= 2
    // distinct pins) compacted into this block's staging area (pins at [pa_r, ...), offsets and
    // weights at [ea, ...)), whose place in the coarse level is known once every block has its
    // totals
    int *s_cc = reinterpret_cast<int *>(smem + kCC);  // distinct counts of the chunk's hyperedges
    int *stage_p = a.p_stage;                         // staged coarse pins
    int *wide_p = a.p_stage + a.P;                    // distinct pins of wide hyperedges
    uint32_t *cbits = reinterpret_cast<uint32_t *>(smem + kBM);  // block-tier bitmap (bm is dead)
    long long run_e = 0, run_p = 0;                   // staged so far by this block
    stream(f, ch, smem, [&](const Win &w) {
        // the distinct pins of every hyperedge replace its own pins in the window (each tier reads
        // all of a hyperedge's pins before writing any); a wide window keeps them in wide_p
        int *dout = w.wide ? wide_p : const_cast<int *>(w.P);
        // each thread: a contiguous run of the chunk's hyperedges (ascending)
        const int nhe = w.e1 - w.e0;
        const int per = (nhe + kTT - 1) / kTT;
        const int i0 = (int)threadIdx.x * per;
        if (threadIdx.x == 0) { s_cnt[0] = 0; s_cnt[1] = 0; s_cnt[2] = 0; }
        __syncthreads();
        for (int j = 0; j < per; ++j) {
            const int i = i0 + j;
            if (i >= nhe) break;
            const int e = w.e0 + i;
            const int b0 = w.H[e], d = w.H[e + 1] - b0;
            if (d <= kSmallDeg) {
                int v[kSmallDeg];
#pragma unroll
                for (int k = 0; k < kSmallDeg; ++k) v[k] = k < d ? s_cmap[w.P[b0 + k]] : INT_MAX;
                sort_net<kSmallDeg>(v);
                int m = 0;
#pragma unroll
                for (int k = 0; k < kSmallDeg; ++k)
                    if (k < d && (k == 0 || v[k] != v[k - 1])) dout[b0 + m++] = v[k];
                s_cc[i] = m;
            } else if (d <= kWarpDeg) {
                clist[atomicAdd(&s_cnt[0], 1)] = i;
            } else {
                clist[kCListMax - 1 - atomicAdd(&s_cnt[1], 1)] = i;
            }
        }
        __syncthreads();
        {
            // warp tier: register bitonic sort of the mapped pins
            const int n = s_cnt[0];
            const int lane = threadIdx.x & 31;
            for (int k = threadIdx.x >> 5; k < n; k += kTT / 32) {
                const int i = clist[k];
                const int e = w.e0 + i;
                const int b0 = w.H[e], d = w.H[e + 1] - b0;
                int m;
                if (d <= 32) m = warp_unique<1, true, CtaTeam>(w.P, s_cmap, b0, d, dout + b0);
                else if (d <= 64) m = warp_unique<2, true, CtaTeam>(w.P, s_cmap, b0, d, dout + b0);
                else if (d <= 128) m = warp_unique<4, true, CtaTeam>(w.P, s_cmap, b0, d, dout + b0);
                else m = warp_unique<8, true, CtaTeam>(w.P, s_cmap, b0, d, dout + b0);
                if (lane == 0) s_cc[i] = m;
            }
        }
        {
            // block tier (rare): one bit per coarse node (Nc <= kNT), read out in order
            const int n = s_cnt[1];
            const int cwords = (Nc + 31) >> 5;
            for (int k = 0; k < n; ++k) {
                const int i = clist[kCListMax - 1 - k];
                const int e = w.e0 + i;
                const int b0 = w.H[e], d = w.H[e + 1] - b0;
                __syncthreads();
                for (int q = threadIdx.x; q < cwords; q += kTT) cbits[q] = 0;
                __syncthreads();
                for (int q = threadIdx.x; q < d; q += kTT) {
                    const int x = s_cmap[w.P[b0 + q]];
                    atomicOr(&cbits[x >> 5], 1u << (x & 31));
                }
                __syncthreads();
                const int t = threadIdx.x;
                const unsigned long long cb = t < cwords ? (unsigned long long)__popc(cbits[t]) : 0ull;
                unsigned long long tot;
                const unsigned long long ex = block_exclusive_scan<unsigned long long>(cb, s_red, &tot);
                if (t < cwords) {
                    unsigned bits = cbits[t];
                    int o = b0 + (int)ex;
                    while (bits) {
                        const int bit = __ffs(bits) - 1;
                        bits &= bits - 1;
                        dout[o++] = 32 * t + bit;
                    }
                }
                if (t == 0) s_cc[i] = (int)tot;
            }
        }
        __syncthreads();
        // ordered compaction of the chunk: (kept, pins) prefix over the threads' runs
        unsigned long long loc = 0;
        for (int j = 0; j < per; ++j) {
            const int i = i0 + j;
            if (i >= nhe) break;
            const int k = s_cc[i];
            if (k >= 2) loc += (1ull << 32) | (unsigned)k;
        }
        unsigned long long ctot;
        const unsigned long long pre = block_exclusive_scan<unsigned long long>(loc, s_red, &ctot);
        long long le = run_e + (long long)(pre >> 32), lp = run_p + (long long)(pre & 0xffffffffu);
        for (int j = 0; j < per; ++j) {
            const int i = i0 + j;
            if (i >= nhe) break;
            const int k = s_cc[i];
            if (k < 2) continue;
            const int e = w.e0 + i;
            a.e_soff[ea + le] = (int)lp;
            if (f.hw) a.e_shw[ea + le] = __ldg(f.hw + e);
            const int b0 = w.H[e];
            if (k <= 16) {
                int *dst = stage_p + pa_r + lp;
                for (int q = 0; q < k; ++q) dst[q] = dout[b0 + q];
            } else {
                const int slot = atomicAdd(&s_cnt[2], 1);  // copied by a warp below
                clist[3 * slot] = b0;
                clist[3 * slot + 1] = (int)(pa_r + lp);
                clist[3 * slot + 2] = k;
            }
            ++le;
            lp += k;
        }
        __syncthreads();
        {
            const int n = s_cnt[2];
            const int lane = threadIdx.x & 31;
            for (int k = threadIdx.x >> 5; k < n; k += kTT / 32) {
                const int b0 = clist[3 * k], o = clist[3 * k + 1], m = clist[3 * k + 2];
                for (int t = lane; t < m; t += 32) stage_p[o + t] = dout[b0 + t];
            }
        }
        run_e += (long long)(ctot >> 32);
        run_p += (long long)(ctot & 0xffffffffu);
    });
    trace(a, lv, 6);
    if (threadIdx.x == 0) {
        a.xchg[2 * r] = run_e;
        a.xchg[2 * r + 1] = run_p;
    }
    csync();
    trace(a, lv, 7);
    long long Eb = 0, Pb = 0, Ec = 0, Pc = 0;
    for (int q = 0; q < C; ++q) {
        const long long eq = __ldcg(a.xchg + 2 * q), pq = __ldcg(a.xchg + 2 * q + 1);
        if (q < r) { Eb += eq; Pb += pq; }
        Ec += eq;
        Pc += pq;
    }
    c.N = Nc;
    c.E = (int)Ec;
    c.P = (int)Pc;
    c.K = tail_chunks(c.P);
    const bool weighted = f.hw != nullptr;
    const TailLayout lay = tail_layout(*top, c.N, c.E, c.P, weighted);
    if (lay.end > a.arena_cap) {
        *need = lay.end;
        return false;  // the same decision in every block
    }
    *top = lay.end;
    char *base = a.arena;
    int *c_nw = reinterpret_cast<int *>(base + lay.nw);
    int *c_hoff = reinterpret_cast<int *>(base + lay.hoff);
    int *c_hw = weighted ? reinterpret_cast<int *>(base + lay.hw) : nullptr;
    int *c_pins = reinterpret_cast<int *>(base + lay.pins);
    c.nw = c_nw;
    c.hoff = c_hoff;
    c.hw = c_hw;
    c.pins = c_pins;
    c.cmap = reinterpret_cast<int *>(base + lay.cmap);
    c.match = reinterpret_cast<int *>(base + lay.match);
    c.ce = reinterpret_cast<int *>(base + lay.ce);
    c.cp = reinterpret_cast<int *>(base + lay.cp);
    // coarse node weights: this block's slice of the coarse nodes
    {
        const int lo = slice_lo(Nc, r, C), hi = slice_lo(Nc, r + 1, C);
        for (int x = lo + (int)threadIdx.x; x < hi; x += kTT) c_nw[x] = s_cw[x];
    }
    // this block's staged hyperedges and pins into place; the coarse level's chunk table
    {
        const int ne = (int)run_e, np = (int)run_p;
        for (int i0 = 8 * (int)threadIdx.x; i0 < np; i0 += 8 * kTT) {
            int x[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = i0 + k < np ? __ldcg(stage_p + pa_r + i0 + k) : 0;
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (i0 + k < np) c_pins[Pb + i0 + k] = x[k];
        }
        for (int i0 = 8 * (int)threadIdx.x; i0 < ne; i0 += 8 * kTT) {
            int o[9], wv[8];
#pragma unroll
            for (int k = 0; k < 9; ++k) o[k] = i0 + k < ne ? __ldcg(a.e_soff + ea + i0 + k) : np;
#pragma unroll
            for (int k = 0; k < 8; ++k) wv[k] = (c_hw && i0 + k < ne) ? __ldcg(a.e_shw + ea + i0 + k) : 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if (i0 + k >= ne) break;
                const int e = (int)Eb + i0 + k;
                const int og = (int)Pb + o[k];
                c_hoff[e] = og;
                if (c_hw) c_hw[e] = wv[k];
                mark_chunks(c.ce, c.cp, e, og, o[k + 1] - o[k]);
            }
        }
        if (r == 0 && threadIdx.x == 0) {
            c_hoff[c.E] = c.P;
            c.ce[0] = 0;
            c.cp[0] = 0;
            c.ce[c.K] = c.E;
            c.cp[c.K] = c.P;
        }
    }
    trace(a, lv, 8);
    csync();
    return true;
}

// ------------------------------------------------------------------------------ refinement
// A pass of per-hyperedge contributions into the partial array gp, then the reduce-scatter: the
// block's slice gets the sum over all blocks (minus the slice's weighted degrees when ds_sub);
// with `all`, every block then gathers the other slices.
struct Refine {
    int *gp, *gf, *ds, *wl, *cnt;
};

template <class One, class Wide>
__device__ void refine_pass(const TailArgs &a, const TLev &L, const Chunks &ch, char *smem,
                            const Refine &R, int *out, bool sub_ds, bool all, int lv, One one,
                            Wide wide) {
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks(), r = (int)cl.block_rank();
    const int N = L.N;
    trace(a, lv, 20);
    for (int v = threadIdx.x; v < N; v += kTT) R.gp[v] = 0;
    __syncthreads();
    stream(L, ch, smem, [&](const Win &w) { win_hedges(w, R.wl, R.cnt, [&](int e, int b, int d) { one(w, e, b, d); },
                                                       [&](int e, int b, int d) { wide(w, e, b, d); }); });
    trace(a, lv, 21);
    csync();
    trace(a, lv, 22);
    const int nlo = slice_lo(N, r, C), nhi = slice_lo(N, r + 1, C);
    for (int v = nlo + (int)threadIdx.x; v < nhi; v += kTT) {
        int x[kTailMaxCluster];
#pragma unroll
        for (int q = 0; q < kTailMaxCluster; ++q) x[q] = q < C ? remote(R.gp, q)[v] : 0;
        int s = 0;
#pragma unroll
        for (int q = 0; q < kTailMaxCluster; ++q) s += x[q];
        out[v - (all ? 0 : nlo)] = sub_ds ? s - R.ds[v - nlo] : s;
    }
    csync();
    trace(a, lv, 23);
    if (all) {
        // the other blocks' slices, eight loads in flight per thread
        for (int v0 = threadIdx.x; v0 < N; v0 += 8 * kTT) {
            int x[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int v = v0 + k * kTT;
                x[k] = 0;
                if (v < N && (v < nlo || v >= nhi)) x[k] = remote(out, slice_of(N, v, C))[v];
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int v = v0 + k * kTT;
                if (v < N && (v < nlo || v >= nhi)) out[v] = x[k];
            }
        }
    }
    __syncthreads();
    trace(a, lv, 24);
}

// Weighted degrees of the block's slice of level L's nodes into R.ds.
__device__ void tail_degrees(const TailArgs &a, const TLev &L, const Chunks &ch, char *smem, const Refine &R,
                             int lv) {
    refine_pass(a, L, ch, smem, R, R.ds, false, false, lv,
                [&](const Win &w, int e, int b0, int d) {
                    const int wt = L.hw ? __ldg(L.hw + e) : 1;
                    for (int i = 0; i < d; ++i) atomicAdd(&R.gp[w.P[b0 + i]], wt);
                },
                [&](const Win &w, int e, int b0, int d) {
                    const int wt = L.hw ? __ldg(L.hw + e) : 1;
                    for (int i = threadIdx.x & 31; i < d; i += 32) atomicAdd(&R.gp[w.P[b0 + i]], wt);
                });
    // the partial array is reused by the next pass once every block has read it
    csync();
}

// Algorithm 4 gains of every node of level L for `side` (shared, identical in every block) into
// R.gf in every block.
__device__ void tail_gains(const TailArgs &a, const TLev &L, const Chunks &ch, char *smem, const Refine &R,
                           const uint8_t *side, int lv) {
    refine_pass(a, L, ch, smem, R, R.gf, true, true, lv,
                [&](const Win &w, int e, int b0, int d) {
                    int n1 = 0;
                    for (int i = 0; i < d; ++i) n1 += side[w.P[b0 + i]];
                    if (n1 == 0 || n1 == d) return;  // uncut: only -w_e, already in -D
                    const int wt = L.hw ? __ldg(L.hw + e) : 1;
                    for (int i = 0; i < d; ++i) {
                        const int u = w.P[b0 + i];
                        const int ns = side[u] ? n1 : d - n1;  // pins on u's side
                        atomicAdd(&R.gp[u], ns == 1 ? 2 * wt : wt);
                    }
                },
                [&](const Win &w, int e, int b0, int d) {
                    const int lane = threadIdx.x & 31;
                    int n1 = 0;
                    for (int i = lane; i < d; i += 32) n1 += side[w.P[b0 + i]];
                    n1 = warp_sum(n1);
                    if (n1 == 0 || n1 == d) return;
                    const int wt = L.hw ? __ldg(L.hw + e) : 1;
                    for (int i = lane; i < d; i += 32) {
                        const int u = w.P[b0 + i];
                        const int ns = side[u] ? n1 : d - n1;
                        atomicAdd(&R.gp[u], ns == 1 ? 2 * wt : wt);
                    }
                });
}

__device__ void tail_side_weights(const TLev &L, const uint8_t *side, RState *st) {
    __shared__ unsigned long long red[33];
    unsigned long long w0 = 0, w1 = 0;
    for (int v = threadIdx.x; v < L.N; v += kTT) {
        const unsigned long long w = (unsigned long long)__ldg(L.nw + v);
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

}  // namespace

__global__ void __launch_bounds__(kTT, 1) k_tail(TailArgs a) {
    extern __shared__ __align__(16) char smem[];
    __shared__ TLev lev[kTailMaxLevels + 1];
    __shared__ int s_ce[kTailMaxChunks + 2], s_cp[kTailMaxChunks + 2];
    __shared__ int s_cnt[2];
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks(), r = (int)cl.block_rank();
    // the starting level and its chunk table
    if (threadIdx.x == 0) {
        TLev &L = lev[0];
        L.N = a.N;
        L.E = a.E;
        L.P = a.P;
        L.K = tail_chunks(a.P);
        L.hoff = a.hoff;
        L.pins = a.pins;
        L.hw = a.hw;
        L.nw = a.nw;
        L.cmap = a.cmap;
        L.match = a.match;
        L.ce = a.ce0;
        L.cp = a.cp0;
    }
    __syncthreads();
    build_chunks(lev[0], r, C);
    csync();
    // coarsening (Sec. 3.4 stop rule, reading C11)
    size_t top = 0, need = 0;
    bool overflow = false;
    int nl = 0;  // coarse levels built
    // algorithmic bytes of the launch (each array streamed once, gathers at element size; the
    // shared-memory traffic is not counted), kept by every thread alike
    double bytes = 4.0 * a.E;  // the chunk table of the starting level
    while (nl < a.max_new && lev[nl].E > 0) {
        TLev c;
        const TLev &f = lev[nl];
        if (!tail_coarsen(a, f, c, &top, &need, nl, smem, s_ce, s_cp)) {
            overflow = true;
            break;
        }
        // keys and matching: hoff, pins, clears; set sizes, groups, coarse ids; contraction:
        // hoff, pins, staged pins out and back, the coarse CSR and its chunk table
        bytes += 24.0 * f.E + 8.0 * f.P + 24.0 * f.N + 12.0 * c.P + 16.0 * c.E + 4.0 * c.N +
                 (f.hw ? 4.0 * (f.E + 2.0 * c.E) : 0.0);
        if (c.N == f.N) break;  // nothing merged (cannot happen with E > 0; kept for C11)
        __syncthreads();
        if (threadIdx.x == 0) lev[nl + 1] = c;
        __syncthreads();
        ++nl;
    }
    if (r == 0 && threadIdx.x == 0) {
        for (int j = 0; j < a.max_new; ++j) {
            a.sizes[3 * j] = j < nl ? lev[j + 1].N : 0;
            a.sizes[3 * j + 1] = j < nl ? lev[j + 1].E : 0;
            a.sizes[3 * j + 2] = j < nl ? lev[j + 1].P : 0;
        }
        a.info[0] = nl;
        a.info[1] = overflow ? (int)((need + 1048575) >> 20) : 0;  // MiB needed
    }
    auto pass_bytes = [&](const TLev &L) { return 4.0 * L.E + 4.0 * L.P + (L.hw ? 4.0 * L.E : 0.0) + 8.0 * L.N; };
    // refinement view of the shared memory (every coarsening access is behind the last barrier)
    Refine R;
    R.gp = reinterpret_cast<int *>(smem + kGP);
    R.gf = reinterpret_cast<int *>(smem + kGF);
    R.ds = reinterpret_cast<int *>(smem + kDS);
    R.wl = reinterpret_cast<int *>(smem + kWL);
    R.cnt = &s_cnt[0];
    uint8_t *sides[2] = {reinterpret_cast<uint8_t *>(smem + kSA), reinterpret_cast<uint8_t *>(smem + kSB)};
    signed char *s_grp = reinterpret_cast<signed char *>(smem + kGR);
    RState *st = reinterpret_cast<RState *>(smem + kST);
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(smem + kKY);
    int *list = reinterpret_cast<int *>(smem + kLS);
    int cur = 0;
    __syncthreads();
    // Algorithm 5 and the rebalance from the coarsest level (after Algorithm 3 there) up to the
    // starting level
    for (int l = nl; l >= 0; --l) {
        const TLev &L = lev[l];
        Chunks ch;
        load_chunks(L, r, C, ch, s_ce, s_cp);
        tail_degrees(a, L, ch, smem, R, l);
        bytes += pass_bytes(L);
        const long long sq = d_ceil_sqrt(L.N);
        if (l == nl) {
            // Algorithm 3 (side 0 grown to its share m0 / m, reading G2)
            uint8_t *side = sides[cur];
            for (int v = threadIdx.x; v < L.N; v += kTT) side[v] = 1;
            if (threadIdx.x == 0) {
                st->rounds = 0;
                st->list_count = 0;
                st->moved_count = 0;
                st->slow = 0;
            }
            __syncthreads();
            tail_side_weights(L, side, st);
            d_initial_cond(st, (long long)L.N + 1, a.status, true, a.m0, a.m);
            __syncthreads();
            while (st->flag) {
                tail_gains(a, L, ch, smem, R, side, l);
                bytes += pass_bytes(L);
                d_sel_small(L.N, SEL_INITIAL, sq, R.gf, side, L.nw, st, a.status, nullptr, nullptr, R.gf,
                            s_grp, st->hist);
                __syncthreads();
                d_initial_cond(st, (long long)L.N + 1, a.status, false, a.m0, a.m);
                __syncthreads();
            }
        } else {
            // projection of the coarser level's sides
            const uint8_t *coarse = sides[cur];
            uint8_t *fine = sides[cur ^ 1];
            for (int v0 = threadIdx.x; v0 < L.N; v0 += 4 * kTT) {
                int cm[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) cm[k] = v0 + k * kTT < L.N ? __ldcg(L.cmap + v0 + k * kTT) : 0;
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (v0 + k * kTT < L.N) fine[v0 + k * kTT] = coarse[cm[k]];
            }
            bytes += 4.0 * L.N;
            cur ^= 1;
            __syncthreads();
        }
        uint8_t *side = sides[cur];
        for (int it = 0; it < a.iters; ++it) {
            tail_gains(a, L, ch, smem, R, side, l);
            bytes += pass_bytes(L);
            d_sel_small(L.N, SEL_REFINE, 0, R.gf, side, L.nw, st, a.status, nullptr, nullptr, R.gf, s_grp,
                        st->hist);
            __syncthreads();
            trace(a, l, 30);
        }
        tail_side_weights(L, side, st);
        d_rebal_cond(st, a.limit0, a.limit1, (long long)L.N + 1, a.status, true);
        __syncthreads();
        while (st->flag) {
            tail_gains(a, L, ch, smem, R, side, l);
            bytes += pass_bytes(L);
            d_sel_small(L.N, SEL_REBAL, sq, R.gf, side, L.nw, st, a.status, list, nullptr, R.gf, s_grp,
                        st->hist);
            __syncthreads();
            d_rebal_move(R.gf, side, L.nw, list, st, sq, keys);
            __syncthreads();
            trace(a, l, 31);
            d_rebal_cond(st, a.limit0, a.limit1, (long long)L.N + 1, a.status, false);
            __syncthreads();
        }
    }
    if (r == 0) {
        const uint8_t *side = sides[cur];
        for (int v = threadIdx.x; v < a.N; v += kTT) a.side_out[v] = side[v];
        if (threadIdx.x == 0) {
            a.gst->warn = st->warn;
            a.info[2] = (int)((bytes + a.N) / 1024.0);  // KiB, with the side written
        }
    }
    // no block leaves while another may still read its shared memory
    csync();
}

// ------------------------------------------------------------------ host side
namespace {
std::once_flag g_tail_once;
int g_tail_cluster = 0;      // blocks per cluster (0: the tail is not used)
int g_tail_nodes = kTailNodes;
int64_t g_tail_pins = kTailStartPins;
}  // namespace

int tail_cluster() {
    std::call_once(g_tail_once, []() {
        if (const char *env = std::getenv("BIPART_TAIL_NODES")) g_tail_nodes = std::min(std::atoi(env), kTailNodes);
        if (const char *env = std::getenv("BIPART_TAIL_PINS")) g_tail_pins = std::min<int64_t>(std::atoll(env), kTailMaxPins);
        if (g_tail_nodes <= 0) return;
        if (cudaFuncSetAttribute(k_tail, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes) != cudaSuccess ||
            cudaFuncSetAttribute(k_tail, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        for (int c : {16, 8, 4}) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(c);
            cfg.blockDim = dim3(kTT);
            cfg.dynamicSmemBytes = kSmemBytes;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = c;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int n = 0;
            if (cudaOccupancyMaxActiveClusters(&n, k_tail, &cfg) == cudaSuccess && n >= 1) {
                g_tail_cluster = c;
                break;
            }
            cudaGetLastError();
        }
    });
    return g_tail_cluster;
}

bool tail_eligible(const Level &L, int max_new, int flags) {
    const int C = tail_cluster();  // first: it also reads the limits' overrides
    if (C <= 0) return false;
    if (flags & BIPART_FLAG_MERGE_PARALLEL) return false;  // the tail runs the paper's contraction
    if (max_new > kTailMaxLevels || L.N < 1) return false;
    if (L.N > g_tail_nodes || (int64_t)L.P > g_tail_pins) return false;
    // every block's share of the chunk table fits its shared-memory copy
    return (tail_chunks(L.P) + C - 1) / C + 1 <= kTailMaxChunks;
}

void run_tail(bipart_graph *g, std::vector<Level *> &levels, const Params &p, const int64_t limit[2],
              uint8_t *d_side) {
    cudaStream_t s = g->stream;
    Work &w = g->w;
    Level &f = *levels.back();
    const int sidx = (int)levels.size() - 1;
    const int max_new = p.levels - sidx;
    const int C = tail_cluster();
    const bool weighted = f.hw() != nullptr;
    const int E1 = std::max(f.E, 1), P1 = std::max(f.P, 1), N1 = std::max(f.N, 1);
    TailArgs a{};
    a.N = f.N;
    a.E = f.E;
    a.P = f.P;
    a.hoff = f.hoff();
    a.pins = f.pins();
    a.hw = f.hw();
    a.nw = f.nw();
    f.b_cmap.ensure(sizeof(int) * (size_t)N1, s);
    f.b_match.ensure(sizeof(int) * (size_t)N1, s);
    a.cmap = f.cmap();
    a.match = f.match();
    a.policy = p.policy;
    a.max_new = max_new;
    a.iters = p.iters;
    a.m0 = p.m0;
    a.m = p.m;
    a.limit0 = limit[0];
    a.limit1 = limit[1];
    a.e_ssize = (int *)w.t_e0.ensure(sizeof(int) * (size_t)E1, s);
    a.e_sweight = (int *)w.t_e1.ensure(sizeof(int) * (size_t)E1, s);
    a.e_rep = (unsigned *)w.t_e2.ensure(sizeof(int) * (size_t)E1, s);
    a.e_soff = (int *)w.t_e3.ensure(sizeof(int) * (size_t)E1, s);
    a.e_shw = (int *)w.t_e4.ensure(sizeof(int) * (size_t)E1, s);
    a.p_stage = (int *)w.t_p.ensure(sizeof(int) * 2 * (size_t)P1, s);
    a.n_grp = (int *)w.t_n.ensure(sizeof(int) * (size_t)N1, s);
    const size_t k1 = (size_t)tail_chunks(f.P) + 1;
    a.ce0 = (int *)w.t_c.ensure(sizeof(int) * 2 * k1, s);
    a.cp0 = a.ce0 + k1;
    a.xchg = (long long *)w.t_x.ensure(sizeof(long long) * 2 * kTailMaxCluster, s);
    a.sizes = level_sizes(g, sidx);
    a.info = tail_info_slot(g);
    a.side_out = d_side;
    a.gst = refine_state(g);
    a.status = dev_status(g);
    static const bool tracing = std::getenv("BIPART_TAIL_TRACE") != nullptr;
    a.trace = nullptr;
    if (tracing && !g->ex.capturing) {
        a.trace = (unsigned long long *)w.t_trace.ensure(sizeof(unsigned long long) * (1 + 2 * kTailTraceMax), s);
        BP_CUDA(cudaMemsetAsync(a.trace, 0, sizeof(unsigned long long), s));
    }
    // arena: a few times the starting level at first, grown when a run reports it too small
    const size_t first = tail_layout(0, f.N, f.E, f.P, weighted).end;
    w.t_arena.ensure(std::min<size_t>((size_t)std::max(max_new, 1), 3) * first + (1 << 20), s);
    for (int attempt = 0;; ++attempt) {
        a.arena = w.t_arena.as<char>();
        a.arena_cap = w.t_arena.cap;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(C);
        cfg.blockDim = dim3(kTT);
        cfg.dynamicSmemBytes = kSmemBytes;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = C;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        ProfScope ps("tail", 0.0, s);
        BP_CUDA(cudaLaunchKernelEx(&cfg, k_tail, a));
        BP_LAUNCH();
        ps.end();
        // the new levels' sizes, their count, the arena check and the launch's algorithmic
        // bytes in one round trip
        const int nv = 3 * max_new + 3;
        std::vector<const int32_t *> ptrs((size_t)nv);
        for (int j = 0; j < 3 * max_new; ++j) ptrs[(size_t)j] = a.sizes + j;
        for (int j = 0; j < 3; ++j) ptrs[(size_t)3 * max_new + j] = a.info + j;
        std::vector<int32_t> v((size_t)nv);
        read_i32s(g, nv, ptrs.data(), v.data());
        const int nl = v[(size_t)3 * max_new];
        const int need_mb = v[(size_t)3 * max_new + 1];
        ps.set_bytes(1024.0 * v[(size_t)3 * max_new + 2]);
        if (a.trace) {
            // diagnostics: time between consecutive stamps, summed per (level, phase), on stderr
            std::vector<unsigned long long> tr(1 + 2 * kTailTraceMax);
            BP_CUDA(cudaMemcpyAsync(tr.data(), a.trace, sizeof(unsigned long long) * tr.size(), cudaMemcpyDeviceToHost, s));
            BP_CUDA(cudaStreamSynchronize(s));
            const int n = (int)std::min<unsigned long long>(tr[0], kTailTraceMax);
            std::vector<std::pair<unsigned long long, double>> acc;
            for (int i = 1; i < n; ++i) {
                const unsigned long long tag = tr[1 + 2 * i];
                const double dt = (double)(tr[2 + 2 * i] - tr[2 * i]) / 1000.0;
                auto it = std::find_if(acc.begin(), acc.end(), [&](auto &x) { return x.first == tag; });
                if (it == acc.end()) acc.emplace_back(tag, dt);
                else it->second += dt;
            }
            double tot = n > 1 ? (double)(tr[2 * n] - tr[2]) / 1000.0 : 0.0;
            std::fprintf(stderr, "[bipart] tail trace: cluster %d, %d stamps, %.1f us\n", C, n, tot);
            for (auto &x : acc)
                std::fprintf(stderr, "[bipart]   level %llu phase %llu: %.1f us\n", x.first >> 8, x.first & 255, x.second);
        }
        if (need_mb > 0) {
            if (g->ex.capturing || attempt > 8) throw Fail{BIPART_ERR_OOM, "tail arena too small"};
            w.t_arena.ensure(std::max<size_t>(2 * w.t_arena.cap, ((size_t)need_mb << 20) * 2), s);
            continue;
        }
        // the new levels as views into the arena (the same layout the kernel used)
        size_t top = 0;
        for (int j = 0; j < nl; ++j) {
            const int idx = sidx + j;
            if ((int)g->lev.size() <= idx) g->lev.emplace_back(new Level);
            Level &c = *g->lev[(size_t)idx];
            const int N = v[(size_t)3 * j], E = v[(size_t)3 * j + 1], P = v[(size_t)3 * j + 2];
            const TailLayout lay = tail_layout(top, N, E, P, weighted);
            top = lay.end;
            char *base = w.t_arena.as<char>();
            c.set_view(N, E, P, reinterpret_cast<int *>(base + lay.hoff), reinterpret_cast<int *>(base + lay.pins),
                       weighted ? reinterpret_cast<int *>(base + lay.hw) : nullptr,
                       reinterpret_cast<int *>(base + lay.nw), reinterpret_cast<int *>(base + lay.cmap),
                       reinterpret_cast<int *>(base + lay.match));
            levels.push_back(&c);
        }
        break;
    }
}

}  // namespace bp
