// Device side of initial partitioning and refinement (Sec. 3.2-3.3: Algorithms 3, 4 and 5 and
// the rebalancing pass), written once for any team of threads (see coarsen_dev.cuh).  Functions
// marked "one block" are run by a single block: a grid launch of one block, or the persistent
// block of an instance.
#pragma once

#include <climits>

#include <cooperative_groups.h>

#include "common.cuh"
#include "lb.cuh"

namespace bp {

constexpr int kHistBits = 11;
constexpr int kHistBins = 1 << kHistBits;
constexpr int kClampLo = -1024;          // fast-path buckets: gains -1023 .. 1022 are exact
constexpr int kRebalMax = 16384;         // largest ceil(sqrt n) handled by the ordered rebalance

enum SelKind : int { SEL_REFINE = 0, SEL_INITIAL = 1, SEL_REBAL = 2 };

// Selection state of one group (one side).  mode: 0 select none, 1 select all candidates,
// 2 threshold known (thr, take_eq), 3 exact radix select in progress over keys in [base, top).
struct SelGroup {
    unsigned cnt, K, thr, take_eq, mode;
    unsigned base, shift, need;
    unsigned long long top;
};

// All device-side state of refinement, resident in the handle's small scratch.
struct RState {
    SelGroup g[2];
    unsigned hist[2][kHistBins];
    unsigned long long W[2];   // side weights
    long long limit[2], room, need;  // per-side limits of the current rebalance
    int heavy;                 // rebalance: heavy side or -1
    unsigned list_count;       // rebalance: selected nodes
    unsigned flag;             // loop-continue flag
    unsigned slow;             // exact radix path needed by the current selection
    unsigned warn;             // rebalance ran out of candidates
    unsigned rounds;           // loop guard
    unsigned status0;          // warn of the level-0 rebalance
    unsigned arrived;          // blocks that finished a fused grid phase (zero at rest)
    unsigned moved_count;      // nodes moved by the current selection (reset by each selection)
    unsigned long long Wacc[2];  // side-weight partial sums of a grid launch (zero at rest)
};

__device__ __forceinline__ unsigned gkey(int gain) { return (unsigned)gain ^ 0x80000000u; }

// Candidate group of node v for a selection (-1: not a candidate).
__device__ __forceinline__ int sel_group(int kind, const RState *st, int gain, uint8_t side, int w) {
    if (kind == SEL_REFINE) return gain >= 0 ? (int)side : -1;
    if (kind == SEL_INITIAL) return side == 1 ? 1 : -1;
    return (side == st->heavy && (long long)w <= st->room) ? st->heavy : -1;
}

// ------------------------------------------------------------------------ Algorithm 4
// n1[e] = number of pins of e on side 1 (load-balanced over pins, integer atomics).
template <class Team>
__device__ void d_hedge_n1(Team t, int E, int P, const int *hoff, const int *pins,
                           const uint8_t *side, int *n1, const int *ts = nullptr) {
    lb_for_each_items<int>(
        hoff, E, P, pins, 0,
        [&](int, int u, int acc) { return acc + Team::ld(side + u); },
        [&](int e, int acc) {
            if (acc) atomicAdd(n1 + e, acc);
        },
        t, ts);
}

// Contribution of e to a pin on side i: +w if n_i == 1 (moving it uncuts e), -w if n_i == |e|
// (moving it cuts e), else 0.
// With `reset`, n1[e] is put back to zero once read (the grid path keeps n1 zero at rest).
template <class Team>
__device__ void d_hedge_contrib(Team t, int E, const int *hoff, const int *hw, int *n1,
                                int2 *hc, bool reset = false) {
    for (int e = t.rank(); e < E; e += t.size()) {
        int d = Team::ld(hoff + e + 1) - Team::ld(hoff + e), a1 = Team::ld(n1 + e), a0 = d - a1;
        if (reset) n1[e] = 0;
        int w = hw ? Team::ld(hw + e) : 1;
        int c0 = a0 == 1 ? w : (a0 == d ? -w : 0);
        int c1 = a1 == 1 ? w : (a1 == d ? -w : 0);
        hc[e] = make_int2(c0, c1);
    }
}

// gain[v] = sum over v's hyperedges of the contribution for v's side (gain zeroed first).
template <class Team>
// With `warp_sum` the last runs of a warp's lanes are summed per node before the atomic (levels
// whose nodes have long incidence lists, where many threads would hit one node).
__device__ void d_node_gain(Team t, int N, int P, const int *noff, const int *nadj, const int2 *hc,
                            const uint8_t *side, int *gain, const int *ts = nullptr,
                            bool warp_sum = true) {
    auto visit = [&](int v, int e, int acc) {
        int2 c = Team::ld(hc + e);
        return acc + (Team::ld(side + v) ? c.y : c.x);
    };
    auto flush = [&](int v, int acc) {
        if (acc) atomicAdd(gain + v, acc);
    };
    if (warp_sum)
        lb_reduce_items<int>(noff, N, P, nadj, 0, cooperative_groups::plus<int>(), visit, flush, t, ts);
    else
        lb_for_each_items<int>(noff, N, P, nadj, 0, visit, flush, t, ts);
}

// The same gains with each hyperedge's contribution formed on the spot from its degree, its
// side-1 count and its weight (no separate contribution pass).
template <class Team>
__device__ void d_node_gain_direct(Team t, int N, int P, const int *noff, const int *nadj,
                                   const int *hoff, const int *hw, const int *n1,
                                   const uint8_t *side, int *gain, const int *ts = nullptr,
                                   bool warp_sum = true) {
    auto visit = [&](int v, int e, int acc) {
        const int d = Team::ld(hoff + e + 1) - Team::ld(hoff + e);
        const int a1 = Team::ld(n1 + e);
        const int w = hw ? Team::ld(hw + e) : 1;
        const int a = Team::ld(side + v) ? a1 : d - a1;  // pins on v's side
        return acc + (a == 1 ? w : (a == d ? -w : 0));
    };
    auto flush = [&](int v, int acc) {
        if (acc) atomicAdd(gain + v, acc);
    };
    if (warp_sum)
        lb_reduce_items<int>(noff, N, P, nadj, 0, cooperative_groups::plus<int>(), visit, flush, t, ts);
    else
        lb_for_each_items<int>(noff, N, P, nadj, 0, visit, flush, t, ts);
}

// ------------------------------------------------------------------------ selection
// Grid-stride loop over the team's nodes that loads gain, side and weight of four nodes (one per
// stride) before visiting any of them (fn(v, gain, side, weight)): the visits update
// shared-memory counters, and without the batching every node's loads would wait for the
// previous node's update.
template <class Team, class Fn>
__device__ __forceinline__ void sel_nodes(Team t, int N, const int *gain, const uint8_t *side,
                                          const int *nw, Fn fn) {
    const int64_t stride = t.size();
    for (int64_t v0 = t.rank(); v0 < N; v0 += 4 * stride) {
        int g[4], w[4];
        uint8_t sd[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t v = v0 + u * stride;
            if (v < N) {
                g[u] = gain[v];
                sd[u] = side[v];
                w[u] = nw[v];
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (v0 + u * stride < N) fn(v0 + u * stride, g[u], sd[u], w[u]);
    }
}

// Fast pass: histogram of clamped gains per group (h: 2 * kHistBins shared counters), added into
// the grid's histogram st->hist.
template <class Team>
__device__ void d_sel_hist(Team t, int N, int kind, const int *gain, const uint8_t *side,
                           const int *nw, RState *st, unsigned (*h)[kHistBins]) {
    for (int i = threadIdx.x; i < 2 * kHistBins; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    sel_nodes(t, N, gain, side, nw, [&](int64_t, int g, uint8_t sd, int w) {
        const int grp = sel_group(kind, st, g, sd, w);
        if (grp < 0) return;
        int b = g - kClampLo;
        b = b < 0 ? 0 : (b > kHistBins - 1 ? kHistBins - 1 : b);
        atomicAdd(&h[grp][b], 1u);
    });
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * kHistBins; i += blockDim.x) {
        unsigned c = (&h[0][0])[i];
        if (c) atomicAdd(&(&st->hist[0][0])[i], c);
    }
}

// Suffix scan of one group's histogram (descending buckets) by one block of 256, 512 or 1024
// threads: returns the bucket holding the need-th largest key (-1 if need is 0 or exceeds the
// total), with *above = keys in buckets above it and *total_out = all keys of the group.
__device__ inline int hist_find(const unsigned *hist, unsigned need, unsigned *above,
                                unsigned *total_out) {
    __shared__ unsigned red[33];
    __shared__ int s_b;
    __shared__ unsigned s_above;
    const int per = kHistBins / blockDim.x;
    unsigned loc[8], tsum = 0;  // per <= 8; fixed indices keep them in registers
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        int b = kHistBins - 1 - (threadIdx.x * per + q);
        loc[q] = q < per ? hist[b] : 0u;
        tsum += loc[q];
    }
    unsigned total;
    unsigned run = block_exclusive_scan<unsigned>(tsum, red, &total);
    if (threadIdx.x == 0) { s_b = -1; s_above = 0; }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        if (q >= per) break;
        int b = kHistBins - 1 - (threadIdx.x * per + q);
        if (need > 0 && run < need && run + loc[q] >= need) {
            s_b = b;
            s_above = run;
        }
        run += loc[q];
    }
    __syncthreads();
    int b = s_b;
    *above = s_above;
    *total_out = total;
    __syncthreads();
    return b;
}

// One block: decides K per group from the fast histogram and fixes the threshold, or starts the
// exact path (st->slow).  Both groups are searched in one suffix scan over the buckets: the two
// 32-bit counts travel packed in one 64-bit value (a count never exceeds N < 2^31, so the fields
// never carry), the scan's total gives both group sizes and so K, and each thread then checks
// its buckets against both needs.
__device__ inline void d_sel_find(int kind, long long s, RState *st, const unsigned (*hist)[kHistBins]) {
    __shared__ unsigned long long red[33];
    __shared__ int s_b[2];
    __shared__ unsigned s_above[2];
    const int per = kHistBins / blockDim.x;  // 256, 512 or 1024 threads
    unsigned l0[8], l1[8];  // per <= 8; fixed indices keep them in registers
    unsigned long long tsum = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int b = kHistBins - 1 - (threadIdx.x * per + q);
        l0[q] = q < per ? hist[0][b] : 0u;
        l1[q] = q < per ? hist[1][b] : 0u;
        tsum += (unsigned long long)l1[q] << 32 | l0[q];
    }
    unsigned long long tot;
    unsigned long long run = block_exclusive_scan<unsigned long long>(tsum, red, &tot);
    const unsigned cnt[2] = {(unsigned)tot, (unsigned)(tot >> 32)};
    unsigned K[2] = {0, 0};
    if (kind == SEL_REFINE) {
        K[0] = K[1] = min(cnt[0], cnt[1]);
    } else {
        int grp = kind == SEL_INITIAL ? 1 : st->heavy;
        if (grp >= 0) K[grp] = (unsigned)min((long long)cnt[grp], s);
    }
    // bucket search only where 0 < K < cnt (else every candidate or none is taken)
    const unsigned need0 = K[0] > 0 && K[0] < cnt[0] ? K[0] : 0u;
    const unsigned need1 = K[1] > 0 && K[1] < cnt[1] ? K[1] : 0u;
    if (threadIdx.x < 2) {
        s_b[threadIdx.x] = -1;
        s_above[threadIdx.x] = 0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        if (q >= per) break;
        const int b = kHistBins - 1 - (threadIdx.x * per + q);
        const unsigned r0 = (unsigned)run, r1 = (unsigned)(run >> 32);
        if (need0 > 0 && r0 < need0 && r0 + l0[q] >= need0) {
            s_b[0] = b;
            s_above[0] = r0;
        }
        if (need1 > 0 && r1 < need1 && r1 + l1[q] >= need1) {
            s_b[1] = b;
            s_above[1] = r1;
        }
        run += (unsigned long long)l1[q] << 32 | l0[q];
    }
    __syncthreads();
    unsigned slow = 0;
    for (int i = 0; i < 2; ++i) {
        SelGroup &G = st->g[i];
        const int b = s_b[i];
        const unsigned above = s_above[i];
        if (threadIdx.x == 0) {
            G.cnt = cnt[i];
            G.K = K[i];
            if (K[i] == 0) {
                G.mode = 0;
            } else if (K[i] >= cnt[i]) {
                G.mode = 1;
            } else if (b > 0 && b < kHistBins - 1) {
                G.mode = 2;
                G.thr = gkey(b + kClampLo);
                G.take_eq = K[i] - above;
            } else {
                // the threshold lies in a clamped end bucket: exact radix select over its keys
                G.mode = 3;
                G.need = K[i] - above;
                if (b == kHistBins - 1) {
                    G.base = gkey(kHistBins - 1 + kClampLo);
                    G.top = 1ull << 32;
                } else {
                    G.base = 0;
                    G.top = (unsigned long long)gkey(kClampLo) + 1ull;
                }
                unsigned long long range = G.top - G.base;  // >= 1
                unsigned bits = range > 1 ? 64 - __clzll(range - 1ull) : 0;
                G.shift = bits > kHistBits ? bits - kHistBits : 0;
                slow = 1;
            }
        }
    }
    if (threadIdx.x == 0) st->slow = slow;
}

// Exact path: histogram of keys in [base, top) by (key - base) >> shift.
template <class Team>
__device__ void d_sel_hist_exact(Team t, int N, int kind, const int *gain, const uint8_t *side,
                                 const int *nw, RState *st, unsigned (*h)[kHistBins],
                                 bool flush = true) {
    __shared__ unsigned s_base[2], s_shift[2], s_on[2];
    __shared__ unsigned long long s_top[2];
    if (threadIdx.x < 2) {
        s_on[threadIdx.x] = st->g[threadIdx.x].mode == 3;
        s_base[threadIdx.x] = st->g[threadIdx.x].base;
        s_shift[threadIdx.x] = st->g[threadIdx.x].shift;
        s_top[threadIdx.x] = st->g[threadIdx.x].top;
    }
    for (int i = threadIdx.x; i < 2 * kHistBins; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    if (!s_on[0] && !s_on[1]) return;
    sel_nodes(t, N, gain, side, nw, [&](int64_t, int g, uint8_t sd, int w) {
        const int grp = sel_group(kind, st, g, sd, w);
        if (grp < 0 || !s_on[grp]) return;
        const unsigned k = gkey(g);
        if (k < s_base[grp] || (unsigned long long)k >= s_top[grp]) return;
        atomicAdd(&h[grp][(k - s_base[grp]) >> s_shift[grp]], 1u);
    });
    __syncthreads();
    if (!flush) return;
    for (int i = threadIdx.x; i < 2 * kHistBins; i += blockDim.x) {
        unsigned c = (&h[0][0])[i];
        if (c) atomicAdd(&(&st->hist[0][0])[i], c);
    }
}

// One block: narrows every group on the exact path to the next digit, or fixes its threshold.
__device__ inline void d_sel_find_exact(RState *st, uint32_t *status, const unsigned (*hist)[kHistBins]) {
    for (int i = 0; i < 2; ++i) {
        SelGroup &G = st->g[i];
        const unsigned mode = G.mode;
        __syncthreads();
        if (mode != 3) continue;  // block-uniform
        unsigned above = 0, total = 0;
        int b = hist_find(hist[i], G.need, &above, &total);
        if (threadIdx.x == 0) {
            if (b < 0) {
                G.mode = 0;
                record_error(status, DEV_OVERFLOW);
            } else {
                unsigned need = G.need - above;
                G.base = G.base + ((unsigned)b << G.shift);
                // the chosen bucket, clipped to the keys still in play (the first range is not
                // a power of two wide, so a bucket may reach past it)
                const unsigned long long end = (unsigned long long)G.base + (1ull << G.shift);
                G.top = end < G.top ? end : G.top;
                if (G.shift == 0) {
                    G.thr = G.base;
                    G.take_eq = need;
                    G.mode = 2;
                } else {
                    G.need = need;
                    G.shift = G.shift > kHistBits ? G.shift - kHistBits : 0;
                }
            }
        }
        __syncthreads();
    }
}

// Tie ranks: value = (ties of group 1) << 31 | ties of group 0; a tie is a candidate whose key
// equals its group's threshold.
struct TieIn {
    int kind;
    const int *gain;
    const uint8_t *side;
    const int *nw;
    const RState *st;
    __device__ uint64_t operator()(int64_t v) const {
        int g = gain[v];
        int grp = sel_group(kind, st, g, side[v], nw[v]);
        if (grp < 0 || st->g[grp].mode != 2 || gkey(g) != st->g[grp].thr) return 0;
        return grp ? (1ull << 31) : 1ull;
    }
};

// Applies the selection to a chosen node v: refine flips it; the initial partition moves it to P0
// and keeps the side weights current; the rebalance collects it.  With `moved`, every flipped node
// is also appended there (st->moved_count; one atomic per group of converged lanes), so the
// side-1 counts can be updated instead of recounted.
__device__ __forceinline__ void d_apply_node(int kind, int64_t v, uint8_t *side, const int *nw,
                                             RState *st, int *list, int *moved) {
    if (kind == SEL_REBAL) {
        list[atomicAdd(&st->list_count, 1u)] = (int)v;
        return;
    }
    side[v] ^= 1;
    if (kind == SEL_INITIAL) {
        atomicAdd(&st->W[0], (unsigned long long)nw[v]);
        atomicAdd(&st->W[1], (unsigned long long)(-(long long)nw[v]));
    }
    if (moved) {
        namespace cg = cooperative_groups;
        const cg::coalesced_group grp = cg::coalesced_threads();
        unsigned base = 0;
        if (grp.thread_rank() == 0) base = atomicAdd(&st->moved_count, grp.size());
        base = grp.shfl(base, 0);
        moved[base + grp.thread_rank()] = (int)v;
    }
}

// The application pass of a grid selection: the tie ranks come from the scan (TieIn).
struct ApplyOut {
    int kind;
    const int *gain;
    uint8_t *side;
    const int *nw;
    RState *st;
    int *list;
    int *moved = nullptr;
    __device__ void operator()(int64_t v, uint64_t pre, uint64_t) const {
        int g = gain[v];
        int grp = sel_group(kind, st, g, side[v], nw[v]);
        if (grp < 0) return;
        const SelGroup &G = st->g[grp];
        bool sel;
        if (G.mode == 1) sel = true;
        else if (G.mode == 2) {
            unsigned k = gkey(g);
            unsigned rank = grp ? (unsigned)(pre >> 31) : (unsigned)(pre & 0x7fffffffu);
            sel = k > G.thr || (k == G.thr && rank < G.take_eq);
        } else {
            sel = false;
        }
        if (sel) d_apply_node(kind, v, side, nw, st, list, moved);
    }
};

// Adds the weights of sides 0 and 1 into acc[0], acc[1].
template <class Team>
__device__ void d_side_weights(Team t, int N, const uint8_t *side, const int *nw,
                               unsigned long long *acc) {
    unsigned long long w0 = 0, w1 = 0;
    for (int v = t.rank(); v < N; v += t.size()) {
        if (Team::ld(side + v)) w1 += Team::ld(nw + v);
        else w0 += Team::ld(nw + v);
    }
    w0 = warp_sum(w0);
    w1 = warp_sum(w1);
    if ((threadIdx.x & 31) == 0) {
        if (w0) atomicAdd(&acc[0], w0);
        if (w1) atomicAdd(&acc[1], w1);
    }
}

// Algorithm 3 loop condition: continue while P0 is below its share, m * W0 < m0 * (W0 + W1)
// (side 0 meant for m0 of m parts; m0 / m = 1 / 2 is "P0 lighter than P1").  Guarded; one
// thread acts.
__device__ inline void d_initial_cond(RState *st, long long max_rounds, uint32_t *status,
                                      bool first = false, int m0 = 1, int m = 2) {
    if (threadIdx.x != 0) return;
    if (first) st->rounds = 0;
    const long long W0 = (long long)st->W[0], W1 = (long long)st->W[1];
    unsigned f = (long long)m * W0 < (long long)m0 * (W0 + W1);
    if (f && (long long)(st->rounds++) >= max_rounds) {
        record_error(status, DEV_TIMEOUT);
        f = 0;
    }
    st->flag = f;
}

// Rebalance loop condition (reading C13): heavy side above the limit and candidates left.  One
// thread acts.
// Side s may hold up to limit_s (both equal for a halving bisection).
__device__ inline void d_rebal_cond(RState *st, long long limit0, long long limit1,
                                    long long max_rounds, uint32_t *status, bool first = false) {
    if (threadIdx.x != 0) return;
    if (first) {
        st->rounds = 0;
        st->warn = 0;
    }
    st->limit[0] = limit0;
    st->limit[1] = limit1;
    long long W0 = (long long)st->W[0], W1 = (long long)st->W[1];
    int H = W0 > limit0 ? 0 : (W1 > limit1 ? 1 : -1);
    st->heavy = H;
    unsigned f = H >= 0 && !st->warn;
    if (H >= 0) {
        long long Wh = H ? W1 : W0, Wo = H ? W0 : W1;
        st->room = (H ? limit0 : limit1) - Wo;
        st->need = Wh - (H ? limit1 : limit0);
    }
    if (f && (long long)(st->rounds++) >= max_rounds) {
        record_error(status, DEV_TIMEOUT);
        f = 0;
    }
    st->flag = f;
}

// Ordered rebalance move (one block): sort the selected nodes by (gain desc, id asc), move the
// shortest prefix whose weight reaches `need`, stopping at s nodes or before exceeding `room`.
// With nothing selected, marks the level imbalanced.  One block; keys: shared memory for the
// next power of two >= the number selected.
__device__ inline void d_rebal_move(const int *gain, uint8_t *side, const int *nw, const int *list,
                                    RState *st, long long s, unsigned long long *keys,
                                    int *moved = nullptr) {
    __shared__ long long red[33];
    __shared__ int s_cut;
    const int n = (int)st->list_count;
    if (n == 0) {
        if (threadIdx.x == 0) st->warn = 1;
        return;
    }
    const int heavy = st->heavy;
    const long long room = st->room, need = st->need;
    int S = 1;
    while (S < n) S <<= 1;
    for (int i = threadIdx.x; i < S; i += blockDim.x) {
        if (i < n) {
            int v = list[i];
            unsigned desc = ~gkey(gain[v]);  // larger gain -> smaller value
            keys[i] = ((unsigned long long)desc << 32) | (unsigned)v;
        } else {
            keys[i] = ~0ull;
        }
    }
    __syncthreads();
    for (int k = 2; k <= S; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < S; i += blockDim.x) {
                int p = i ^ j;
                if (p > i) {
                    unsigned long long x = keys[i], y = keys[p];
                    bool up = (i & k) == 0;
                    if ((x > y) == up) { keys[i] = y; keys[p] = x; }
                }
            }
            __syncthreads();
        }
    }
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int i0 = threadIdx.x * per;
    long long loc = 0;
    for (int q = 0; q < per && i0 + q < n; ++q) loc += nw[(int)(keys[i0 + q] & 0xffffffffu)];
    long long tot;
    long long run = block_exclusive_scan<long long>(loc, red, &tot);
    if (threadIdx.x == 0) s_cut = (int)min((long long)n, s);
    __syncthreads();
    for (int q = 0; q < per && i0 + q < n; ++q) {
        int i = i0 + q;
        long long w = nw[(int)(keys[i] & 0xffffffffu)];
        if (run + w > room) atomicMin(&s_cut, i);             // node i would exceed room
        else if (run + w >= need) atomicMin(&s_cut, i + 1);   // prefix [0, i] reaches need
        run += w;
    }
    __syncthreads();
    const int cut = s_cut;
    long long wmoved = 0;
    for (int i = threadIdx.x; i < cut; i += blockDim.x) {
        int v = (int)(keys[i] & 0xffffffffu);
        side[v] = (uint8_t)(1 - heavy);
        wmoved += nw[v];
        if (moved) moved[i] = v;  // the selection that collected the candidates reset the count
    }
    wmoved = block_sum(wmoved, red);
    if (threadIdx.x == 0) {
        atomicAdd(&st->W[1 - heavy], (unsigned long long)wmoved);
        atomicAdd(&st->W[heavy], (unsigned long long)(-wmoved));
        if (moved) st->moved_count = (unsigned)cut;
    }
}

// Selection of a level of at most kSelOneBlock nodes by one block, every phase after the first
// on shared memory: the clamped-gain histogram (each node's gain and group cached on the way in
// s_gain, s_grp: N entries each; s_gain may be `gain` itself when that is in shared memory), the
// threshold (and the exact radix passes when it falls in a clamped end bucket), the ranks of the
// threshold's ties by ascending id from a bitmap with per-word prefix counts, and the
// application.  h: 2 x kHistBins counters.  The rebalancing list and the moved list are emptied
// first.  Deterministic: the same inputs give the same sides in every block that runs it.
constexpr int kSelOneBlock = 16384;
constexpr int kSelSmallWords = kSelOneBlock / 32;

__device__ inline void d_sel_small(int N, int kind, long long s, const int *gain, uint8_t *side,
                                   const int *nw, RState *st, uint32_t *status, int *list,
                                   int *moved, int *s_gain, signed char *s_grp,
                                   unsigned (*h)[kHistBins]) {
    __shared__ unsigned tie[2][kSelSmallWords];
    __shared__ unsigned pre[2][kSelSmallWords];
    __shared__ unsigned long long red[33];
    __shared__ unsigned s_mode[2], s_thr[2], s_take[2];
    for (int i = threadIdx.x; i < 2 * kHistBins; i += blockDim.x) (&h[0][0])[i] = 0;
    for (int i = threadIdx.x; i < 2 * kSelSmallWords; i += blockDim.x) (&tie[0][0])[i] = 0;
    __syncthreads();
    sel_nodes(CtaTeam(), N, gain, side, nw, [&](int64_t v, int g, uint8_t sd, int w) {
        const int grp = sel_group(kind, st, g, sd, w);
        s_gain[v] = g;
        s_grp[v] = (signed char)grp;
        if (grp < 0) return;
        int b = g - kClampLo;
        b = b < 0 ? 0 : (b > kHistBins - 1 ? kHistBins - 1 : b);
        atomicAdd(&h[grp][b], 1u);
    });
    __syncthreads();
    d_sel_find(kind, s, st, h);
    if (threadIdx.x == 0) {
        st->list_count = 0;
        st->moved_count = 0;
    }
    __syncthreads();
    if (*(volatile unsigned *)&st->slow) {
        for (int pass = 0; pass < 3; ++pass) {
            d_sel_hist_exact(CtaTeam(), N, kind, gain, side, nw, st, h, false);
            d_sel_find_exact(st, status, h);
        }
        if (threadIdx.x == 0) st->slow = 0;
        __syncthreads();
    }
    if (threadIdx.x < 2) {
        s_mode[threadIdx.x] = st->g[threadIdx.x].mode;
        s_thr[threadIdx.x] = st->g[threadIdx.x].thr;
        s_take[threadIdx.x] = st->g[threadIdx.x].take_eq;
    }
    __syncthreads();
    // the threshold's ties, one bit per node
    for (int v = threadIdx.x; v < N; v += blockDim.x) {
        const int grp = s_grp[v];
        if (grp >= 0 && s_mode[grp] == 2 && gkey(s_gain[v]) == s_thr[grp])
            atomicOr(&tie[grp][v >> 5], 1u << (v & 31));
    }
    __syncthreads();
    // ties before each word, both groups in one packed scan (a count stays below 2^31)
    const int words = (N + 31) >> 5;  // <= kSelSmallWords <= blockDim.x
    const int t = threadIdx.x;
    unsigned long long c = 0;
    if (t < words) c = (unsigned long long)__popc(tie[1][t]) << 32 | (unsigned)__popc(tie[0][t]);
    unsigned long long total;
    const unsigned long long ex = block_exclusive_scan<unsigned long long>(c, red, &total);
    if (t < words) {
        pre[0][t] = (unsigned)ex;
        pre[1][t] = (unsigned)(ex >> 32);
    }
    __syncthreads();
    for (int v = threadIdx.x; v < N; v += blockDim.x) {
        const int grp = s_grp[v];
        if (grp < 0) continue;
        const unsigned mode = s_mode[grp];
        bool sel = mode == 1;
        if (mode == 2) {
            const unsigned k = gkey(s_gain[v]), thr = s_thr[grp];
            if (k > thr) {
                sel = true;
            } else if (k == thr) {
                const unsigned below = tie[grp][v >> 5] & ((1u << (v & 31)) - 1u);
                sel = pre[grp][v >> 5] + (unsigned)__popc(below) < s_take[grp];
            }
        }
        if (sel) d_apply_node(kind, v, side, nw, st, list, moved);
    }
}

template <class Team>
__device__ void d_project(Team t, int N, const int *cmap, const uint8_t *coarse, uint8_t *fine) {
    for (int v = t.rank(); v < N; v += t.size()) fine[v] = Team::ld(coarse + Team::ld(cmap + v));
}


}  // namespace bp
