// Initial partitioning and refinement on sm_103a (Sec. 3.2-3.3): Algorithm 4 move gains from
// per-hyperedge side counts, Algorithm 3 growth of P0 by the top ceil(sqrt n) gains, Algorithm 5
// swaps of the gain >= 0 lists and the rebalancing pass.
//
// Node order is always (gain descending, node id ascending).  A top-K is found without sorting:
// one histogram pass over gains clamped to [-1024, 1023] fixes the threshold gain exactly unless
// it falls in one of the two clamped end buckets, in which case an exact radix select (up to
// three 11-bit passes over the order-preserving key gain ^ 0x80000000) narrows it down; a scan
// over node ids then takes the lowest ids among nodes whose gain equals the threshold.  Only the
// rebalancing pass needs the chosen nodes in order; it sorts at most ceil(sqrt n) of them in one
// block.  The two data-dependent loops (Algorithm 3's rounds and the rebalancing rounds) are
// driven by a device-side flag, so they run unchanged inside a CUDA graph (WHILE nodes).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "lb.cuh"
#include "scan.cuh"

namespace bp {

namespace {

constexpr int kBlock = 256;
constexpr int kHistBits = 11;
constexpr int kHistBins = 1 << kHistBits;
constexpr int kClampLo = -1024;          // fast-path buckets: gains -1023 .. 1022 are exact
constexpr int kRebalMax = 16384;         // largest ceil(sqrt n) handled by the ordered rebalance

inline int grid_for(int64_t n, int per_block = kBlock, int cap = 152 * 16) {
    int64_t b = (n + per_block - 1) / per_block;
    if (b < 1) b = 1;
    return (int)std::min<int64_t>(b, cap);
}

}  // namespace

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
    long long limit, room, need;
    int heavy;                 // rebalance: heavy side or -1
    unsigned list_count;       // rebalance: selected nodes
    unsigned flag;             // loop-continue flag
    unsigned slow;             // exact radix path needed by the current selection
    unsigned warn;             // rebalance ran out of candidates
    unsigned rounds;           // loop guard
    unsigned status0;          // warn of the level-0 rebalance
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
__global__ void __launch_bounds__(kLbBlock)
k_hedge_n1(int E, int P, const int *__restrict__ hoff, const int *__restrict__ pins,
           const uint8_t *__restrict__ side, int *__restrict__ n1) {
    lb_for_each<int>(
        hoff, E, P, 0,
        [&](int, int i, int acc) { return acc + __ldg(side + __ldg(pins + i)); },
        [&](int e, int acc) {
            if (acc) atomicAdd(n1 + e, acc);
        });
}

// Contribution of e to a pin on side i: +w if n_i == 1 (moving it uncuts e), -w if n_i == |e|
// (moving it cuts e), else 0.
__global__ void k_hedge_contrib(int E, const int *__restrict__ hoff, const int *__restrict__ hw,
                                const int *__restrict__ n1, int2 *__restrict__ hc) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
        int d = hoff[e + 1] - hoff[e], a1 = n1[e], a0 = d - a1, w = hw ? hw[e] : 1;
        int c0 = a0 == 1 ? w : (a0 == d ? -w : 0);
        int c1 = a1 == 1 ? w : (a1 == d ? -w : 0);
        hc[e] = make_int2(c0, c1);
    }
}

// gain[v] = sum over v's hyperedges of the contribution for v's side (gain zeroed first).
__global__ void __launch_bounds__(kLbBlock)
k_node_gain(int N, int P, const int *__restrict__ noff, const int *__restrict__ nadj,
            const int2 *__restrict__ hc, const uint8_t *__restrict__ side, int *__restrict__ gain) {
    lb_for_each<int>(
        noff, N, P, 0,
        [&](int v, int j, int acc) {
            int2 c = __ldg(hc + __ldg(nadj + j));
            return acc + (__ldg(side + v) ? c.y : c.x);
        },
        [&](int v, int acc) {
            if (acc) atomicAdd(gain + v, acc);
        });
}

// ------------------------------------------------------------------------ selection
// Fast pass: histogram of clamped gains per group.
__global__ void __launch_bounds__(kBlock)
k_sel_hist(int N, int kind, const int *__restrict__ gain, const uint8_t *__restrict__ side,
           const int *__restrict__ nw, RState *st) {
    __shared__ unsigned h[2][kHistBins];
    for (int i = threadIdx.x; i < 2 * kHistBins; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) {
        int g = gain[v];
        int grp = sel_group(kind, st, g, side[v], nw[v]);
        if (grp < 0) continue;
        int b = g - kClampLo;
        b = b < 0 ? 0 : (b > kHistBins - 1 ? kHistBins - 1 : b);
        atomicAdd(&h[grp][b], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * kHistBins; i += blockDim.x) {
        unsigned c = (&h[0][0])[i];
        if (c) atomicAdd(&(&st->hist[0][0])[i], c);
    }
}

// Suffix scan of one group's histogram (descending buckets) by a block of 1024 threads: returns
// the bucket holding the need-th largest key (-1 if need is 0 or exceeds the total), with
// *above = keys in buckets above it and *total_out = all keys of the group.
__device__ int hist_find(const unsigned *hist, unsigned need, unsigned *above, unsigned *total_out) {
    __shared__ unsigned red[33];
    __shared__ int s_b;
    __shared__ unsigned s_above;
    constexpr int per = kHistBins / 1024;
    unsigned loc[per], tsum = 0;
    for (int q = 0; q < per; ++q) {
        int b = kHistBins - 1 - (threadIdx.x * per + q);
        loc[q] = hist[b];
        tsum += loc[q];
    }
    unsigned total;
    unsigned run = block_exclusive_scan<unsigned>(tsum, red, &total);
    if (threadIdx.x == 0) { s_b = -1; s_above = 0; }
    __syncthreads();
    for (int q = 0; q < per; ++q) {
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

// Decides K per group from the fast histogram and fixes the threshold, or starts the exact path.
__global__ void __launch_bounds__(1024) k_sel_find(int kind, long long s, RState *st) {
    unsigned cnt[2];
    for (int i = 0; i < 2; ++i) {
        unsigned above, total;
        hist_find(st->hist[i], 0, &above, &total);
        cnt[i] = total;
    }
    unsigned K[2] = {0, 0};
    if (kind == SEL_REFINE) {
        K[0] = K[1] = min(cnt[0], cnt[1]);
    } else {
        int grp = kind == SEL_INITIAL ? 1 : st->heavy;
        if (grp >= 0) K[grp] = (unsigned)min((long long)cnt[grp], s);
    }
    unsigned slow = 0;
    for (int i = 0; i < 2; ++i) {
        SelGroup &G = st->g[i];
        unsigned above = 0, total = 0;
        int b = -1;
        if (K[i] > 0 && K[i] < cnt[i]) b = hist_find(st->hist[i], K[i], &above, &total);
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
__global__ void __launch_bounds__(kBlock)
k_sel_hist_exact(int N, int kind, const int *__restrict__ gain, const uint8_t *__restrict__ side,
                 const int *__restrict__ nw, RState *st) {
    __shared__ unsigned h[2][kHistBins];
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
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) {
        int g = gain[v];
        int grp = sel_group(kind, st, g, side[v], nw[v]);
        if (grp < 0 || !s_on[grp]) continue;
        unsigned k = gkey(g);
        if (k < s_base[grp] || (unsigned long long)k >= s_top[grp]) continue;
        atomicAdd(&h[grp][(k - s_base[grp]) >> s_shift[grp]], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * kHistBins; i += blockDim.x) {
        unsigned c = (&h[0][0])[i];
        if (c) atomicAdd(&(&st->hist[0][0])[i], c);
    }
}

__global__ void __launch_bounds__(1024) k_sel_find_exact(RState *st, uint32_t *status) {
    for (int i = 0; i < 2; ++i) {
        SelGroup &G = st->g[i];
        const unsigned mode = G.mode;
        __syncthreads();
        if (mode != 3) continue;  // block-uniform
        unsigned above = 0, total = 0;
        int b = hist_find(st->hist[i], G.need, &above, &total);
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

// Applies the selection: refine flips both sides' chosen nodes; the initial partition moves its
// chosen nodes to P0 and keeps the side weights current; the rebalance collects its chosen nodes.
struct ApplyOut {
    int kind;
    const int *gain;
    uint8_t *side;
    const int *nw;
    RState *st;
    int *list;
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
        if (!sel) return;
        if (kind == SEL_REBAL) {
            list[atomicAdd(&st->list_count, 1u)] = (int)v;
        } else {
            side[v] ^= 1;
            if (kind == SEL_INITIAL) {
                atomicAdd(&st->W[0], (unsigned long long)nw[v]);
                atomicAdd(&st->W[1], (unsigned long long)(-(long long)nw[v]));
            }
        }
    }
};

__global__ void __launch_bounds__(kBlock)
k_side_weights(int N, const uint8_t *__restrict__ side, const int *__restrict__ nw, RState *st) {
    unsigned long long w0 = 0, w1 = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) {
        if (side[v]) w1 += nw[v];
        else w0 += nw[v];
    }
    w0 = warp_sum(w0);
    w1 = warp_sum(w1);
    if ((threadIdx.x & 31) == 0) {
        if (w0) atomicAdd(&st->W[0], w0);
        if (w1) atomicAdd(&st->W[1], w1);
    }
}

// Algorithm 3 loop condition: continue while P0 is lighter than P1 (guarded).
__global__ void k_initial_cond(RState *st, long long max_rounds, uint32_t *status) {
    if (threadIdx.x != 0) return;
    unsigned f = (long long)st->W[0] < (long long)st->W[1];
    if (f && (long long)(st->rounds++) >= max_rounds) {
        record_error(status, DEV_TIMEOUT);
        f = 0;
    }
    st->flag = f;
}

// Rebalance loop condition (reading C13): heavy side above the limit and candidates left.
__global__ void k_rebal_cond(RState *st, long long limit, long long max_rounds, uint32_t *status) {
    if (threadIdx.x != 0) return;
    st->limit = limit;
    long long W0 = (long long)st->W[0], W1 = (long long)st->W[1];
    int H = W0 > limit ? 0 : (W1 > limit ? 1 : -1);
    st->heavy = H;
    unsigned f = H >= 0 && !st->warn;
    if (H >= 0) {
        long long Wh = H ? W1 : W0, Wo = H ? W0 : W1;
        st->room = limit - Wo;
        st->need = Wh - limit;
    }
    if (f && (long long)(st->rounds++) >= max_rounds) {
        record_error(status, DEV_TIMEOUT);
        f = 0;
    }
    st->flag = f;
}

// Ordered rebalance move (one block): sort the selected nodes by (gain desc, id asc), move the
// shortest prefix whose weight reaches `need`, stopping at s nodes or before exceeding `room`.
// With nothing selected, marks the level imbalanced.
__global__ void __launch_bounds__(1024)
k_rebal_move(const int *__restrict__ gain, uint8_t *__restrict__ side, const int *__restrict__ nw,
             const int *__restrict__ list, RState *st, long long s) {
    extern __shared__ unsigned long long keys[];
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
    long long moved = 0;
    for (int i = threadIdx.x; i < cut; i += blockDim.x) {
        int v = (int)(keys[i] & 0xffffffffu);
        side[v] = (uint8_t)(1 - heavy);
        moved += nw[v];
    }
    moved = block_sum(moved, red);
    if (threadIdx.x == 0) {
        atomicAdd(&st->W[1 - heavy], (unsigned long long)moved);
        atomicAdd(&st->W[heavy], (unsigned long long)(-moved));
    }
}

__global__ void k_project(int N, const int *__restrict__ cmap, const uint8_t *__restrict__ coarse,
                          uint8_t *__restrict__ fine) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x)
        fine[v] = coarse[cmap[v]];
}

__global__ void k_keep_status(RState *st) {
    if (threadIdx.x == 0) st->status0 = st->warn;
}

// ------------------------------------------------------------------------ host side
int64_t balance_limit(int64_t W, double eps) {
    long long e6 = llround(eps * 1e6);
    int64_t a = (W + 1) / 2;
    int64_t b = (W * (1000000 + e6)) / 2000000;
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

void compute_gains(bipart_graph *g, Level &L, const uint8_t *side, int *gain) {
    cudaStream_t s = g->stream;
    int *n1 = g->w.e_d.as<int>();
    int2 *hc = g->w.hc.as<int2>();
    if (L.E > 0) {
        BP_CUDA(cudaMemsetAsync(n1, 0, sizeof(int) * (size_t)L.E, s));
        {
            // hoff, pins, one side byte per pin, one atomic per hyperedge run
            ProfScope ps("hedge_n1", 8.0 * L.E + 5.0 * L.P, s);
            k_hedge_n1<<<lb_grid(L.P), kLbBlock, 0, s>>>(L.E, L.P, L.hoff(), L.pins(), side, n1);
            BP_LAUNCH();
        }
        {
            ProfScope ps("hedge_contrib", 16.0 * L.E + (L.hw() ? 4.0 * L.E : 0.0), s);
            k_hedge_contrib<<<grid_for(L.E), kBlock, 0, s>>>(L.E, L.hoff(), L.hw(), n1, hc);
            BP_LAUNCH();
        }
    }
    if (L.N > 0) BP_CUDA(cudaMemsetAsync(gain, 0, sizeof(int) * (size_t)L.N, s));
    if (L.P > 0) {
        // noff, nadj, 8-byte contribution gather per incidence, side, gain
        ProfScope ps("node_gain", 9.0 * L.N + 12.0 * L.P, s);
        k_node_gain<<<lb_grid(L.P), kLbBlock, 0, s>>>(L.N, L.P, L.noff(), L.nadj(), hc, side, gain);
        BP_LAUNCH();
    }
}

// Top-K selection per `kind` and its application (flip, or collect for the ordered rebalance).
void select_apply(bipart_graph *g, Level &L, int kind, long long sq, const int *gain,
                  uint8_t *side, int *list) {
    cudaStream_t s = g->stream;
    RState *st = rstate(g);
    BP_CUDA(cudaMemsetAsync(&st->hist[0][0], 0, sizeof(st->hist), s));
    if (kind == SEL_REBAL) BP_CUDA(cudaMemsetAsync(&st->list_count, 0, sizeof(unsigned), s));
    {
        ProfScope ps("select_hist", 9.0 * L.N, s);
        k_sel_hist<<<grid_for(L.N), kBlock, 0, s>>>(L.N, kind, gain, side, L.nw(), st);
        BP_LAUNCH();
    }
    k_sel_find<<<1, 1024, 0, s>>>(kind, sq, st);
    BP_LAUNCH();
    device_if(g, &st->slow, [&]() {
        for (int pass = 0; pass < 3; ++pass) {
            BP_CUDA(cudaMemsetAsync(&st->hist[0][0], 0, sizeof(st->hist), g->stream));
            k_sel_hist_exact<<<grid_for(L.N), kBlock, 0, g->stream>>>(L.N, kind, gain, side, L.nw(), st);
            BP_LAUNCH();
            k_sel_find_exact<<<1, 1024, 0, g->stream>>>(st, dev_status(g));
            BP_LAUNCH();
        }
    });
    s = g->stream;
    ProfScope ps("select_apply", 10.0 * L.N, s);
    scan(L.N, TieIn{kind, gain, side, L.nw(), st}, ApplyOut{kind, gain, side, L.nw(), st, list},
         g->w.scan.ensure(scan_state_bytes(L.N), s), dev_status(g), s);
}

void side_weights(bipart_graph *g, Level &L, const uint8_t *side) {
    cudaStream_t s = g->stream;
    RState *st = rstate(g);
    BP_CUDA(cudaMemsetAsync(&st->W[0], 0, 2 * sizeof(unsigned long long), s));
    if (L.N > 0) {
        k_side_weights<<<grid_for(L.N), kBlock, 0, s>>>(L.N, side, L.nw(), st);
        BP_LAUNCH();
    }
}

// Algorithm 3 on the coarsest level.
void initial_partition(bipart_graph *g, Level &L, uint8_t *side, int *gain) {
    cudaStream_t s = g->stream;
    if (L.N == 0) return;
    RState *st = rstate(g);
    const long long sq = ceil_sqrt64(L.N);
    BP_CUDA(cudaMemsetAsync(side, 1, (size_t)L.N, s));
    BP_CUDA(cudaMemsetAsync(&st->rounds, 0, sizeof(unsigned), s));
    side_weights(g, L, side);
    k_initial_cond<<<1, 32, 0, s>>>(st, (long long)L.N + 1, dev_status(g));
    BP_LAUNCH();
    device_while(g, &st->flag, (int64_t)L.N + 2, [&]() {
        compute_gains(g, L, side, gain);
        select_apply(g, L, SEL_INITIAL, sq, gain, side, nullptr);
        k_initial_cond<<<1, 32, 0, g->stream>>>(st, (long long)L.N + 1, dev_status(g));
        BP_LAUNCH();
    });
}

void refine_iter(bipart_graph *g, Level &L, uint8_t *side, int *gain) {
    if (L.N == 0) return;
    compute_gains(g, L, side, gain);
    select_apply(g, L, SEL_REFINE, 0, gain, side, nullptr);
}

// Rebalance of reading C13; leaves warn = 1 when it ran out of candidates.
void rebalance(bipart_graph *g, Level &L, uint8_t *side, int *gain, int64_t limit) {
    cudaStream_t s = g->stream;
    RState *st = rstate(g);
    const int64_t sq = ceil_sqrt64(L.N);
    if (sq > kRebalMax) throw Fail{BIPART_ERR_OOM, "level too large for the ordered rebalance"};
    int *list = (int *)g->w.list.ensure(sizeof(int) * (size_t)std::max<int64_t>(sq, 1), s);
    int S = 1;
    while (S < sq) S <<= 1;
    const size_t smem = sizeof(unsigned long long) * (size_t)S;
    BP_CUDA(cudaMemsetAsync(&st->warn, 0, sizeof(unsigned), s));
    BP_CUDA(cudaMemsetAsync(&st->rounds, 0, sizeof(unsigned), s));
    side_weights(g, L, side);
    k_rebal_cond<<<1, 32, 0, s>>>(st, (long long)limit, (long long)L.N + 1, dev_status(g));
    BP_LAUNCH();
    device_while(g, &st->flag, (int64_t)L.N + 2, [&]() {
        compute_gains(g, L, side, gain);
        select_apply(g, L, SEL_REBAL, sq, gain, side, list);
        k_rebal_move<<<1, 1024, smem, g->stream>>>(gain, side, L.nw(), list, st, sq);
        BP_LAUNCH();
        k_rebal_cond<<<1, 32, 0, g->stream>>>(st, (long long)limit, (long long)L.N + 1, dev_status(g));
        BP_LAUNCH();
    });
}

}  // namespace

void uncoarsen(bipart_graph *g, std::vector<Level *> &levels, int64_t limit, int32_t iters,
               uint8_t *d_side0) {
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
    g->w.e_d.ensure(sizeof(int) * (size_t)emax, s);

    uint8_t *cur = sa, *other = sb;
    initial_partition(g, *levels[Lc], cur, gain);
    for (int l = Lc; l >= 0; --l) {
        Level *L = levels[l];
        s = g->stream;
        if (l < Lc) {
            if (L->N > 0) {
                ProfScope ps("project", 6.0 * L->N, s);
                k_project<<<grid_for(L->N), kBlock, 0, s>>>(L->N, L->cmap(), cur, other);
                BP_LAUNCH();
            }
            std::swap(cur, other);
        }
        for (int it = 0; it < iters; ++it) refine_iter(g, *L, cur, gain);
        if (L->N > 0) rebalance(g, *L, cur, gain, limit);
        else BP_CUDA(cudaMemsetAsync(&rstate(g)->warn, 0, sizeof(unsigned), g->stream));
    }
    s = g->stream;
    k_keep_status<<<1, 32, 0, s>>>(rstate(g));
    BP_LAUNCH();
    if (levels[0]->N > 0)
        BP_CUDA(cudaMemcpyAsync(d_side0, cur, (size_t)levels[0]->N, cudaMemcpyDeviceToDevice, s));
}

const unsigned *bisect_status_word(bipart_graph *g) { return &rstate(g)->status0; }

void refine_init() {
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, []() {
        err = cudaFuncSetAttribute(k_rebal_move, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(sizeof(unsigned long long) * kRebalMax));
    });
    BP_CUDA(err);
}

}  // namespace bp
