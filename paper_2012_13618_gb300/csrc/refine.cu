// Initial partitioning and refinement on sm_103a (Sec. 3.2-3.3): Algorithm 4 move gains from
// per-hyperedge side counts, Algorithm 3 growth of P0 by the top ceil(sqrt n) gains, Algorithm 5
// swaps of the gain >= 0 lists and the rebalancing pass.
//
// Ordering of nodes is always (gain descending, node id ascending).  The top-K of a candidate set
// is found without sorting: a radix select over the order-preserving 32-bit key
// key = gain ^ 0x80000000 (up to three 11-bit histogram passes) fixes the threshold key and how
// many nodes with exactly that key are taken; a scan over node ids then takes the lowest ids
// among the ties.  Only the rebalancing pass needs the selected nodes in order; it sorts at most
// ceil(sqrt n) of them in shared memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>

#include "common.cuh"
#include "internal.h"
#include "lb.cuh"
#include "scan.cuh"

namespace bp {

namespace {

constexpr int kBlock = 256;
constexpr int kHistBits = 11;
constexpr int kHistBins = 1 << kHistBits;
constexpr int kWarpDeg = 32;          // hyperedges above this degree: one warp each
constexpr int kRebalMax = 16384;      // largest ceil(sqrt n) handled by the ordered rebalance

inline int grid_for(int64_t n, int per_block = kBlock, int cap = 152 * 16) {
    int64_t b = (n + per_block - 1) / per_block;
    if (b < 1) b = 1;
    return (int)std::min<int64_t>(b, cap);
}

}  // namespace

// Candidate predicate of a selection.
enum SelKind : int { SEL_REFINE = 0, SEL_INITIAL = 1, SEL_REBAL = 2 };

// Selection state of one group (one side).  mode: 0 none, 1 all candidates, 2 threshold final,
// 3 threshold in progress.
struct SelGroup {
    unsigned kmin, kmax, cnt, K;
    unsigned base, shift, need, thr, take_eq, mode;
    unsigned long long top;  // exclusive upper bound of the keys still in play
    unsigned pad[4];
};
struct SelState {
    SelGroup g[2];
    unsigned hist[2][kHistBins];
    unsigned long long W[2];      // side weights
    unsigned list_count;
};

struct SelArgs {
    int kind;
    int heavy;        // SEL_REBAL: heavy side
    long long room;   // SEL_REBAL: weight room on the light side
    long long s;      // ceil(sqrt n) for SEL_INITIAL / SEL_REBAL
};

__device__ __forceinline__ unsigned gkey(int gain) { return (unsigned)gain ^ 0x80000000u; }

__device__ __forceinline__ int sel_group(const SelArgs &a, int gain, uint8_t side, int w) {
    if (a.kind == SEL_REFINE) return gain >= 0 ? (int)side : -1;
    if (a.kind == SEL_INITIAL) return side == 1 ? 1 : -1;
    return (side == a.heavy && (long long)w <= a.room) ? a.heavy : -1;
}

// ------------------------------------------------------------------------ Algorithm 4
// Per hyperedge: n1 = pins on side 1; contribution to a pin on side i:
// +w if n_i == 1 (moving it uncuts e), -w if n_i == |e| (moving it cuts e), else 0.
__device__ __forceinline__ int2 contrib(int n1, int d, int w) {
    int n0 = d - n1;
    int c0 = n0 == 1 ? w : (n0 == d ? -w : 0);
    int c1 = n1 == 1 ? w : (n1 == d ? -w : 0);
    return make_int2(c0, c1);
}

__global__ void __launch_bounds__(kBlock)
k_hedge_side_small(int E, const int *__restrict__ hoff, const int *__restrict__ pins,
                   const int *__restrict__ hw, const uint8_t *__restrict__ side,
                   int2 *__restrict__ hc) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
        int a = hoff[e], d = hoff[e + 1] - a;
        if (d > kWarpDeg) continue;
        int n1 = 0;
        for (int i = 0; i < d; ++i) n1 += side[pins[a + i]];
        hc[e] = contrib(n1, d, hw ? hw[e] : 1);
    }
}

__global__ void __launch_bounds__(kBlock)
k_hedge_side_big(const int *__restrict__ hoff, const int *__restrict__ pins,
                 const int *__restrict__ hw, const uint8_t *__restrict__ side,
                 const int *__restrict__ list, const int *__restrict__ count,
                 int2 *__restrict__ hc) {
    const int n = *count;
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < n; w += warps) {
        int e = list[w];
        int a = hoff[e], d = hoff[e + 1] - a;
        int n1 = 0;
        for (int i = lane; i < d; i += 32) n1 += side[pins[a + i]];
        n1 = warp_sum(n1);
        if (lane == 0) hc[e] = contrib(n1, d, hw ? hw[e] : 1);
    }
}

__global__ void k_big_list(int E, const int *__restrict__ hoff, int *__restrict__ list,
                           int *__restrict__ count) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x)
        if (hoff[e + 1] - hoff[e] > kWarpDeg) list[atomicAdd(count, 1)] = e;
}

// gain[v] = sum over v's hyperedges of the contribution for v's side; load-balanced over the
// incidence array, per-node partial sums combined with integer atomicAdd (gain zeroed first).
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
__global__ void k_sel_reset(SelState *st) {
    for (int i = threadIdx.x; i < 2; i += blockDim.x) {
        st->g[i].kmin = 0xffffffffu;
        st->g[i].kmax = 0;
        st->g[i].cnt = 0;
        st->g[i].K = 0;
        st->g[i].mode = 0;
    }
    if (threadIdx.x == 0) st->list_count = 0;
}

__global__ void __launch_bounds__(kBlock)
k_sel_count(int N, SelArgs a, const int *__restrict__ gain, const uint8_t *__restrict__ side,
            const int *__restrict__ nw, SelState *st) {
    unsigned mn[2] = {0xffffffffu, 0xffffffffu}, mx[2] = {0, 0}, c[2] = {0, 0};
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) {
        int g = gain[v];
        int grp = sel_group(a, g, side[v], nw[v]);
        if (grp < 0) continue;
        unsigned k = gkey(g);
        mn[grp] = min(mn[grp], k);
        mx[grp] = max(mx[grp], k);
        c[grp]++;
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        mn[i] = warp_min(mn[i]);
        mx[i] = warp_max(mx[i]);
        c[i] = warp_sum(c[i]);
        if ((threadIdx.x & 31) == 0 && c[i]) {
            atomicMin(&st->g[i].kmin, mn[i]);
            atomicMax(&st->g[i].kmax, mx[i]);
            atomicAdd(&st->g[i].cnt, c[i]);
        }
    }
}

__device__ __forceinline__ unsigned bitlen(unsigned x) { return x ? 32u - __clz(x) : 0u; }

// Decides K per group and prepares the first histogram pass.
__global__ void k_sel_plan(SelArgs a, SelState *st) {
    if (threadIdx.x != 0) return;
    unsigned K[2];
    if (a.kind == SEL_REFINE) {
        unsigned l = min(st->g[0].cnt, st->g[1].cnt);
        K[0] = K[1] = l;
    } else {
        int grp = a.kind == SEL_INITIAL ? 1 : a.heavy;
        K[grp] = (unsigned)min((long long)st->g[grp].cnt, a.s);
        K[1 - grp] = 0;
    }
    for (int i = 0; i < 2; ++i) {
        SelGroup &g = st->g[i];
        g.K = K[i];
        if (K[i] == 0) { g.mode = 0; continue; }
        if (K[i] >= g.cnt) { g.mode = 1; continue; }
        unsigned range = g.kmax - g.kmin;  // keys span [kmin, kmax]
        unsigned b = bitlen(range);
        g.base = g.kmin;
        g.top = (unsigned long long)g.kmax + 1ull;
        g.shift = b > kHistBits ? b - kHistBits : 0;
        g.need = K[i];
        g.mode = 3;
    }
}

__global__ void k_sel_clear_hist(SelState *st) {
    for (int i = threadIdx.x; i < 2 * kHistBins; i += blockDim.x) (&st->hist[0][0])[i] = 0;
}

__global__ void __launch_bounds__(kBlock)
k_sel_hist(int N, SelArgs a, const int *__restrict__ gain, const uint8_t *__restrict__ side,
           const int *__restrict__ nw, SelState *st) {
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
        int grp = sel_group(a, g, side[v], nw[v]);
        if (grp < 0 || !s_on[grp]) continue;
        unsigned k = gkey(g);
        if (k < s_base[grp] || (unsigned long long)k >= s_top[grp]) continue;
        unsigned long long off = (unsigned long long)(k - s_base[grp]) >> s_shift[grp];
        if (off >= kHistBins) continue;
        atomicAdd(&h[grp][off], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * kHistBins; i += blockDim.x) {
        unsigned c = (&h[0][0])[i];
        if (c) atomicAdd(&(&st->hist[0][0])[i], c);
    }
}

// One block of 1024 threads: for each group in progress, find the bucket holding the need-th
// largest key; either finish (bucket width 1) or narrow to that bucket for the next pass.
__global__ void __launch_bounds__(1024) k_sel_find(SelState *st, uint32_t *status) {
    __shared__ unsigned suf[kHistBins];
    __shared__ unsigned red[33];
    __shared__ int s_bucket;
    for (int i = 0; i < 2; ++i) {
        SelGroup &g = st->g[i];
        if (g.mode != 3) continue;  // uniform across the block
        // suffix sums: suf[b] = count of keys in buckets > b
        const int per = kHistBins / 1024;
        unsigned loc[kHistBins / 1024];
        unsigned tsum = 0;
        for (int q = 0; q < per; ++q) {
            int b = kHistBins - 1 - (threadIdx.x * per + q);  // descending bucket order
            loc[q] = st->hist[i][b];
            tsum += loc[q];
        }
        unsigned total;
        unsigned ex = block_exclusive_scan<unsigned>(tsum, red, &total);
        if (threadIdx.x == 0) s_bucket = -1;
        __syncthreads();
        unsigned run = ex;
        for (int q = 0; q < per; ++q) {
            int b = kHistBins - 1 - (threadIdx.x * per + q);
            suf[b] = run;  // keys strictly above bucket b
            if (run < g.need && run + loc[q] >= g.need) s_bucket = b;
            run += loc[q];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int b = s_bucket;
            if (b < 0) {  // inconsistent counts: select nothing and report it
                g.mode = 0;
                record_error(status, DEV_OVERFLOW);
            } else {
                unsigned need = g.need - suf[b];
                g.base = g.base + ((unsigned)b << g.shift);
                g.top = (unsigned long long)g.base + (1ull << g.shift);
                if (g.shift == 0) {
                    g.thr = g.base;
                    g.take_eq = need;
                    g.mode = 2;
                } else {
                    g.need = need;
                    g.shift = g.shift > kHistBits ? g.shift - kHistBits : 0;
                }
            }
        }
        __syncthreads();
    }
}

// Tie ranks: value = (ties of group 1) << 31 | ties of group 0, ties = candidates with key == thr.
struct TieIn {
    SelArgs a;
    const int *gain;
    const uint8_t *side;
    const int *nw;
    const SelState *st;
    __device__ uint64_t operator()(int64_t v) const {
        int g = gain[v];
        int grp = sel_group(a, g, side[v], nw[v]);
        if (grp < 0 || st->g[grp].mode != 2 || gkey(g) != st->g[grp].thr) return 0;
        return grp ? (1ull << 31) : 1ull;
    }
};

// Applies the selection: flips the side (refine / initial) or appends to the ordered-rebalance list.
struct ApplyOut {
    SelArgs a;
    const int *gain;
    uint8_t *side;
    const int *nw;
    SelState *st;
    int *list;
    __device__ void operator()(int64_t v, uint64_t pre, uint64_t val) const {
        int g = gain[v];
        int grp = sel_group(a, g, side[v], nw[v]);
        if (grp < 0) return;
        const SelGroup &G = st->g[grp];
        bool sel;
        if (G.mode == 1) sel = true;
        else if (G.mode == 2) {
            unsigned k = gkey(g);
            unsigned rank = grp ? (unsigned)(pre >> 31) : (unsigned)(pre & 0x7fffffffu);
            sel = k > G.thr || (k == G.thr && rank < G.take_eq);
        } else sel = false;
        if (!sel) return;
        if (a.kind == SEL_REBAL) list[atomicAdd(&st->list_count, 1u)] = (int)v;
        else side[v] ^= 1;
    }
};

__global__ void __launch_bounds__(kBlock)
k_side_weights(int N, const uint8_t *__restrict__ side, const int *__restrict__ nw, SelState *st) {
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

// Ordered rebalance move (one block): sort the selected nodes by (gain desc, id asc), then move
// the shortest prefix whose weight reaches `need`, stopping at s nodes or before exceeding room.
__global__ void __launch_bounds__(1024)
k_rebal_move(const int *__restrict__ gain, uint8_t *__restrict__ side, const int *__restrict__ nw,
             const int *__restrict__ list, SelState *st, int heavy, long long need, long long room,
             long long s) {
    extern __shared__ unsigned long long keys[];
    __shared__ long long red[33];
    __shared__ int s_cut;
    const int n = (int)st->list_count;
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
    // prefix weights in sorted order: each thread owns a contiguous chunk
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
    for (int i = threadIdx.x; i < cut; i += blockDim.x) side[(int)(keys[i] & 0xffffffffu)] = (uint8_t)(1 - heavy);
}

__global__ void k_project(int N, const int *__restrict__ cmap, const uint8_t *__restrict__ coarse,
                          uint8_t *__restrict__ fine) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x)
        fine[v] = coarse[cmap[v]];
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

struct LevelCtx {
    Level *L;
    int *big_list;
    int *big_count;
};

void compute_gains(bipart_graph *g, const LevelCtx &lc, const uint8_t *side, int *gain) {
    cudaStream_t s = g->stream;
    Level &L = *lc.L;
    int2 *hc = (int2 *)g->w.hc.as<int2>();
    if (L.E > 0) {
        // hoff, pins, one side byte per pin, weights; writes two contributions per hyperedge
        ProfScope ps("hedge_side", 12.0 * L.E + 5.0 * L.P + (L.hw() ? 4.0 * L.E : 0.0), s);
        k_hedge_side_small<<<grid_for(L.E), kBlock, 0, s>>>(L.E, L.hoff(), L.pins(), L.hw(), side, hc);
        BP_LAUNCH();
        k_hedge_side_big<<<grid_for((int64_t)L.P / (kWarpDeg + 1) * 32 + 32), kBlock, 0, s>>>(
            L.hoff(), L.pins(), L.hw(), side, lc.big_list, lc.big_count, hc);
        BP_LAUNCH();
    }
    if (L.N > 0) BP_CUDA(cudaMemsetAsync(gain, 0, sizeof(int) * (size_t)L.N, s));
    if (L.P > 0) {
        // noff, nadj, 8-byte contribution gather per incidence, side, gain
        ProfScope ps("node_gain", 9.0 * L.N + 12.0 * L.P, s);
        k_node_gain<<<lb_grid(L.P), kLbBlock, 0, s>>>(L.N, L.P, L.noff(), L.nadj(), hc, side, gain);
        BP_LAUNCH();
    }
}

SelState *sel_state(bipart_graph *g) {
    return reinterpret_cast<SelState *>(g->w.small.as<char>() + 256);
}

// Selects per SelArgs and applies (flip or list).  Returns nothing; state stays on the device.
void select_apply(bipart_graph *g, Level &L, const SelArgs &a, const int *gain, uint8_t *side,
                  int *list) {
    cudaStream_t s = g->stream;
    SelState *st = sel_state(g);
    k_sel_reset<<<1, 32, 0, s>>>(st);
    BP_LAUNCH();
    {
        ProfScope ps("select_count", 9.0 * L.N, s);
        k_sel_count<<<grid_for(L.N), kBlock, 0, s>>>(L.N, a, gain, side, L.nw(), st);
        BP_LAUNCH();
    }
    k_sel_plan<<<1, 32, 0, s>>>(a, st);
    BP_LAUNCH();
    for (int pass = 0; pass < 3; ++pass) {
        k_sel_clear_hist<<<1, 1024, 0, s>>>(st);
        BP_LAUNCH();
        {
            ProfScope ps("select_hist", 9.0 * L.N, s);
            k_sel_hist<<<grid_for(L.N), kBlock, 0, s>>>(L.N, a, gain, side, L.nw(), st);
            BP_LAUNCH();
        }
        k_sel_find<<<1, 1024, 0, s>>>(st, dev_status(g));
        BP_LAUNCH();
    }
    ProfScope ps("select_apply", 10.0 * L.N, s);
    scan(L.N, TieIn{a, gain, side, L.nw(), st}, ApplyOut{a, gain, side, L.nw(), st, list},
         g->w.scan.ensure(scan_state_bytes(L.N), s), dev_status(g), s);
}

void side_weights(bipart_graph *g, Level &L, const uint8_t *side, int64_t W[2]) {
    cudaStream_t s = g->stream;
    SelState *st = sel_state(g);
    BP_CUDA(cudaMemsetAsync(&st->W[0], 0, 2 * sizeof(unsigned long long), s));
    if (L.N > 0) {
        k_side_weights<<<grid_for(L.N), kBlock, 0, s>>>(L.N, side, L.nw(), st);
        BP_LAUNCH();
    }
    BP_CUDA(cudaMemcpyAsync(g->w.host_small, &st->W[0], 2 * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, s));
    sync(g);
    check_status(g);
    const unsigned long long *hw = reinterpret_cast<const unsigned long long *>(g->w.host_small);
    W[0] = (int64_t)hw[0];
    W[1] = (int64_t)hw[1];
}

// Algorithm 3 on the coarsest level.
void initial_partition(bipart_graph *g, const LevelCtx &lc, uint8_t *side, int *gain) {
    cudaStream_t s = g->stream;
    Level &L = *lc.L;
    if (L.N == 0) return;
    BP_CUDA(cudaMemsetAsync(side, 1, (size_t)L.N, s));
    SelArgs a{SEL_INITIAL, 1, 0, ceil_sqrt64(L.N)};
    int64_t W[2];
    side_weights(g, L, side, W);
    int64_t rounds = 0;
    while (W[0] < W[1]) {
        if (++rounds > (int64_t)L.N + 1) throw Fail{BIPART_ERR_TIMEOUT, "initial partition made no progress"};
        compute_gains(g, lc, side, gain);
        select_apply(g, L, a, gain, side, nullptr);
        side_weights(g, L, side, W);
    }
}

void refine_iter(bipart_graph *g, const LevelCtx &lc, uint8_t *side, int *gain) {
    Level &L = *lc.L;
    if (L.N == 0) return;
    compute_gains(g, lc, side, gain);
    SelArgs a{SEL_REFINE, 0, 0, 0};
    select_apply(g, L, a, gain, side, nullptr);
}

int rebalance(bipart_graph *g, const LevelCtx &lc, uint8_t *side, int *gain, int64_t limit) {
    cudaStream_t s = g->stream;
    Level &L = *lc.L;
    const int64_t sq = ceil_sqrt64(L.N);
    if (sq > kRebalMax) throw Fail{BIPART_ERR_OOM, "level too large for the ordered rebalance"};
    int *list = (int *)g->w.list.ensure(sizeof(int) * (size_t)std::max<int64_t>(sq, 1), s);
    for (int64_t rounds = 0;; ++rounds) {
        if (rounds > (int64_t)L.N + 1) throw Fail{BIPART_ERR_TIMEOUT, "rebalance made no progress"};
        int64_t W[2];
        side_weights(g, L, side, W);
        int H;
        if (W[0] > limit) H = 0;
        else if (W[1] > limit) H = 1;
        else return BIPART_OK;
        const int64_t room = limit - W[1 - H], need = W[H] - limit;
        compute_gains(g, lc, side, gain);
        SelArgs a{SEL_REBAL, H, (long long)room, (long long)sq};
        select_apply(g, L, a, gain, side, list);
        SelState *st = sel_state(g);
        BP_CUDA(cudaMemcpyAsync(g->w.host_small, &st->list_count, sizeof(unsigned),
                                cudaMemcpyDeviceToHost, s));
        sync(g);
        const unsigned n = g->w.host_small[0];
        if (n == 0) return BIPART_WARN_IMBALANCED;
        int S = 1;
        while (S < (int)n) S <<= 1;
        size_t smem = sizeof(unsigned long long) * (size_t)S;
        if (smem > 48 * 1024)
            BP_CUDA(cudaFuncSetAttribute(k_rebal_move, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_rebal_move<<<1, 1024, smem, s>>>(gain, side, L.nw(), list, st, H, (long long)need,
                                          (long long)room, (long long)sq);
        BP_LAUNCH();
    }
}

}  // namespace

int uncoarsen(bipart_graph *g, std::vector<Level *> &levels, int64_t limit, int32_t iters,
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
    int *big_list = (int *)g->w.e_c.ensure(sizeof(int) * (size_t)emax, s);
    int *big_count = g->w.small.as<int>() + 8;

    auto level_ctx = [&](Level *L) {
        BP_CUDA(cudaMemsetAsync(big_count, 0, sizeof(int), s));
        if (L->E > 0) {
            k_big_list<<<grid_for(L->E), kBlock, 0, s>>>(L->E, L->hoff(), big_list, big_count);
            BP_LAUNCH();
        }
        return LevelCtx{L, big_list, big_count};
    };

    uint8_t *cur = sa, *other = sb;
    LevelCtx lc = level_ctx(levels[Lc]);
    initial_partition(g, lc, cur, gain);
    int status = BIPART_OK;
    for (int l = Lc; l >= 0; --l) {
        Level *L = levels[l];
        if (l < Lc) {
            lc = level_ctx(L);
            if (L->N > 0) {
                ProfScope ps("project", 6.0 * L->N, s);
                k_project<<<grid_for(L->N), kBlock, 0, s>>>(L->N, L->cmap(), cur, other);
                BP_LAUNCH();
            }
            std::swap(cur, other);
        }
        for (int it = 0; it < iters; ++it) refine_iter(g, lc, cur, gain);
        status = rebalance(g, lc, cur, gain, limit);
    }
    if (levels[0]->N > 0)
        BP_CUDA(cudaMemcpyAsync(d_side0, cur, (size_t)levels[0]->N, cudaMemcpyDeviceToDevice, s));
    return status;
}

}  // namespace bp
