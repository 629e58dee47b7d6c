// Batched bisection in one persistent launch: every thread block takes whole instances from a
// global queue (largest first) and runs the complete multilevel bisection of an instance on its
// own -- level-0 normalisation, coarsening (Algorithms 1-2), the initial partition (Algorithm
// 3), refinement and rebalancing (Algorithms 4-5) -- with the phases separated by
// __syncthreads() instead of kernel boundaries.  The phase code is the same device code the grid
// kernels run (coarsen_dev.cuh, refine_dev.cuh) instantiated for a one-block team, so an
// instance's result is identical to the single-instance path.
//
// Each block owns an arena in HBM (sized by the host for the largest instance it may receive)
// from which it carves the level store and scratch of its current instance with a bump
// pointer.  An instance whose hierarchy does not fit is marked deferred and the host runs it
// through the single-instance path instead.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cmath>
#include <cstdlib>
#include <vector>

#include "coarsen_dev.cuh"
#include "common.cuh"
#include "internal.h"
#include "refine_dev.cuh"
#include "scan.cuh"

namespace bp {

namespace {

constexpr int kBT = 512;                  // threads per block
constexpr int kMaxLev = 64;
constexpr size_t kSmemBytes = 32 * 1024;  // union: bitmap window / gain histogram / sort keys

}  // namespace


struct BArgs {
    BInst *inst;
    int n;
    int *next;                 // queue head
    const int *hoff, *pins, *nw, *hw;
    uint8_t *side_out;
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
    RState *st;
};

// Sorted-unique of every hyperedge (mapped through map, or as is) into scratch + cnt, then the
// compacted hyperedge CSR of `c` (hyperedges with >= 2 distinct pins) with its degrees counted.
// Returns false if the arena overflowed.
template <bool MAP>
__device__ bool blk_contract(Ctx &x, int E, int P, const int *hoff, const int *pins, const int *hw,
                             const int *map, DLevel &c) {
    int *cnt = x.e_a, *emap = x.e_b, *mid = x.e_c, *big = x.e_d, *counters = x.cnt4;
    if (threadIdx.x == 0) { counters[0] = 0; counters[1] = 0; counters[2] = 0; counters[3] = 0; }
    __syncthreads();
    d_seg_small<MAP>(x.t, E, hoff, pins, map, x.p_a, cnt, mid, big, counters);
    __syncthreads();
    d_seg_mid<MAP>(x.t, hoff, pins, map, x.p_a, cnt, mid, counters);
    __syncthreads();
    d_seg_big<MAP>(x.t, hoff, pins, map, x.p_a, cnt, big, counters, reinterpret_cast<uint32_t *>(x.smem));
    __syncthreads();
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
__device__ bool blk_incidence(Ctx &x, DLevel &c) {
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
__device__ bool blk_coarsen(Ctx &x, const DLevel &f, DLevel &c, int policy) {
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
    if (!blk_contract<true>(x, E, f.P, f.hoff, f.pins, f.hw, f.cmap, c)) return false;
    return blk_incidence(x, c);
}

// ----------------------------------------------------------------- refinement (block versions)
__device__ void blk_gains(Ctx &x, const DLevel &L, const uint8_t *side) {
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

__device__ void blk_select_apply(Ctx &x, const DLevel &L, int kind, long long sq, uint8_t *side) {
    RState *st = x.st;
    unsigned(*h)[kHistBins] = reinterpret_cast<unsigned(*)[kHistBins]>(x.smem);
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

__device__ void blk_initial(Ctx &x, const DLevel &L, uint8_t *side) {
    if (L.N == 0) return;
    RState *st = x.st;
    const long long sq = (long long)ceilf(sqrtf((float)L.N));
    long long s = sq;
    while (s * s < L.N) ++s;
    while (s > 1 && (s - 1) * (s - 1) >= L.N) --s;
    blk_fill(side, (size_t)L.N, (uint8_t)1);
    if (threadIdx.x == 0) st->rounds = 0;
    __syncthreads();
    blk_side_weights(x, L, side);
    if (threadIdx.x == 0) d_initial_cond(st, (long long)L.N + 1, x.status);
    __syncthreads();
    while (st->flag) {
        blk_gains(x, L, side);
        blk_select_apply(x, L, SEL_INITIAL, s, side);
        if (threadIdx.x == 0) d_initial_cond(st, (long long)L.N + 1, x.status);
        __syncthreads();
    }
}

__device__ void blk_rebalance(Ctx &x, const DLevel &L, uint8_t *side, long long limit) {
    RState *st = x.st;
    long long s = (long long)ceilf(sqrtf((float)L.N));
    while (s * s < L.N) ++s;
    while (s > 1 && (s - 1) * (s - 1) >= L.N) --s;
    if (threadIdx.x == 0) { st->warn = 0; st->rounds = 0; }
    __syncthreads();
    blk_side_weights(x, L, side);
    if (threadIdx.x == 0) d_rebal_cond(st, limit, limit, (long long)L.N + 1, x.status);
    __syncthreads();
    while (st->flag) {
        blk_gains(x, L, side);
        blk_select_apply(x, L, SEL_REBAL, s, side);
        d_rebal_move(x.gain, side, L.nw, x.list, st, s, reinterpret_cast<unsigned long long *>(x.smem));
        __syncthreads();
        if (threadIdx.x == 0) d_rebal_cond(st, limit, limit, (long long)L.N + 1, x.status);
        __syncthreads();
    }
}

// One whole instance.  Returns its status (0 ok, 1 imbalanced, 2 deferred).
__device__ int blk_bisect(Ctx &x, const BArgs &a, const BInst &I, DLevel *lev) {
    const int N = I.N, E = I.E, P = I.P;
    // scratch sized by the input
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
    x.p_a = x.ar.take<int>(P);
    long long sq0 = (long long)ceilf(sqrtf((float)(N > 0 ? N : 1))) + 2;
    x.list = x.ar.take<int>((size_t)sq0);
    x.cnt4 = x.ar.take<int>(8);
    x.st = x.ar.take<RState>(1);
    if (x.ar.overflow) return 2;
    // level 0: normalised input
    const int *hoff = a.hoff + I.hoff, *pins = a.pins + I.pins;
    const int *hw = I.hw >= 0 ? a.hw + I.hw : nullptr;
    DLevel &L0 = lev[0];
    L0.N = N;
    if (!blk_contract<false>(x, E, P, hoff, pins, hw, nullptr, L0)) return 2;
    L0.nw = x.ar.take<int>(N);
    if (x.ar.overflow) return 2;
    for (int v = threadIdx.x; v < N; v += blockDim.x) L0.nw[v] = I.nw >= 0 ? a.nw[I.nw + v] : 1;
    __syncthreads();
    if (!blk_incidence(x, L0)) return 2;
    // coarsening (Sec. 3.4 stop rule, reading C11)
    int nl = 1;
    while (nl - 1 < I.levels && nl < kMaxLev && lev[nl - 1].E > 0) {
        const size_t mark = x.ar.top;
        if (!blk_coarsen(x, lev[nl - 1], lev[nl], I.policy)) return 2;
        if (lev[nl].N == lev[nl - 1].N) {
            x.ar.top = mark;
            break;
        }
        ++nl;
    }
    // initial partition, then refinement from the coarsest level to level 0
    uint8_t *cur = x.side_a, *other = x.side_b;
    blk_initial(x, lev[nl - 1], cur);
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
        if (L.N > 0) blk_rebalance(x, L, cur, I.limit);
        else if (threadIdx.x == 0) x.st->warn = 0;
        __syncthreads();
    }
    for (int v = threadIdx.x; v < N; v += blockDim.x) a.side_out[I.out + v] = cur[v];
    __syncthreads();
    return x.st->warn ? 1 : 0;
}

}  // namespace

__global__ void __launch_bounds__(kBT, 1) k_batch_bisect(BArgs a) {
    extern __shared__ __align__(16) char smem[];
    __shared__ DLevel lev[kMaxLev];
    __shared__ int s_inst;
    for (;;) {
        if (threadIdx.x == 0) s_inst = atomicAdd(a.next, 1);
        __syncthreads();
        const int i = s_inst;
        __syncthreads();
        if (i >= a.n) break;
        Ctx x;
        x.ar.base = a.arena + (size_t)blockIdx.x * a.arena_bytes;
        x.ar.cap = a.arena_bytes;
        x.ar.top = 0;
        // a misaligned arena would fault on its 8-byte arrays: defer instead of touching it
        x.ar.overflow = ((uintptr_t)x.ar.base & 255) != 0;
        x.smem = smem;
        x.status = a.status;
        const BInst I = a.inst[i];
        const int st = blk_bisect(x, a, I, lev);
        if (threadIdx.x == 0) a.inst[i].status = st;
        __syncthreads();
    }
}

// ------------------------------------------------------------------ host side
// Upper bound of the arena bytes an instance may need (level store over all levels plus
// scratch); instances above the arena given to the launch are deferred by the device.
size_t block_arena_estimate(int64_t N, int64_t E, int64_t P) {
    const int64_t level0 = 4 * (E + 1) + 4 * E + 4 * P + 4 * N + 4 * (N + 1) + 4 * P + 8 * N;
    const int64_t scratch = E * (4 * 4 + 8 + 8) + N * (4 * 3 + 8 + 4 + 2) + 4 * P + 64 * 1024;
    return (size_t)(scratch + 5 * level0 + (4 << 20));
}

bool block_eligible(int64_t N, int64_t E, int64_t P, int k) {
    (void)E;
    return k == 2 && N <= (1 << 18) && P <= (1 << 24);
}

// Runs the eligible instances of a batch with the persistent kernel.  inst[] descriptors are
// completed with offsets; returns per-instance status (2 = deferred to the caller).
void run_block_batch(std::vector<BInst> &inst, const std::vector<const int32_t *> &hoff,
                     const std::vector<const int32_t *> &pins, const std::vector<const int32_t *> &nw,
                     const std::vector<const int32_t *> &hw, std::vector<std::vector<uint8_t>> &sides,
                     cudaStream_t s) {
    const int n = (int)inst.size();
    if (n == 0) return;
    const bool timing = std::getenv("BIPART_TIMING") != nullptr;
    auto t_host0 = std::chrono::steady_clock::now();
    int dev = 0, sms = 0;
    BP_CUDA(cudaGetDevice(&dev));
    BP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    static bool attr = false;
    if (!attr) {
        BP_CUDA(cudaFuncSetAttribute(k_batch_bisect, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kSmemBytes));
        attr = true;
    }
    int per_sm = 0;
    BP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_bisect, kBT, kSmemBytes));
    per_sm = std::max(per_sm, 1);
    // concatenated inputs
    int64_t sh = 0, sp = 0, sn = 0, sw = 0;
    size_t arena = 0;
    for (int i = 0; i < n; ++i) {
        BInst &I = inst[i];
        I.hoff = sh;
        I.pins = sp;
        I.nw = nw[i] ? sn : -1;
        I.hw = hw[i] ? sw : -1;
        I.out = sn;
        sh += I.E + 1;
        sp += I.P;
        sn += I.N;
        if (hw[i]) sw += I.E;
        arena = std::max(arena, block_arena_estimate(I.N, I.E, I.P));
    }
    // optional override (tuning, and tests of the deferral path): arena bytes per block in MiB
    if (const char *env = std::getenv("BIPART_BLOCK_ARENA_MB")) {
        long long mb = std::atoll(env);
        if (mb > 0) arena = (size_t)mb << 20;
    }
    // every block's arena must start on a 256-byte boundary (8-byte arrays are carved from it)
    arena = (arena + 255) & ~size_t(255);
    std::vector<int> h_hoff((size_t)sh), h_pins((size_t)std::max<int64_t>(sp, 1));
    std::vector<int> h_nw((size_t)std::max<int64_t>(sn, 1)), h_hw((size_t)std::max<int64_t>(sw, 1));
    for (int i = 0; i < n; ++i) {
        const BInst &I = inst[i];
        std::copy(hoff[i], hoff[i] + I.E + 1, h_hoff.begin() + I.hoff);
        std::copy(pins[i], pins[i] + I.P, h_pins.begin() + I.pins);
        if (nw[i]) std::copy(nw[i], nw[i] + I.N, h_nw.begin() + I.nw);
        if (hw[i]) std::copy(hw[i], hw[i] + I.E, h_hw.begin() + I.hw);
    }
    const int blocks = std::min(n, sms * per_sm);
    Buf b_inst, b_hoff, b_pins, b_nw, b_hw, b_side, b_arena, b_misc;
    BInst *d_inst = (BInst *)b_inst.ensure(sizeof(BInst) * (size_t)n, s);
    int *d_hoff = (int *)b_hoff.ensure(sizeof(int) * (size_t)sh, s);
    int *d_pins = (int *)b_pins.ensure(sizeof(int) * h_pins.size(), s);
    int *d_nw = (int *)b_nw.ensure(sizeof(int) * h_nw.size(), s);
    int *d_hw = (int *)b_hw.ensure(sizeof(int) * h_hw.size(), s);
    uint8_t *d_side = (uint8_t *)b_side.ensure((size_t)std::max<int64_t>(sn, 1), s);
    char *d_arena = (char *)b_arena.ensure(arena * (size_t)blocks, s);
    int *d_misc = (int *)b_misc.ensure(64, s);
    BP_CUDA(cudaMemcpyAsync(d_inst, inst.data(), sizeof(BInst) * (size_t)n, cudaMemcpyHostToDevice, s));
    BP_CUDA(cudaMemcpyAsync(d_hoff, h_hoff.data(), sizeof(int) * (size_t)sh, cudaMemcpyHostToDevice, s));
    BP_CUDA(cudaMemcpyAsync(d_pins, h_pins.data(), sizeof(int) * h_pins.size(), cudaMemcpyHostToDevice, s));
    BP_CUDA(cudaMemcpyAsync(d_nw, h_nw.data(), sizeof(int) * h_nw.size(), cudaMemcpyHostToDevice, s));
    BP_CUDA(cudaMemcpyAsync(d_hw, h_hw.data(), sizeof(int) * h_hw.size(), cudaMemcpyHostToDevice, s));
    BP_CUDA(cudaMemsetAsync(d_misc, 0, 64, s));
    BArgs a{d_inst, n, d_misc, d_hoff, d_pins, d_nw, d_hw, d_side, d_arena, arena,
            reinterpret_cast<uint32_t *>(d_misc + 8)};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (timing) {
        cudaEventCreate(&ev0);
        cudaEventCreate(&ev1);
        cudaEventRecord(ev0, s);
    }
    k_batch_bisect<<<blocks, kBT, kSmemBytes, s>>>(a);
    BP_LAUNCH();
    if (timing) cudaEventRecord(ev1, s);
    std::vector<uint8_t> h_side((size_t)std::max<int64_t>(sn, 1));
    BP_CUDA(cudaMemcpyAsync(inst.data(), d_inst, sizeof(BInst) * (size_t)n, cudaMemcpyDeviceToHost, s));
    BP_CUDA(cudaMemcpyAsync(h_side.data(), d_side, (size_t)std::max<int64_t>(sn, 1), cudaMemcpyDeviceToHost, s));
    uint32_t dst = 0;
    BP_CUDA(cudaMemcpyAsync(&dst, d_misc + 8, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    BP_CUDA(cudaStreamSynchronize(s));
    if (timing) {
        float ms = 0;
        cudaEventElapsedTime(&ms, ev0, ev1);
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        const double host_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_host0).count();
        std::fprintf(stderr, "[bipart] block batch: %d instances, %d blocks x %d threads, arena %.1f MiB/block, kernel %.2f ms, total %.2f ms\n",
                     n, blocks, kBT, arena / 1048576.0, ms, host_ms);
    }
    if (dst & DEV_TIMEOUT) throw Fail{BIPART_ERR_TIMEOUT, "a bounded device loop expired in the batch kernel"};
    sides.resize(n);
    for (int i = 0; i < n; ++i)
        sides[i].assign(h_side.begin() + inst[i].out, h_side.begin() + inst[i].out + inst[i].N);
}

}  // namespace bp
