// Coarsening on sm_103a: Algorithm 1 (matching) and Algorithm 2 (merge, singleton attach,
// contraction) of Sec. 3.1, plus the level-0 normalisation and the node -> hyperedge incidence.
//
// Per level, with N nodes, E hyperedges and P pins:
//   k_level_init     hkey[e] = priority(e) << 32 | mix32(e), matching accumulators reset
//                    (Alg. 1, Table 1; runs inside the previous level's incidence fill)
//   k_match_min      per node, the smallest hkey over its hyperedges (64-bit atomicMin)  (Alg. 1)
//   k_match_set      match[v], and the size / weight of every matched set S(e) by integer
//                    atomics (order-independent)                                      (Alg. 1)
//   k_single_best    per singleton set, the lightest step-1 merged node among its pins  (Alg. 2)
//   k_group          the final groups, smallest member id of every group              (Alg. 2)
//   scan             coarse ids in ascending order of the smallest member          (reading C8)
//   k_cmap           cmap[v] and coarse node weights
//   seg_unique       per hyperedge: pins mapped through cmap, sorted, de-duplicated in three
//                    tiers (thread, warp, block)                                      (Alg. 2)
//   scan + k_seg_copy   compaction of the hyperedges with >= 2 distinct pins, coarse degrees
//   incidence        node -> hyperedge CSR of the coarse level (offsets scan + fill)
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "coarsen_dev.cuh"
#include "lb.cuh"
#include "scan.cuh"

namespace bp {

namespace {

constexpr int kBlock = 256;
constexpr int kBigThreads = 512;  // block tier: one block per hyperedge
constexpr int kFuseTiersPins = 2'000'000;  // mid and big tiers share a launch up to this many pins

inline int grid_for(int64_t n, int per_block = kBlock, int cap = 152 * 16) {
    int64_t b = (n + per_block - 1) / per_block;
    if (b < 1) b = 1;
    return (int)std::min<int64_t>(b, cap);
}

}  // namespace

// Grid kernels: one launch per phase (device code in coarsen_dev.cuh).
template <bool MAP>
__global__ void __launch_bounds__(kBlock)
k_seg_small(int E, const int *__restrict__ hoff, const int *__restrict__ pins,
            const int *__restrict__ cmap, int *__restrict__ scratch, int *__restrict__ cnt,
            int *__restrict__ mid_list, int *__restrict__ big_list, int *__restrict__ counters) {
    d_seg_small<MAP>(GridTeam(), E, hoff, pins, cmap, scratch, cnt, mid_list, big_list, counters,
                     kGridMidDeg);
}

template <bool MAP>
__global__ void __launch_bounds__(kBlock)
k_seg_mid(const int *__restrict__ hoff, const int *__restrict__ pins, const int *__restrict__ cmap,
          int *__restrict__ scratch, int *__restrict__ cnt, const int *__restrict__ list,
          const int *__restrict__ counters) {
    d_seg_mid<MAP, GridTeam, kGridMidDeg / 32>(GridTeam(), hoff, pins, cmap, scratch, cnt, list, counters);
}

template <bool MAP>
__global__ void __launch_bounds__(kBigThreads, 3)
k_seg_big(const int *__restrict__ hoff, const int *__restrict__ pins, const int *__restrict__ cmap,
          int *__restrict__ scratch, int *__restrict__ cnt, const int *__restrict__ list,
          const int *__restrict__ counters) {
    __shared__ uint32_t bits[kBigWords];
    d_seg_big<MAP>(GridTeam(), hoff, pins, cmap, scratch, cnt, list, counters, bits);
}

// Mid and big tiers in one launch (small levels, where the launch is the larger cost; on large
// levels the big tier's blocks would hold the GPU while the mid tier waits): blocks [0, nbig) take the big list (one block per
// hyperedge, shared-memory bitmap), the others the mid list (one warp per hyperedge).  The two
// lists are disjoint, so the tiers run side by side.
template <bool MAP>
__global__ void __launch_bounds__(kBigThreads)
k_seg_midbig(int nbig, const int *__restrict__ hoff, const int *__restrict__ pins,
             const int *__restrict__ cmap, int *__restrict__ scratch, int *__restrict__ cnt,
             const int *__restrict__ mid_list, const int *__restrict__ big_list,
             const int *__restrict__ counters) {
    __shared__ uint32_t bits[kBigWords];
    if ((int)blockIdx.x < nbig)
        d_seg_big<MAP>(SubGridTeam{0, nbig}, hoff, pins, cmap, scratch, cnt, big_list, counters, bits);
    else
        d_seg_mid<MAP, SubGridTeam, kGridMidDeg / 32>(SubGridTeam{nbig, (int)gridDim.x - nbig}, hoff, pins, cmap, scratch, cnt, mid_list,
                       counters);
}

__global__ void __launch_bounds__(kLbBlock)
k_seg_copy(int E, int P, const int *__restrict__ hoff, const int *__restrict__ scratch,
           const int *__restrict__ cnt, const int *__restrict__ emap,
           const int *__restrict__ hoff_out, int *__restrict__ pins_out, int *__restrict__ deg,
           const int *__restrict__ ts) {
    d_seg_copy(GridTeam(), E, P, hoff, scratch, cnt, emap, hoff_out, pins_out, deg, ts);
}

// Start of a level's coarsening: hyperedge keys (Algorithm 1, Table 1), and every
// per-hyperedge / per-node accumulator of the matching reset in the same pass (ssize, sweight,
// rep, best; nkey).  Runs alone, or as the second job of the previous level's incidence fill.
struct LevelInit {
    int E = 0, N = 0, policy = 0;
    const int *hoff = nullptr, *hw = nullptr;
    unsigned long long *hkey = nullptr, *best = nullptr, *nkey = nullptr;
    int *ssize = nullptr, *sweight = nullptr;
    unsigned *rep = nullptr;
};

__device__ __forceinline__ void d_level_init(const LevelInit &li) {
    d_hedge_key(GridTeam(), li.E, li.policy, li.hoff, li.hw, li.hkey);
    const int n = li.E > li.N ? li.E : li.N;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (i < li.E) {
            li.ssize[i] = 0;
            li.sweight[i] = 0;
            li.rep[i] = ~0u;
            li.best[i] = ~0ull;
        }
        if (i < li.N) li.nkey[i] = ~0ull;
    }
}

// Coarse levels with at most kPrivNodes nodes count degrees and claim incidence positions in
// block-private shared-memory counters: few nodes means many pins per node, and one global
// atomic per pin would serialise on the heaviest nodes.  Each block merges its counts with one
// global atomic per node it touched.
constexpr int kPrivNodes = 24576;
constexpr int kPrivBlock = 1024;  // large blocks: clearing and merging N counters is per block

__global__ void __launch_bounds__(kPrivBlock)
k_seg_copy_priv(int E, int P, int N, const int *__restrict__ hoff, const int *__restrict__ scratch,
                const int *__restrict__ cnt, const int *__restrict__ emap,
                const int *__restrict__ hoff_out, int *__restrict__ pins_out, int *__restrict__ deg,
                const int *__restrict__ ts) {
    extern __shared__ int s_cnt[];
    for (int v = threadIdx.x; v < N; v += blockDim.x) s_cnt[v] = 0;
    __syncthreads();
    lb_runs(
        hoff, E, P,
        [&](int e, int a, int b) {
            const int ee = emap[e];
            if (ee < 0) return;
            const int base = hoff[e], c = cnt[e], o = hoff_out[ee];
            const int stop = base + c < b ? base + c : b;
            for (int i = a; i < stop; ++i) {
                const int v = scratch[i];
                pins_out[o + (i - base)] = v;
                atomicAdd(s_cnt + v, 1);
            }
        },
        GridTeam(), ts);
    __syncthreads();
    for (int v = threadIdx.x; v < N; v += blockDim.x) {
        const int c = s_cnt[v];
        if (c) atomicAdd(deg + v, c);
    }
}

// Pass 1 counts this block's pins per node, one global atomic per touched node reserves the
// block's range, pass 2 hands out positions inside the range by shared-memory atomics.  Both
// passes visit the same tiles.
__global__ void __launch_bounds__(kPrivBlock, 2)
k_fill_adj_priv(int E, int P, int N, const int *__restrict__ hoff, const int *__restrict__ pins,
                int *__restrict__ cursor, int *__restrict__ nadj, const int *__restrict__ ts,
                LevelInit next) {
    d_level_init(next);  // the next coarsening's keys and resets (E = N = 0: nothing)
    extern __shared__ int s_cnt[];
    for (int v = threadIdx.x; v < N; v += blockDim.x) s_cnt[v] = 0;
    __syncthreads();
    const int tile = blockDim.x * kLbItems;
    for (int64_t t0 = (int64_t)blockIdx.x * tile; t0 < P; t0 += (int64_t)gridDim.x * tile) {
        const int j1 = (int)(t0 + tile < P ? t0 + tile : P);
        for (int j = (int)t0 + threadIdx.x; j < j1; j += blockDim.x) atomicAdd(s_cnt + pins[j], 1);
    }
    __syncthreads();
    // each touched node's range reserved in the global cursor, eight nodes' atomics in flight at
    // once (their returns are stored only after all eight are issued)
    for (int v0 = threadIdx.x; v0 < N; v0 += 8 * blockDim.x) {
        int c[8], r[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int v = v0 + k * (int)blockDim.x;
            c[k] = v < N ? s_cnt[v] : 0;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) r[k] = c[k] ? atomicAdd(cursor + v0 + k * (int)blockDim.x, c[k]) : 0;
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (c[k]) s_cnt[v0 + k * (int)blockDim.x] = r[k];
    }
    __syncthreads();
    d_fill_adj_with(GridTeam(), E, P, hoff, pins, nadj, [&](int v) { return atomicAdd(s_cnt + v, 1); }, ts);
}

// Blocks for the private-counter kernels: one tile of kPrivBlock * kLbItems pins each, at most
// two blocks per SM (up to 96 KB of counters each); blocks loop over further tiles.
inline int priv_grid(int P) {
    int64_t b = ((int64_t)P + kPrivBlock * kLbItems - 1) / (kPrivBlock * kLbItems);
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 2 * 152));
}

__global__ void k_fill(int n, int val, int *__restrict__ a) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = val;
}

__global__ void __launch_bounds__(kLbBlock, 6)
k_fill_adj(int E, int P, const int *__restrict__ hoff, const int *__restrict__ pins,
           int *__restrict__ cursor, int *__restrict__ nadj, const int *__restrict__ ts,
           LevelInit next) {
    d_fill_adj(GridTeam(), E, P, hoff, pins, cursor, nadj, ts);
    d_level_init(next);
}

__global__ void k_level_init(LevelInit li) { d_level_init(li); }

__global__ void __launch_bounds__(kLbBlock)
k_match_min(int N, int P, const int *__restrict__ noff, const int *__restrict__ nadj,
            const unsigned long long *__restrict__ hkey, unsigned long long *__restrict__ nkey,
            const int *__restrict__ ts, bool warp_min) {
    d_match_min(GridTeam(), N, P, noff, nadj, hkey, nkey, ts, warp_min);
}

__global__ void __launch_bounds__(kBlock)
k_match_set(int N, const unsigned long long *__restrict__ nkey, const int *__restrict__ nw,
            int *__restrict__ match, int *__restrict__ ssize, int *__restrict__ sweight) {
    d_match_set(GridTeam(), N, nkey, nw, match, ssize, sweight);
}

__global__ void __launch_bounds__(kLbBlock)
k_single_best(int E, int P, const int *__restrict__ hoff, const int *__restrict__ pins,
              const int *__restrict__ match, const int *__restrict__ ssize,
              const int *__restrict__ sweight, unsigned long long *__restrict__ best,
              const int *__restrict__ ts) {
    d_single_best(GridTeam(), E, P, hoff, pins, match, ssize, sweight, best, ts);
}

// Groups, plus the coarse level's accumulators cleared for later phases of this level: node
// weights (k_cmap), degree counters (contraction copy) for up to N coarse nodes, and the two
// hyperedge list counters of seg_unique.
__global__ void __launch_bounds__(kBlock)
k_group(int N, const int *__restrict__ match, const int *__restrict__ ssize,
        const unsigned long long *__restrict__ best, int *__restrict__ grp,
        unsigned *__restrict__ rep, int *__restrict__ cw, int *__restrict__ deg,
        int *__restrict__ list_counts) {
    d_group(GridTeam(), N, match, ssize, best, grp, rep);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        cw[i] = 0;
        deg[i] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x < 2) list_counts[threadIdx.x] = 0;
}

__global__ void k_cmap(int N, const int *__restrict__ grp, const int *__restrict__ gcid,
                       const int *__restrict__ nw, int *__restrict__ cmap, int *__restrict__ cw) {
    d_cmap(GridTeam(), N, grp, gcid, nw, cmap, cw);
}

// ------------------------------------------------------------------ parallel-net merging
// Reading M1 (a switch, off by default): after contraction, hyperedges with the same sorted pin
// list become the smallest-id one with the summed weight.  Groups are found without sorting:
// a fingerprint per list (sum of SplitMix64-mixed (position, pin) terms, so the partial sums can
// be combined in any order), an open-addressing table giving the smallest id per fingerprint,
// an exact list comparison against it, and an exact scan for the (practically never) hyperedges
// whose fingerprint collided with a different list.

__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_merge_clear(int E, int T, unsigned long long *__restrict__ fp,
                              int *__restrict__ wsum, unsigned long long *__restrict__ tkey,
                              int *__restrict__ tmin, unsigned *__restrict__ flag) {
    const int n = E > T ? E : T;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (i < E) {
            fp[i] = 0ull;
            wsum[i] = 0;
        }
        if (i < T) {
            tkey[i] = 0ull;
            tmin[i] = INT_MAX;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *flag = 0u;
}

__global__ void __launch_bounds__(kLbBlock)
k_merge_fp(int E, int P, const int *__restrict__ hoff, const int *__restrict__ scratch,
           const int *__restrict__ cnt, unsigned long long *__restrict__ fp,
           const int *__restrict__ ts) {
    lb_runs(
        hoff, E, P,
        [&](int e, int a, int b) {
            const int c = cnt[e];
            if (c < 2) return;
            const int base = hoff[e];
            const int stop = base + c < b ? base + c : b;
            unsigned long long acc = 0;
            for (int i = a; i < stop; ++i)
                acc += splitmix64(((uint64_t)(uint32_t)(i - base) << 32) | (uint32_t)scratch[i]);
            if (stop > a) atomicAdd(fp + e, acc);
        },
        GridTeam(), ts);
}

// Final key of a kept list (its length mixed in; 0 marks an empty table slot).
__device__ __forceinline__ unsigned long long merge_key(unsigned long long f, int c) {
    unsigned long long k = f ^ splitmix64(0xFFFFFFFF00000000ull | (uint32_t)c);
    return k ? k : 1ull;
}

__global__ void k_merge_insert(int E, int T, const int *__restrict__ cnt,
                               unsigned long long *__restrict__ fp,
                               unsigned long long *__restrict__ tkey, int *__restrict__ tmin) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
        const int c = cnt[e];
        if (c < 2) continue;
        const unsigned long long k = merge_key(fp[e], c);
        fp[e] = k;
        unsigned slot = (unsigned)(k & (unsigned long long)(T - 1));
        for (int probe = 0; probe < T; ++probe) {  // the table is at least twice the key count
            const unsigned long long prev = atomicCAS(tkey + slot, 0ull, k);
            if (prev == 0ull || prev == k) {
                atomicMin(tmin + slot, e);
                break;
            }
            slot = (slot + 1) & (unsigned)(T - 1);
        }
    }
}

__device__ __forceinline__ bool same_list(const int *scratch, const int *hoff, int a, int b, int c) {
    const int *la = scratch + hoff[a], *lb = scratch + hoff[b];
    for (int i = 0; i < c; ++i)
        if (la[i] != lb[i]) return false;
    return true;
}

// rep[e] = smallest id with e's list; -1 - e when the fingerprint's smallest id has another list
// (a collision, settled by k_merge_exact).
__global__ void k_merge_rep(int E, int T, const int *__restrict__ hoff, const int *__restrict__ scratch,
                            const int *__restrict__ cnt, const unsigned long long *__restrict__ fp,
                            const unsigned long long *__restrict__ tkey, const int *__restrict__ tmin,
                            int *__restrict__ rep, unsigned *__restrict__ flag) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
        const int c = cnt[e];
        if (c < 2) {
            rep[e] = e;
            continue;
        }
        const unsigned long long k = fp[e];
        unsigned slot = (unsigned)(k & (unsigned long long)(T - 1));
        int r = e;
        for (int probe = 0; probe < T; ++probe) {
            if (tkey[slot] == k) {
                r = tmin[slot];
                break;
            }
            slot = (slot + 1) & (unsigned)(T - 1);
        }
        if (r == e || (cnt[r] == c && same_list(scratch, hoff, r, e, c))) {
            rep[e] = r;
        } else {
            rep[e] = -1 - e;
            atomicOr(flag, 1u);
        }
    }
}

__global__ void k_merge_exact(int E, const int *__restrict__ hoff, const int *__restrict__ scratch,
                              const int *__restrict__ cnt, const unsigned long long *__restrict__ fp,
                              int *__restrict__ rep, const unsigned *__restrict__ flag) {
    if (*flag == 0u) return;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
        if (rep[e] >= 0) continue;
        const int c = cnt[e];
        int r = e;
        for (int q = 0; q < e; ++q) {
            if (cnt[q] == c && fp[q] == fp[e] && same_list(scratch, hoff, q, e, c)) {
                r = q;
                break;
            }
        }
        rep[e] = r;
    }
}

__global__ void k_merge_weights(int E, const int *__restrict__ cnt, const int *__restrict__ hw,
                                const int *__restrict__ rep, int *__restrict__ wsum) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x)
        if (cnt[e] >= 2) atomicAdd(wsum + rep[e], hw ? hw[e] : 1);
}

// ------------------------------------------------------------------ host side
namespace {

// Per hyperedge: pins mapped through `map` (identity when null), sorted and de-duplicated into
// scratch at the hyperedge's own offset; cnt[e] = number of distinct values.
// `counters_zero`: small[0..1] are known to be zero already (else they are cleared here).
void seg_unique(bipart_graph *g, int32_t E, int32_t P, const int *hoff, const int *pins,
                const int *map, int *scratch, int *cnt, bool counters_zero) {
    cudaStream_t s = g->stream;
    Work &w = g->w;
    int *mid = (int *)w.e_c.ensure(sizeof(int) * (size_t)std::max(E, 1), s);
    int *big = (int *)w.e_d.ensure(sizeof(int) * (size_t)std::max(E, 1), s);
    int *small = w.small.as<int>();  // [0] mid count, [1] big count
    if (E == 0) return;
    if (!counters_zero) BP_CUDA(cudaMemsetAsync(small, 0, 2 * sizeof(int), s));
    // reads hoff, pins, map gathers; writes distinct pins (<= P) and counts
    ProfScope ps("contract_unique", 8.0 * E + 4.0 * P * (map ? 3 : 2), s);
    if (map) k_seg_small<true><<<grid_for(E), kBlock, 0, s>>>(E, hoff, pins, map, scratch, cnt, mid, big, small);
    else k_seg_small<false><<<grid_for(E), kBlock, 0, s>>>(E, hoff, pins, map, scratch, cnt, mid, big, small);
    BP_LAUNCH();
    // warps for the mid tier (at most one per 9 pins), blocks for the big tier (at most one per
    // kGridMidDeg + 1 pins); the list lengths are only known on the device
    const int mid_warps = std::max(1, std::min(152 * 16 * (kBlock / 32), P / (kSmallDeg + 1) + 1));
    const int nbig = std::max(1, std::min(152 * 3, P / (kGridMidDeg + 1) + 1));
    if (P <= kFuseTiersPins) {
        const int nmid = ceil_div_i(mid_warps, kBigThreads / 32);
        if (map) k_seg_midbig<true><<<nbig + nmid, kBigThreads, 0, s>>>(nbig, hoff, pins, map, scratch, cnt, mid, big, small);
        else k_seg_midbig<false><<<nbig + nmid, kBigThreads, 0, s>>>(nbig, hoff, pins, map, scratch, cnt, mid, big, small);
        BP_LAUNCH();
    } else {
        const int mid_grid = ceil_div_i(mid_warps, kBlock / 32);
        if (map) k_seg_mid<true><<<mid_grid, kBlock, 0, s>>>(hoff, pins, map, scratch, cnt, mid, small);
        else k_seg_mid<false><<<mid_grid, kBlock, 0, s>>>(hoff, pins, map, scratch, cnt, mid, small);
        BP_LAUNCH();
        if (map) k_seg_big<true><<<nbig, kBigThreads, 0, s>>>(hoff, pins, map, scratch, cnt, big, small);
        else k_seg_big<false><<<nbig, kBigThreads, 0, s>>>(hoff, pins, map, scratch, cnt, big, small);
        BP_LAUNCH();
    }
}

// Sorted-unique of every hyperedge's (mapped) pins into the coarse CSR of `c`.
// Sets c.E and c.P.  `map` null means identity (level-0 normalisation).
// sizes: two device ints receiving {E', P'}; ts_in: tile starts of the input CSR (or null).
// n_slot (or null): the device int holding c.N, read in the same round trip as E' and P'
// (otherwise c.N must be set by the caller).
void contract(bipart_graph *g, int32_t E, int32_t P, const int *hoff, const int *pins,
              const int *hw, const int *map, Level &c, int *deg, bool counters_zero, int32_t *sizes,
              const int *ts_in, bool merge, const int32_t *n_slot) {
    cudaStream_t s = g->stream;
    Work &w = g->w;
    int *scratch = (int *)w.p_a.ensure(sizeof(int) * (size_t)std::max(P, 1), s);
    int *cnt = (int *)w.e_a.ensure(sizeof(int) * (size_t)std::max(E, 1), s);
    int *emap = (int *)w.e_b.ensure(sizeof(int) * (size_t)std::max(E, 1), s);
    int *small = w.small.as<int>();
    seg_unique(g, E, P, hoff, pins, map, scratch, cnt, counters_zero);
    c.b_hoff.ensure(sizeof(int) * ((size_t)E + 1), s);
    c.b_pins.ensure(sizeof(int) * (size_t)std::max(P, 1), s);
    c.b_tsh.ensure(sizeof(int) * ((size_t)P / kTsGran + 2), s);
    merge = merge && E > 1;
    bool unit = (hw == nullptr) && !merge;  // merged groups carry summed weights
    if (!unit) c.b_hw.ensure(sizeof(int) * (size_t)std::max(E, 1), s);
    c.unit_hw = unit;
    int *rep = nullptr, *wsum = nullptr;
    if (merge) {
        int T = 1;
        while (T < 2 * E) T <<= 1;
        auto *fp = (unsigned long long *)w.m_fp.ensure(sizeof(uint64_t) * (size_t)E, s);
        auto *tkey = (unsigned long long *)w.m_tkey.ensure(sizeof(uint64_t) * (size_t)T, s);
        int *tmin = (int *)w.m_tmin.ensure(sizeof(int) * (size_t)T, s);
        rep = (int *)w.m_rep.ensure(sizeof(int) * (size_t)E, s);
        wsum = (int *)w.m_wsum.ensure(sizeof(int) * (size_t)E, s);
        unsigned *flag = reinterpret_cast<unsigned *>(small + 6);
        ProfScope ps("merge_parallel", 8.0 * P + 48.0 * E + 12.0 * T, s);
        k_merge_clear<<<grid_for(std::max(E, T)), kBlock, 0, s>>>(E, T, fp, wsum, tkey, tmin, flag);
        BP_LAUNCH();
        k_merge_fp<<<lb_grid(P), kLbBlock, 0, s>>>(E, P, hoff, scratch, cnt, fp, ts_in);
        BP_LAUNCH();
        k_merge_insert<<<grid_for(E), kBlock, 0, s>>>(E, T, cnt, fp, tkey, tmin);
        BP_LAUNCH();
        k_merge_rep<<<grid_for(E), kBlock, 0, s>>>(E, T, hoff, scratch, cnt, fp, tkey, tmin, rep, flag);
        BP_LAUNCH();
        k_merge_exact<<<grid_for(E), kBlock, 0, s>>>(E, hoff, scratch, cnt, fp, rep, flag);
        BP_LAUNCH();
        k_merge_weights<<<grid_for(E), kBlock, 0, s>>>(E, cnt, hw, rep, wsum);
        BP_LAUNCH();
    }
    if (E > 0) {
        CompactOut out{E, hw, c.hoff(), unit ? nullptr : c.b_hw.as<int>(), emap, sizes, c.tsh(), wsum};
        {
            ProfScope ps("contract_offsets", 16.0 * E, s);
            scan(E, CompactIn{cnt, rep}, out, w.scan, dev_status(g), s);
        }
        const int32_t *ptr[3] = {sizes, sizes + 1, n_slot};
        int32_t v[3];
        read_i32s(g, n_slot ? 3 : 2, ptr, v);
        c.E = v[0];
        c.P = v[1];
        if (n_slot) c.N = v[2];
        {
            // scratch, coarse pins, degree atomics, per-hyperedge offsets
            ProfScope ps("contract_copy", 12.0 * P + 12.0 * E, s);
            if (c.N <= kPrivNodes)
                k_seg_copy_priv<<<priv_grid(P), kPrivBlock, sizeof(int) * (size_t)std::max(c.N, 1), s>>>(
                    E, P, c.N, hoff, scratch, cnt, emap, c.hoff(), c.pins(), deg, ts_in);
            else
                k_seg_copy<<<lb_grid(P), kLbBlock, 0, s>>>(E, P, hoff, scratch, cnt, emap, c.hoff(), c.pins(), deg,
                                                           ts_in);
            BP_LAUNCH();
        }
    } else {
        BP_CUDA(cudaMemsetAsync(c.hoff(), 0, sizeof(int), s));
        c.E = 0;
        c.P = 0;
        if (n_slot) c.N = read_i32(g, n_slot);
    }
}

}  // namespace

void distinct_counts(bipart_graph *g, Level &L, const int *d_map, int *cnt) {
    int *scratch = (int *)g->w.p_a.ensure(sizeof(int) * (size_t)std::max(L.P, 1), g->stream);
    seg_unique(g, L.E, L.P, L.hoff(), L.pins(), d_map, scratch, cnt, false);
}

// Node -> hyperedge incidence of a level whose degrees were counted by its contraction
// (deg[N], in the per-node scratch n_a).
void build_incidence_and_init(bipart_graph *g, Level &L, const LevelInit &next);

void build_incidence(bipart_graph *g, Level &L) { build_incidence_and_init(g, L, LevelInit()); }

// The incidence fill of L also runs `next` (the keys and resets of L's own coarsening).
void build_incidence_and_init(bipart_graph *g, Level &L, const LevelInit &next) {
    cudaStream_t s = g->stream;
    Work &w = g->w;
    L.b_noff.ensure(sizeof(int) * ((size_t)L.N + 1), s);
    L.b_nadj.ensure(sizeof(int) * (size_t)std::max(L.P, 1), s);
    if (L.N == 0) {
        BP_CUDA(cudaMemsetAsync(L.noff(), 0, sizeof(int), s));
        return;
    }
    int *deg = w.n_a.as<int>();
    int *cursor = (int *)w.n_b.ensure(sizeof(int) * (size_t)L.N, s);
    L.b_tsn.ensure(sizeof(int) * ((size_t)L.P / kTsGran + 2), s);
    {
        ProfScope ps("incidence_offsets", 12.0 * L.N, s);
        scan(L.N, DegIn{deg}, DegOut{L.N, L.noff(), cursor, L.tsn()}, w.scan,
             dev_status(g), s);
    }
    if (L.P > 0) {
        ProfScope ps("incidence_fill", 12.0 * L.P + 4.0 * L.E + 32.0 * next.E + 8.0 * next.N, s);
        if (L.N <= kPrivNodes)
            k_fill_adj_priv<<<priv_grid(L.P), kPrivBlock, sizeof(int) * (size_t)L.N, s>>>(
                L.E, L.P, L.N, L.hoff(), L.pins(), cursor, L.nadj(), L.tsh(), next);
        else
            k_fill_adj<<<lb_grid(L.P), kLbBlock, 0, s>>>(L.E, L.P, L.hoff(), L.pins(), cursor, L.nadj(),
                                                        L.tsh(), next);
        BP_LAUNCH();
    } else if (next.E > 0 || next.N > 0) {
        k_level_init<<<grid_for(std::max(next.E, next.N)), kBlock, 0, s>>>(next);
        BP_LAUNCH();
    }
}

// Zeroed degree counters for a level of N nodes (filled by the contraction's copy).
int *degree_counters(bipart_graph *g, int32_t N) {
    int *deg = (int *)g->w.n_a.ensure(sizeof(int) * (size_t)std::max(N, 1), g->stream);
    if (N > 0) BP_CUDA(cudaMemsetAsync(deg, 0, sizeof(int) * (size_t)N, g->stream));
    return deg;
}

void build_level0(bipart_graph *g, Level &L, int32_t N, int32_t E, int32_t P, const int32_t *d_hoff,
                  const int32_t *d_pins, const int32_t *d_nw, const int32_t *d_hw) {
    cudaStream_t s = g->stream;
    L.N = N;
    contract(g, E, P, d_hoff, d_pins, d_hw, nullptr, L, degree_counters(g, N), false,
             g->w.small.as<int32_t>() + 2, nullptr, false, nullptr);
    L.b_nw.ensure(sizeof(int) * (size_t)std::max(N, 1), s);
    if (d_nw) {
        BP_CUDA(cudaMemcpyAsync(L.nw(), d_nw, sizeof(int) * (size_t)N, cudaMemcpyDeviceToDevice, s));
    } else if (N > 0) {
        k_fill<<<grid_for(N), kBlock, 0, s>>>(N, 1, L.nw());
        BP_LAUNCH();
    }
    build_incidence(g, L);
    L.b_cmap.ensure(sizeof(int) * (size_t)std::max(N, 1), s);
    L.b_match.ensure(sizeof(int) * (size_t)std::max(N, 1), s);
}

bool coarsen_level(bipart_graph *g, Level &f, Level &c, int policy, int32_t *sizes, bool merge,
                   bool init_done, bool more_levels, int tail_new, int flags, bool *to_tail) {
    if (to_tail) *to_tail = false;
    cudaStream_t s = g->stream;
    Work &w = g->w;
    const int N = f.N, E = f.E;
    unsigned long long *hkey = (unsigned long long *)w.e_key.ensure(sizeof(uint64_t) * (size_t)std::max(E, 1), s);
    unsigned long long *best = (unsigned long long *)w.e_best.ensure(sizeof(uint64_t) * (size_t)std::max(E, 1), s);
    unsigned long long *nkey = (unsigned long long *)w.n_key.ensure(sizeof(uint64_t) * (size_t)std::max(N, 1), s);
    int *ssize = (int *)w.e_a.ensure(sizeof(int) * (size_t)std::max(E, 1), s);
    int *sweight = (int *)w.e_b.ensure(sizeof(int) * (size_t)std::max(E, 1), s);
    unsigned *rep = (unsigned *)w.e_c.ensure(sizeof(int) * (size_t)std::max(E, 1), s);
    int *gcid = (int *)w.e_d.ensure(sizeof(int) * (size_t)std::max(E, 1), s);
    int *grp = (int *)w.n_c.ensure(sizeof(int) * (size_t)std::max(N, 1), s);
    // the coarse level has at most N nodes: its weights and degree counters are sized (and
    // cleared by k_group) for N before N' is known
    int *deg = (int *)w.n_a.ensure(sizeof(int) * (size_t)std::max(N, 1), s);
    c.b_nw.ensure(sizeof(int) * (size_t)std::max(N, 1), s);
    int *small = w.small.as<int>();
    if ((N > 0 || E > 0) && !init_done) {
        ProfScope ps("hedge_key", 12.0 * E + (f.hw() ? 4.0 * E : 0.0) + 20.0 * E + 8.0 * N, s);
        LevelInit li;
        li.E = E; li.N = N; li.policy = policy; li.hoff = f.hoff(); li.hw = f.hw();
        li.hkey = hkey; li.best = best; li.nkey = nkey; li.ssize = ssize; li.sweight = sweight;
        li.rep = rep;
        k_level_init<<<grid_for(std::max(E, N)), kBlock, 0, s>>>(li);
        BP_LAUNCH();
    }
    if (N > 0) {
        if (f.P > 0) {
            // noff, nadj, 8-byte key gather per incidence, one 8-byte atomic per node run
            ProfScope ps("match_min", 4.0 * N + 12.0 * f.P + 8.0 * N, s);
            k_match_min<<<lb_grid(f.P), kLbBlock, 0, s>>>(N, f.P, f.noff(), f.nadj(), hkey, nkey, f.tsn(),
                                                           (int64_t)f.P > 64 * (int64_t)N);
            BP_LAUNCH();
        }
        {
            ProfScope ps("match_set", 24.0 * N, s);
            k_match_set<<<grid_for(N), kBlock, 0, s>>>(N, nkey, f.nw(), f.match(), ssize, sweight);
            BP_LAUNCH();
        }
        if (f.P > 0) {
            ProfScope ps("single_best", 4.0 * E + 4.0 * f.P, s);
            k_single_best<<<lb_grid(f.P), kLbBlock, 0, s>>>(E, f.P, f.hoff(), f.pins(), f.match(), ssize, sweight, best,
                                                            f.tsh());
            BP_LAUNCH();
        }
        {
            ProfScope ps("group", 20.0 * N + 8.0 * N, s);
            k_group<<<grid_for(N), kBlock, 0, s>>>(N, f.match(), ssize, best, grp, rep, c.nw(), deg, small);
            BP_LAUNCH();
        }
        {
            ProfScope ps("renumber", 12.0 * N, s);
            scan(N, RenumIn{grp, rep}, RenumOut{N, grp, f.cmap(), gcid, sizes},
                 w.scan, dev_status(g), s);
        }
    }
    // N' is read with the contraction's sizes (one host round trip for the three)
    c.N = 0;
    if (N > 0) {
        ProfScope ps("cmap", 24.0 * N, s);
        k_cmap<<<grid_for(N), kBlock, 0, s>>>(N, grp, gcid, f.nw(), f.cmap(), c.nw());
        BP_LAUNCH();
    }
    contract(g, E, f.P, f.hoff(), f.pins(), f.hw(), f.cmap(), c, deg, N > 0, sizes + 1, f.tsh(), merge,
             N > 0 ? sizes : nullptr);
    const int Nc = c.N;
    if (to_tail && tail_new >= 0 && c.N != f.N && tail_eligible(c, tail_new, flags)) {
        // the cluster tail takes over from c and reads only its hyperedge CSR
        c.b_cmap.ensure(sizeof(int) * (size_t)std::max(Nc, 1), s);
        c.b_match.ensure(sizeof(int) * (size_t)std::max(Nc, 1), s);
        *to_tail = true;
        return false;
    }
    // when c will be coarsened in turn (the stop rule of reading C11 lets it), its key and reset
    // pass rides along with its incidence fill
    const bool prep = more_levels && c.E > 0 && c.N != f.N;
    LevelInit next;
    if (prep) {
        next.E = c.E; next.N = c.N; next.policy = policy; next.hoff = c.hoff(); next.hw = c.hw();
        next.hkey = hkey; next.best = best; next.nkey = nkey; next.ssize = ssize;
        next.sweight = sweight; next.rep = rep;
    }
    build_incidence_and_init(g, c, next);
    c.b_cmap.ensure(sizeof(int) * (size_t)std::max(Nc, 1), s);
    c.b_match.ensure(sizeof(int) * (size_t)std::max(Nc, 1), s);
    return prep;
}

void coarsen_init() {
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, []() {
        const int bytes = (int)(sizeof(int) * kPrivNodes);
        err = cudaFuncSetAttribute(k_seg_copy_priv, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (err == cudaSuccess)
            err = cudaFuncSetAttribute(k_fill_adj_priv, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    });
    BP_CUDA(err);
}

}  // namespace bp
