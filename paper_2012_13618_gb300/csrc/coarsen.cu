// Coarsening on sm_103a: Algorithm 1 (matching) and Algorithm 2 (merge, singleton attach,
// contraction) of Sec. 3.1, plus the level-0 normalisation and the node -> hyperedge incidence.
//
// Per level, with N nodes, E hyperedges and P pins:
//   k_hedge_key      hkey[e] = priority(e) << 32 | mix32(e)                  (Alg. 1, Table 1)
//   k_match          match[v] = argmin of hkey over v's hyperedges, and the size / weight of
//                    every matched set S(e) by integer atomics (order-independent)   (Alg. 1)
//   k_group          singleton sets join the lightest merged node of their hyperedge
//                    (step-1 snapshot), smallest member id of every group          (Alg. 2)
//   scan             coarse ids in ascending order of the smallest member          (reading C8)
//   k_cmap           cmap[v] and coarse node weights
//   seg_unique       per hyperedge: pins mapped through cmap, sorted, de-duplicated   (Alg. 2)
//   scan + k_seg_copy   compaction of the hyperedges with >= 2 distinct pins
//   incidence        node -> hyperedge CSR of the coarse level (counting + fill)
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
constexpr int kSmallDeg = 8;      // hyperedges up to this degree: one thread each
constexpr int kMidDeg = 1024;     // up to this degree: one warp each (register bitonic sort)
constexpr int kBigThreads = 512;  // above: one block each (shared-memory bitmap windows)
constexpr int kBigWords = 8192;   // 32 KB bitmap = 262,144 ids per window

inline int grid_for(int64_t n, int per_block = kBlock, int cap = 152 * 16) {
    int64_t b = (n + per_block - 1) / per_block;
    if (b < 1) b = 1;
    return (int)std::min<int64_t>(b, cap);
}

// ------------------------------------------------------------------ small fixed sorting network
template <int n>
__device__ __forceinline__ void sort_net(int (&v)[n]) {
    // odd-even transposition sort: n rounds of compare-exchange on alternating pairs
#pragma unroll
    for (int r = 0; r < n; ++r) {
#pragma unroll
        for (int i = (r & 1); i + 1 < n; i += 2) {
            int a = v[i], b = v[i + 1];
            v[i] = min(a, b);
            v[i + 1] = max(a, b);
        }
    }
}

// ------------------------------------------------------------------ warp bitonic sort, R per lane
// Blocked layout: element index = lane * R + r.  Sorts 32 * R ints ascending.
template <int R>
__device__ __forceinline__ void warp_bitonic(int (&v)[R]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= 32 * R; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= R) {
                const int lj = j / R;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int idx = lane * R + r;
                    int p = __shfl_xor_sync(0xffffffffu, v[r], lj);
                    bool up = (idx & k) == 0;
                    bool lower = (idx & j) == 0;
                    v[r] = (lower == up) ? min(v[r], p) : max(v[r], p);
                }
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int r2 = r ^ j;
                    if (r2 > r) {
                        const int idx = lane * R + r;
                        bool up = (idx & k) == 0;
                        int a = v[r], b = v[r2];
                        int lo = min(a, b), hi = max(a, b);
                        v[r] = up ? lo : hi;
                        v[r2] = up ? hi : lo;
                    }
                }
            }
        }
    }
}

template <bool MAP>
__device__ __forceinline__ int mapped(const int *__restrict__ pins, const int *__restrict__ cmap,
                                      int i) {
    int p = __ldg(pins + i);
    return MAP ? __ldg(cmap + p) : p;
}

// Warp-cooperative sorted-unique of one hyperedge of degree d <= 32 * R.
template <int R, bool MAP>
__device__ __forceinline__ int warp_unique(const int *pins, const int *cmap, int a, int d,
                                           int *out) {
    const int lane = threadIdx.x & 31;
    int v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        int idx = lane * R + r;
        v[r] = idx < d ? mapped<MAP>(pins, cmap, a + idx) : INT_MAX;
    }
    warp_bitonic<R>(v);
    int prev_last = __shfl_up_sync(0xffffffffu, v[R - 1], 1);
    int keep_cnt = 0;
    bool keep[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        int idx = lane * R + r;
        int prev = r == 0 ? prev_last : v[r - 1];
        keep[r] = idx < d && (idx == 0 || v[r] != prev);
        keep_cnt += keep[r];
    }
    int incl = warp_inclusive_scan(keep_cnt);
    int pos = incl - keep_cnt;
#pragma unroll
    for (int r = 0; r < R; ++r)
        if (keep[r]) out[pos++] = v[r];
    return __shfl_sync(0xffffffffu, incl, 31);
}

}  // namespace

// Small tier: one thread per hyperedge of degree <= 8 (the vast majority); larger hyperedges are
// appended to the mid / big work lists (list order is irrelevant: every hyperedge writes only
// its own slots).
template <bool MAP>
__global__ void __launch_bounds__(kBlock)
k_seg_small(int E, const int *__restrict__ hoff, const int *__restrict__ pins,
            const int *__restrict__ cmap, int *__restrict__ scratch, int *__restrict__ cnt,
            int *__restrict__ mid_list, int *__restrict__ big_list, int *__restrict__ counters) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
        int a = hoff[e], d = hoff[e + 1] - a;
        if (d > kSmallDeg) {
            if (d > kMidDeg) big_list[atomicAdd(&counters[1], 1)] = e;
            else mid_list[atomicAdd(&counters[0], 1)] = e;
            continue;
        }
        int v[kSmallDeg];
#pragma unroll
        for (int k = 0; k < kSmallDeg; ++k) v[k] = k < d ? mapped<MAP>(pins, cmap, a + k) : INT_MAX;
        sort_net<kSmallDeg>(v);
        int m = 0;
#pragma unroll
        for (int k = 0; k < kSmallDeg; ++k) {
            bool keep = k < d && (k == 0 || v[k] != v[k - 1]);
            if (keep) scratch[a + m] = v[k];
            m += keep;
        }
        cnt[e] = m;
    }
}

// Mid tier: one warp per listed hyperedge (8 < d <= 1024), register bitonic sort.
template <bool MAP>
__global__ void __launch_bounds__(kBlock)
k_seg_mid(const int *__restrict__ hoff, const int *__restrict__ pins, const int *__restrict__ cmap,
          int *__restrict__ scratch, int *__restrict__ cnt, const int *__restrict__ list,
          const int *__restrict__ counters) {
    const int n = counters[0];
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < n; w += warps) {
        int e = list[w];
        int a = hoff[e], d = hoff[e + 1] - a;
        int *out = scratch + a;
        int m;
        if (d <= 32) m = warp_unique<1, MAP>(pins, cmap, a, d, out);
        else if (d <= 64) m = warp_unique<2, MAP>(pins, cmap, a, d, out);
        else if (d <= 128) m = warp_unique<4, MAP>(pins, cmap, a, d, out);
        else if (d <= 256) m = warp_unique<8, MAP>(pins, cmap, a, d, out);
        else if (d <= 512) m = warp_unique<16, MAP>(pins, cmap, a, d, out);
        else m = warp_unique<32, MAP>(pins, cmap, a, d, out);
        if (lane == 0) cnt[e] = m;
    }
}

// Big tier: one block per listed hyperedge (d > 1024).  Distinct values are found with a
// shared-memory bitmap over a window of ids [lo, lo + 32 * kBigWords); windows sweep the range
// [min, max] of the mapped pins, so the output comes out ascending without a sort.
template <bool MAP>
__global__ void __launch_bounds__(kBigThreads)
k_seg_big(const int *__restrict__ hoff, const int *__restrict__ pins, const int *__restrict__ cmap,
          int *__restrict__ scratch, int *__restrict__ cnt, const int *__restrict__ list,
          const int *__restrict__ counters) {
    __shared__ uint32_t bits[kBigWords];
    __shared__ int red[33];
    __shared__ int s_minmax[2];
    const int n = counters[1];
    for (int w = blockIdx.x; w < n; w += gridDim.x) {
        const int e = list[w];
        const int a = hoff[e], d = hoff[e + 1] - a;
        int lo = INT_MAX, hi = INT_MIN;
        for (int i = threadIdx.x; i < d; i += blockDim.x) {
            int x = mapped<MAP>(pins, cmap, a + i);
            lo = min(lo, x);
            hi = max(hi, x);
        }
        lo = warp_min(lo);
        hi = warp_max(hi);
        if (threadIdx.x == 0) { s_minmax[0] = INT_MAX; s_minmax[1] = INT_MIN; }
        __syncthreads();
        if ((threadIdx.x & 31) == 0) { atomicMin(&s_minmax[0], lo); atomicMax(&s_minmax[1], hi); }
        __syncthreads();
        lo = s_minmax[0];
        hi = s_minmax[1];
        int written = 0;
        for (int64_t wlo = lo; wlo <= hi; wlo += 32 * kBigWords) {
            const int64_t rest = (int64_t)hi - wlo + 1;
            const int64_t span = rest < 32 * (int64_t)kBigWords ? rest : 32 * (int64_t)kBigWords;
            const int words = (int)((span + 31) >> 5);
            for (int i = threadIdx.x; i < words; i += blockDim.x) bits[i] = 0;
            __syncthreads();
            for (int i = threadIdx.x; i < d; i += blockDim.x) {
                int64_t x = (int64_t)mapped<MAP>(pins, cmap, a + i) - wlo;
                if (x >= 0 && x < span) atomicOr(&bits[x >> 5], 1u << (x & 31));
            }
            __syncthreads();
            // each thread owns a contiguous run of words; block scan of their popcounts
            const int per = (words + blockDim.x - 1) / blockDim.x;
            const int w0 = threadIdx.x * per;
            int c = 0;
            for (int q = 0; q < per; ++q)
                if (w0 + q < words) c += __popc(bits[w0 + q]);
            int tot;
            int pos = block_exclusive_scan<int>(c, red, &tot);
            int *out = scratch + a + written;
            for (int q = 0; q < per; ++q) {
                if (w0 + q >= words) break;
                uint32_t b = bits[w0 + q];
                while (b) {
                    int t = __ffs(b) - 1;
                    b &= b - 1;
                    out[pos++] = (int)(wlo + 32 * (int64_t)(w0 + q) + t);
                }
            }
            written += tot;
            __syncthreads();
        }
        if (threadIdx.x == 0) cnt[e] = written;
        __syncthreads();
    }
}

// Compaction offsets: value = (kept << 31) | distinct pins for hyperedges with >= 2 distinct pins.
struct CompactIn {
    const int *cnt;
    __device__ uint64_t operator()(int64_t e) const {
        int c = cnt[e];
        return c >= 2 ? ((1ull << 31) | (uint64_t)c) : 0ull;
    }
};
struct CompactOut {
    int64_t n;
    const int *hw_in;
    int *hoff_out, *hw_out, *emap, *sizes;  // sizes[0] = E', sizes[1] = P'
    __device__ void operator()(int64_t e, uint64_t pre, uint64_t val) const {
        int ei = (int)(pre >> 31), pi = (int)(pre & 0x7fffffffu);
        if (val) {
            hoff_out[ei] = pi;
            if (hw_out) hw_out[ei] = hw_in ? hw_in[e] : 1;
            emap[e] = ei;
        } else {
            emap[e] = -1;
        }
        if (e == n - 1) {
            uint64_t t = pre + val;
            int Et = (int)(t >> 31), Pt = (int)(t & 0x7fffffffu);
            hoff_out[Et] = Pt;
            sizes[0] = Et;
            sizes[1] = Pt;
        }
    }
};

// Segment of pin slot i: largest e with hoff[e] <= i, searched within [e_lo, e_hi].
__device__ __forceinline__ int seg_of(const int *hoff, int i, int e_lo, int e_hi) {
    while (e_lo < e_hi) {
        int m = (e_lo + e_hi + 1) >> 1;
        if (hoff[m] <= i) e_lo = m;
        else e_hi = m - 1;
    }
    return e_lo;
}

// Block-level search bounds for pin slots [b0, b1): first and last segment touched.
__device__ __forceinline__ void block_seg_range(const int *hoff, int E, int b0, int b1, int *s_rng) {
    if (threadIdx.x == 0) s_rng[0] = seg_of(hoff, b0, 0, E - 1);
    if (threadIdx.x == 1) s_rng[1] = seg_of(hoff, b1 - 1, 0, E - 1);
    __syncthreads();
}

// Copies the distinct pins of kept hyperedges from scratch (at fine offsets) to the coarse CSR
// and counts the coarse node degrees (integer atomics) for the incidence build.  Load-balanced
// over fine pin slots: per-hyperedge values are loaded once per run of slots.
__global__ void __launch_bounds__(kLbBlock)
k_seg_copy(int E, int P, const int *__restrict__ hoff, const int *__restrict__ scratch,
           const int *__restrict__ cnt, const int *__restrict__ emap,
           const int *__restrict__ hoff_out, int *__restrict__ pins_out, int *__restrict__ deg) {
    lb_runs(hoff, E, P, [&](int e, int a, int b) {
        const int ee = __ldg(emap + e);
        if (ee < 0) return;
        const int base = __ldg(hoff + e), c = __ldg(cnt + e), o = __ldg(hoff_out + ee);
        const int stop = base + c < b ? base + c : b;
        for (int i = a; i < stop; ++i) {
            const int v = __ldg(scratch + i);
            pins_out[o + (i - base)] = v;
            atomicAdd(deg + v, 1);
        }
    });
}

__global__ void k_fill(int n, int val, int *__restrict__ a) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = val;
}

// ------------------------------------------------------------------------------- incidence
struct DegIn {
    const int *deg;
    __device__ uint64_t operator()(int64_t v) const { return (uint64_t)deg[v]; }
};
struct DegOut {
    int64_t n;
    int *noff, *cursor;
    __device__ void operator()(int64_t v, uint64_t pre, uint64_t val) const {
        noff[v] = (int)pre;
        cursor[v] = (int)pre;
        if (v == n - 1) noff[n] = (int)(pre + val);
    }
};

// Fills the node -> hyperedge incidence: every pin slot takes the next free position of its node
// (cursor starts at the node's offset).  Each thread owns kLbItems consecutive slots: it finds
// their hyperedges with one search, then issues all its atomics before any store, so the
// atomics' round trips overlap.  The order inside a node's list depends on the atomics' order;
// every consumer is order-independent.
__global__ void __launch_bounds__(kLbBlock)
k_fill_adj(int E, int P, const int *__restrict__ hoff, const int *__restrict__ pins,
           int *__restrict__ cursor, int *__restrict__ nadj) {
    __shared__ int s_rng[2];
    for (int64_t t0 = (int64_t)blockIdx.x * kLbTile; t0 < P; t0 += (int64_t)gridDim.x * kLbTile) {
        const int j0 = (int)t0;
        const int j1 = (int)(t0 + kLbTile < P ? t0 + kLbTile : P);
        __syncthreads();
        if (threadIdx.x == 0) s_rng[0] = lb_seg(hoff, j0, 0, E - 1);
        if (threadIdx.x == 32) s_rng[1] = lb_seg(hoff, j1 - 1, 0, E - 1);
        __syncthreads();
        const int j = j0 + threadIdx.x * kLbItems;
        if (j >= j1) continue;
        const int n = j1 - j < kLbItems ? j1 - j : kLbItems;
        int s = lb_seg(hoff, j, s_rng[0], s_rng[1]);
        int send = __ldg(hoff + s + 1);
        int v[kLbItems], e[kLbItems], pos[kLbItems];
#pragma unroll
        for (int k = 0; k < kLbItems; ++k) {
            if (k < n) {
                while (j + k >= send) { ++s; send = __ldg(hoff + s + 1); }
                e[k] = s;
                v[k] = __ldg(pins + j + k);
            }
        }
#pragma unroll
        for (int k = 0; k < kLbItems; ++k)
            if (k < n) pos[k] = atomicAdd(cursor + v[k], 1);
#pragma unroll
        for (int k = 0; k < kLbItems; ++k)
            if (k < n) nadj[pos[k]] = e[k];
    }
}

// ------------------------------------------------------------------ Algorithm 1
__global__ void k_hedge_key(int E, int policy, const int *__restrict__ hoff,
                            const int *__restrict__ hw, unsigned long long *__restrict__ hkey) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
        uint32_t deg = (uint32_t)(hoff[e + 1] - hoff[e]);
        uint32_t w = hw ? (uint32_t)hw[e] : 1u;
        uint32_t h = mix32((uint32_t)e);
        uint32_t pr = policy_priority(policy, deg, w, h);
        hkey[e] = ((unsigned long long)pr << 32) | h;
    }
}

// Every node takes the incident hyperedge with the smallest key (lexicographic (priority, hash);
// the hash is a bijection so the key also identifies the hyperedge).  Load-balanced over the
// incidence array: per-node partial minima are combined with 64-bit atomicMin, whose result does
// not depend on the order of the atomics.
__global__ void __launch_bounds__(kLbBlock)
k_match_min(int N, int P, const int *__restrict__ noff, const int *__restrict__ nadj,
            const unsigned long long *__restrict__ hkey, unsigned long long *__restrict__ nkey) {
    lb_for_each<unsigned long long>(
        noff, N, P, ~0ull,
        [&](int, int j, unsigned long long acc) {
            unsigned long long k = __ldg(hkey + __ldg(nadj + j));
            return k < acc ? k : acc;
        },
        [&](int v, unsigned long long acc) {
            if (acc != ~0ull) atomicMin(nkey + v, acc);
        });
}

// match[v] from the winning key; sizes and weights of the matched sets S(e) (integer atomics).
__global__ void __launch_bounds__(kBlock)
k_match_set(int N, const unsigned long long *__restrict__ nkey, const int *__restrict__ nw,
            int *__restrict__ match, int *__restrict__ ssize, int *__restrict__ sweight) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) {
        unsigned long long k = nkey[v];
        int m = k == ~0ull ? -1 : (int)unmix32((uint32_t)k);
        match[v] = m;
        if (m >= 0) {
            atomicAdd(&ssize[m], 1);
            atomicAdd(&sweight[m], nw[v]);
        }
    }
}

// Algorithm 2, second loop, for every singleton set S(e) = {u}: the lightest step-1 merged node
// among e's pins, as the key (merged weight << 32 | group id), minimum over e's pins.
// Load-balanced over all pins; hyperedges that are not singleton sets are skipped.
__global__ void __launch_bounds__(kLbBlock)
k_single_best(int E, int P, const int *__restrict__ hoff, const int *__restrict__ pins,
              const int *__restrict__ match, const int *__restrict__ ssize,
              const int *__restrict__ sweight, unsigned long long *__restrict__ best) {
    lb_for_each<unsigned long long>(
        hoff, E, P, ~0ull,
        [&](int e, int i, unsigned long long acc) {
            if (__ldg(ssize + e) != 1) return acc;
            int mv = __ldg(match + __ldg(pins + i));
            if (mv >= 0 && __ldg(ssize + mv) >= 2) {
                unsigned long long k = ((unsigned long long)(unsigned)__ldg(sweight + mv) << 32) | (unsigned)mv;
                acc = k < acc ? k : acc;
            }
            return acc;
        },
        [&](int e, unsigned long long acc) {
            if (acc != ~0ull) atomicMin(best + e, acc);
        });
}

// grp[v] = matched hyperedge of v's final group, or -1 when v stays alone; rep[g] receives the
// smallest member of group g.
__global__ void __launch_bounds__(kBlock)
k_group(int N, const int *__restrict__ match, const int *__restrict__ ssize,
        const unsigned long long *__restrict__ best, int *__restrict__ grp,
        unsigned *__restrict__ rep) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < N; u += gridDim.x * blockDim.x) {
        int m = match[u];
        int g = -1;
        if (m >= 0) {
            if (ssize[m] >= 2) g = m;
            else if (best[m] != ~0ull) g = (int)(best[m] & 0xffffffffu);
        }
        grp[u] = g;
        if (g >= 0) atomicMin(&rep[g], (unsigned)u);
    }
}

struct RenumIn {
    const int *grp;
    const unsigned *rep;
    __device__ uint64_t operator()(int64_t v) const {
        int g = grp[v];
        return (g < 0 || rep[g] == (unsigned)v) ? 1ull : 0ull;
    }
};
struct RenumOut {
    int64_t n;
    const int *grp;
    int *cmap, *gcid, *nc_out;  // *nc_out = N'
    __device__ void operator()(int64_t v, uint64_t pre, uint64_t val) const {
        if (val) {
            cmap[v] = (int)pre;
            int g = grp[v];
            if (g >= 0) gcid[g] = (int)pre;
        }
        if (v == n - 1) *nc_out = (int)(pre + val);
    }
};

__global__ void k_cmap(int N, const int *__restrict__ grp, const int *__restrict__ gcid,
                       const int *__restrict__ nw, int *__restrict__ cmap, int *__restrict__ cw) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) {
        int g = grp[v];
        int c = g >= 0 ? gcid[g] : cmap[v];
        cmap[v] = c;
        atomicAdd(&cw[c], nw[v]);
    }
}

// ------------------------------------------------------------------ host side
namespace {

// Per hyperedge: pins mapped through `map` (identity when null), sorted and de-duplicated into
// scratch at the hyperedge's own offset; cnt[e] = number of distinct values.
void seg_unique(bipart_graph *g, int32_t E, int32_t P, const int *hoff, const int *pins,
                const int *map, int *scratch, int *cnt) {
    cudaStream_t s = g->stream;
    Work &w = g->w;
    int *mid = (int *)w.e_c.ensure(sizeof(int) * (size_t)std::max(E, 1), s);
    int *big = (int *)w.e_d.ensure(sizeof(int) * (size_t)std::max(E, 1), s);
    int *small = w.small.as<int>();  // [0] mid count, [1] big count
    BP_CUDA(cudaMemsetAsync(small, 0, 2 * sizeof(int), s));
    if (E == 0) return;
    // reads hoff, pins, map gathers; writes distinct pins (<= P) and counts
    ProfScope ps("contract_unique", 8.0 * E + 4.0 * P * (map ? 3 : 2), s);
    if (map) k_seg_small<true><<<grid_for(E), kBlock, 0, s>>>(E, hoff, pins, map, scratch, cnt, mid, big, small);
    else k_seg_small<false><<<grid_for(E), kBlock, 0, s>>>(E, hoff, pins, map, scratch, cnt, mid, big, small);
    BP_LAUNCH();
    int mid_grid = std::max(1, std::min(152 * 16, ceil_div_i(P / (kSmallDeg + 1) + 1, kBlock / 32)));
    if (map) k_seg_mid<true><<<mid_grid, kBlock, 0, s>>>(hoff, pins, map, scratch, cnt, mid, small);
    else k_seg_mid<false><<<mid_grid, kBlock, 0, s>>>(hoff, pins, map, scratch, cnt, mid, small);
    BP_LAUNCH();
    int big_grid = std::max(1, std::min(152 * 4, P / (kMidDeg + 1) + 1));
    if (map) k_seg_big<true><<<big_grid, kBigThreads, 0, s>>>(hoff, pins, map, scratch, cnt, big, small);
    else k_seg_big<false><<<big_grid, kBigThreads, 0, s>>>(hoff, pins, map, scratch, cnt, big, small);
    BP_LAUNCH();
}

// Sorted-unique of every hyperedge's (mapped) pins into the coarse CSR of `c`.
// Sets c.E and c.P.  `map` null means identity (level-0 normalisation).
void contract(bipart_graph *g, int32_t E, int32_t P, const int *hoff, const int *pins,
              const int *hw, const int *map, Level &c, int *deg) {
    cudaStream_t s = g->stream;
    Work &w = g->w;
    int *scratch = (int *)w.p_a.ensure(sizeof(int) * (size_t)std::max(P, 1), s);
    int *cnt = (int *)w.e_a.ensure(sizeof(int) * (size_t)std::max(E, 1), s);
    int *emap = (int *)w.e_b.ensure(sizeof(int) * (size_t)std::max(E, 1), s);
    int *small = w.small.as<int>();
    BP_CUDA(cudaMemsetAsync(small, 0, 8 * sizeof(int), s));
    seg_unique(g, E, P, hoff, pins, map, scratch, cnt);
    c.b_hoff.ensure(sizeof(int) * ((size_t)E + 1), s);
    c.b_pins.ensure(sizeof(int) * (size_t)std::max(P, 1), s);
    bool unit = (hw == nullptr);
    if (!unit) c.b_hw.ensure(sizeof(int) * (size_t)std::max(E, 1), s);
    c.unit_hw = unit;
    if (E > 0) {
        CompactOut out{E, hw, c.hoff(), unit ? nullptr : c.b_hw.as<int>(), emap, small + 2};
        {
            ProfScope ps("contract_offsets", 16.0 * E, s);
            scan(E, CompactIn{cnt}, out, w.scan.ensure(scan_state_bytes(E), s), dev_status(g), s);
        }
        {
            // scratch, coarse pins, degree atomics, per-hyperedge offsets
            ProfScope ps("contract_copy", 12.0 * P + 12.0 * E, s);
            k_seg_copy<<<lb_grid(P), kLbBlock, 0, s>>>(E, P, hoff, scratch, cnt, emap, c.hoff(), c.pins(), deg);
            BP_LAUNCH();
        }
    } else {
        BP_CUDA(cudaMemsetAsync(c.hoff(), 0, sizeof(int), s));
    }
    c.E = E > 0 ? read_i32(g, small + 2) : 0;
    c.P = E > 0 ? read_i32(g, small + 3) : 0;
}

}  // namespace

void distinct_counts(bipart_graph *g, Level &L, const int *d_map, int *cnt) {
    int *scratch = (int *)g->w.p_a.ensure(sizeof(int) * (size_t)std::max(L.P, 1), g->stream);
    seg_unique(g, L.E, L.P, L.hoff(), L.pins(), d_map, scratch, cnt);
}

// Node -> hyperedge incidence of a level whose degrees were counted by its contraction
// (deg[N], in the per-node scratch n_a).
void build_incidence(bipart_graph *g, Level &L) {
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
    {
        ProfScope ps("incidence_offsets", 12.0 * L.N, s);
        scan(L.N, DegIn{deg}, DegOut{L.N, L.noff(), cursor}, w.scan.ensure(scan_state_bytes(L.N), s),
             dev_status(g), s);
    }
    if (L.P > 0) {
        ProfScope ps("incidence_fill", 12.0 * L.P + 4.0 * L.E, s);
        k_fill_adj<<<lb_grid(L.P), kLbBlock, 0, s>>>(L.E, L.P, L.hoff(), L.pins(), cursor, L.nadj());
        BP_LAUNCH();
    }
}

// Zeroed degree counters for a level of N nodes (filled by the contraction's copy).
int *degree_counters(bipart_graph *g, int32_t N) {
    int *deg = (int *)g->w.n_a.ensure(sizeof(int) * (size_t)std::max(N, 1), g->stream);
    if (N > 0) BP_CUDA(cudaMemsetAsync(deg, 0, sizeof(int) * (size_t)N, g->stream));
    return deg;
}

void build_level0(bipart_graph *g, Level &L, int32_t N, int32_t E, const int32_t *d_hoff,
                  const int32_t *d_pins, const int32_t *d_nw, const int32_t *d_hw) {
    cudaStream_t s = g->stream;
    int32_t P = 0;
    if (E > 0) {
        BP_CUDA(cudaMemcpyAsync(g->w.host_small, d_hoff + E, sizeof(int), cudaMemcpyDeviceToHost, s));
        sync(g);
        P = (int32_t)g->w.host_small[0];
    }
    L.N = N;
    contract(g, E, P, d_hoff, d_pins, d_hw, nullptr, L, degree_counters(g, N));
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

void coarsen_level(bipart_graph *g, Level &f, Level &c, int policy) {
    cudaStream_t s = g->stream;
    Work &w = g->w;
    const int N = f.N, E = f.E;
    unsigned long long *hkey = (unsigned long long *)w.e_key.ensure(sizeof(uint64_t) * (size_t)std::max(E, 1), s);
    int *ssize = (int *)w.e_a.ensure(sizeof(int) * (size_t)std::max(E, 1), s);
    int *sweight = (int *)w.e_b.ensure(sizeof(int) * (size_t)std::max(E, 1), s);
    unsigned *rep = (unsigned *)w.e_c.ensure(sizeof(int) * (size_t)std::max(E, 1), s);
    int *gcid = (int *)w.e_d.ensure(sizeof(int) * (size_t)std::max(E, 1), s);
    int *grp = (int *)w.n_c.ensure(sizeof(int) * (size_t)std::max(N, 1), s);
    int *small = w.small.as<int>();
    if (E > 0) {
        {
            ProfScope ps("hedge_key", 12.0 * E + (f.hw() ? 4.0 * E : 0.0), s);
            k_hedge_key<<<grid_for(E), kBlock, 0, s>>>(E, policy, f.hoff(), f.hw(), hkey);
            BP_LAUNCH();
        }
        BP_CUDA(cudaMemsetAsync(ssize, 0, sizeof(int) * (size_t)E, s));
        BP_CUDA(cudaMemsetAsync(sweight, 0, sizeof(int) * (size_t)E, s));
        BP_CUDA(cudaMemsetAsync(rep, 0xff, sizeof(int) * (size_t)E, s));
    }
    if (N > 0) {
        unsigned long long *nkey = (unsigned long long *)w.n_key.ensure(sizeof(uint64_t) * (size_t)N, s);
        BP_CUDA(cudaMemsetAsync(nkey, 0xff, sizeof(uint64_t) * (size_t)N, s));
        if (f.P > 0) {
            // noff, nadj, 8-byte key gather per incidence, one 8-byte atomic per node run
            ProfScope ps("match_min", 4.0 * N + 12.0 * f.P + 8.0 * N, s);
            k_match_min<<<lb_grid(f.P), kLbBlock, 0, s>>>(N, f.P, f.noff(), f.nadj(), hkey, nkey);
            BP_LAUNCH();
        }
        {
            ProfScope ps("match_set", 24.0 * N, s);
            k_match_set<<<grid_for(N), kBlock, 0, s>>>(N, nkey, f.nw(), f.match(), ssize, sweight);
            BP_LAUNCH();
        }
        unsigned long long *best = hkey;  // the hyperedge keys are no longer needed
        BP_CUDA(cudaMemsetAsync(best, 0xff, sizeof(uint64_t) * (size_t)E, s));
        if (f.P > 0) {
            ProfScope ps("single_best", 4.0 * E + 4.0 * f.P, s);
            k_single_best<<<lb_grid(f.P), kLbBlock, 0, s>>>(E, f.P, f.hoff(), f.pins(), f.match(), ssize, sweight, best);
            BP_LAUNCH();
        }
        {
            ProfScope ps("group", 20.0 * N, s);
            k_group<<<grid_for(N), kBlock, 0, s>>>(N, f.match(), ssize, best, grp, rep);
            BP_LAUNCH();
        }
        {
            ProfScope ps("renumber", 12.0 * N, s);
            scan(N, RenumIn{grp, rep}, RenumOut{N, grp, f.cmap(), gcid, small + 4},
                 w.scan.ensure(scan_state_bytes(N), s), dev_status(g), s);
        }
    }
    const int Nc = N > 0 ? read_i32(g, small + 4) : 0;
    c.N = Nc;
    c.b_nw.ensure(sizeof(int) * (size_t)std::max(Nc, 1), s);
    if (N > 0) {
        BP_CUDA(cudaMemsetAsync(c.nw(), 0, sizeof(int) * (size_t)Nc, s));
        ProfScope ps("cmap", 24.0 * N, s);
        k_cmap<<<grid_for(N), kBlock, 0, s>>>(N, grp, gcid, f.nw(), f.cmap(), c.nw());
        BP_LAUNCH();
    }
    contract(g, E, f.P, f.hoff(), f.pins(), f.hw(), f.cmap(), c, degree_counters(g, Nc));
    build_incidence(g, c);
    c.b_cmap.ensure(sizeof(int) * (size_t)std::max(Nc, 1), s);
    c.b_match.ensure(sizeof(int) * (size_t)std::max(Nc, 1), s);
}

}  // namespace bp
