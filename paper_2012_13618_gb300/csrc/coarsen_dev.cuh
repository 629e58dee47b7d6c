// Device side of coarsening (Algorithms 1 and 2, Sec. 3.1) and of the level-0 normalisation,
// written once for any team of threads: the grid kernels in coarsen.cu run each phase as its own
// launch; the persistent block path in block.cu runs all phases of an instance inside one block.
#pragma once

#include <climits>

#include <cooperative_groups.h>

#include "common.cuh"
#include "lb.cuh"

namespace bp {

constexpr int kSmallDeg = 8;      // hyperedges up to this degree: one thread each
constexpr int kMidDeg = 1024;     // up to this degree: one warp each (register bitonic sort)
constexpr int kGridMidDeg = 256;  // the same bound for the grid kernels, where one warp sorting
                                  // up to 1024 keys would hold up the whole launch
constexpr int kBigWords = 8192;   // bitmap window of the block tier: 32 KB = 262,144 ids
constexpr int kBigCache = 12;     // mapped pins a block-tier thread keeps in registers

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

// Pin i mapped through cmap (MAP) or as is.
template <bool MAP, class Team>
__device__ __forceinline__ int mapped(const int *pins, const int *cmap, int i) {
    int p = Team::ld(pins + i);
    return MAP ? Team::ld(cmap + p) : p;
}

// Warp-cooperative sorted-unique of one hyperedge of degree d <= 32 * R.
template <int R, bool MAP, class Team>
__device__ __forceinline__ int warp_unique(const int *pins, const int *cmap, int a, int d, int *out) {
    const int lane = threadIdx.x & 31;
    int v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        int idx = lane * R + r;
        v[r] = idx < d ? mapped<MAP, Team>(pins, cmap, a + idx) : INT_MAX;
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

// Appends x to a work list whose length is *n, with one atomic per group of converged lanes (a
// single counter shared by a whole grid would otherwise take one atomic per entry).
__device__ __forceinline__ void append_aggregated(int *list, int *n, int x) {
    namespace cg = cooperative_groups;
    const cg::coalesced_group grp = cg::coalesced_threads();
    int base = 0;
    if (grp.thread_rank() == 0) base = atomicAdd(n, (int)grp.size());
    base = grp.shfl(base, 0);
    list[base + (int)grp.thread_rank()] = x;
}

// Small tier: one thread per hyperedge of degree <= 8 (the vast majority): mapped pins sorted by
// a register network, unique values written at the hyperedge's own offset in scratch, cnt[e] =
// their number.  Larger hyperedges are appended to the mid / big work lists (list order is
// irrelevant: every hyperedge writes only its own slots).
template <bool MAP, class Team>
__device__ void d_seg_small(Team t, int E, const int *hoff, const int *pins, const int *cmap,
                            int *scratch, int *cnt, int *mid_list, int *big_list, int *counters,
                            int mid_max = kMidDeg) {
    for (int e = t.rank(); e < E; e += t.size()) {
        int a = Team::ld(hoff + e), d = Team::ld(hoff + e + 1) - a;
        if (d > kSmallDeg) {
            if (d > mid_max) append_aggregated(big_list, &counters[1], e);
            else append_aggregated(mid_list, &counters[0], e);
            continue;
        }
        int v[kSmallDeg];
#pragma unroll
        for (int k = 0; k < kSmallDeg; ++k) v[k] = k < d ? mapped<MAP, Team>(pins, cmap, a + k) : INT_MAX;
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

// Mid tier: one warp per listed hyperedge (8 < d <= 32 * kMaxR), register bitonic sort.
template <bool MAP, class Team, int kMaxR = kMidDeg / 32>
__device__ void d_seg_mid(Team t, const int *hoff, const int *pins, const int *cmap, int *scratch,
                          int *cnt, const int *list, const int *counters) {
    const int n = Team::ld(counters);
    const int lane = threadIdx.x & 31;
    for (int w = t.warp(); w < n; w += t.warps()) {
        int e = Team::ld(list + w);
        int a = Team::ld(hoff + e), d = Team::ld(hoff + e + 1) - a;
        int *out = scratch + a;
        int m;
        if (d <= 32) m = warp_unique<1, MAP, Team>(pins, cmap, a, d, out);
        else if (d <= 64) m = warp_unique<2, MAP, Team>(pins, cmap, a, d, out);
        else if (d <= 128) m = warp_unique<4, MAP, Team>(pins, cmap, a, d, out);
        else if (kMaxR <= 8 || d <= 256) m = warp_unique<8, MAP, Team>(pins, cmap, a, d, out);
        else if constexpr (kMaxR > 8) {
            if (d <= 512) m = warp_unique<16, MAP, Team>(pins, cmap, a, d, out);
            else m = warp_unique<32, MAP, Team>(pins, cmap, a, d, out);
        }
        if (lane == 0) cnt[e] = m;
    }
}

// Big tier: one block per listed hyperedge (d > 1024).  Distinct values are found with a
// shared-memory bitmap `bits` (kBigWords words) over a window of ids [lo, lo + 32 * kBigWords);
// windows sweep the range [min, max] of the mapped pins, so the output comes out ascending
// without a sort.
template <bool MAP, class Team>
__device__ void d_seg_big(Team t, const int *hoff, const int *pins, const int *cmap, int *scratch,
                          int *cnt, const int *list, const int *counters, uint32_t *bits) {
    __shared__ int red[33];
    __shared__ int s_minmax[2];
    const int n = Team::ld(counters + 1);
    const int cached = kBigCache * (int)blockDim.x;
    for (int w = t.block(); w < n; w += t.blocks()) {
        const int e = Team::ld(list + w);
        const int a = Team::ld(hoff + e), d = Team::ld(hoff + e + 1) - a;
        // the thread's first kBigCache mapped pins (i = threadIdx.x + k * blockDim.x), gathered
        // together and kept in registers for every pass; pins beyond are gathered per pass
        int xs[kBigCache];
#pragma unroll
        for (int k = 0; k < kBigCache; ++k) {
            const int i = threadIdx.x + k * (int)blockDim.x;
            xs[k] = i < d ? mapped<MAP, Team>(pins, cmap, a + i) : 0;
        }
        int lo = INT_MAX, hi = INT_MIN;
#pragma unroll
        for (int k = 0; k < kBigCache; ++k) {
            if (threadIdx.x + k * (int)blockDim.x < d) {
                lo = min(lo, xs[k]);
                hi = max(hi, xs[k]);
            }
        }
        for (int i = cached + threadIdx.x; i < d; i += blockDim.x) {
            int x = mapped<MAP, Team>(pins, cmap, a + i);
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
#pragma unroll
            for (int k = 0; k < kBigCache; ++k) {
                const int64_t x = (int64_t)xs[k] - wlo;
                if (threadIdx.x + k * (int)blockDim.x < d && x >= 0 && x < span)
                    atomicOr(&bits[x >> 5], 1u << (x & 31));
            }
            for (int i = cached + threadIdx.x; i < d; i += blockDim.x) {
                int64_t x = (int64_t)mapped<MAP, Team>(pins, cmap, a + i) - wlo;
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
                    int bit = __ffs(b) - 1;
                    b &= b - 1;
                    out[pos++] = (int)(wlo + 32 * (int64_t)(w0 + q) + bit);
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
// With parallel-net merging (rep non-null) only the representative of each group is kept.
struct CompactIn {
    const int *cnt;
    const int *rep = nullptr;
    __device__ uint64_t operator()(int64_t e) const {
        int c = cnt[e];
        const bool keep = c >= 2 && (!rep || rep[e] == (int)e);
        return keep ? ((1ull << 31) | (uint64_t)c) : 0ull;
    }
};
struct CompactOut {
    int64_t n;
    const int *hw_in;
    int *hoff_out, *hw_out, *emap, *sizes;  // sizes[0] = E', sizes[1] = P'
    int *ts;                                // tile starts of the compacted CSR (or null)
    const int *wsum = nullptr;              // merged group weights (parallel-net merging)
    __device__ void operator()(int64_t e, uint64_t pre, uint64_t val) const {
        int ei = (int)(pre >> 31), pi = (int)(pre & 0x7fffffffu);
        if (val) {
            hoff_out[ei] = pi;
            lb_mark_tiles(ts, ei, pi, (int64_t)(val & 0x7fffffffu));
            if (hw_out) hw_out[ei] = wsum ? wsum[e] : (hw_in ? hw_in[e] : 1);
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

// Copies the distinct pins of kept hyperedges from scratch (at fine offsets) to the coarse CSR
// and counts the coarse node degrees (integer atomics) for the incidence build.  Load-balanced
// over fine pin slots: per-hyperedge values are loaded once per run of slots.
template <class Team>
__device__ void d_seg_copy(Team t, int E, int P, const int *hoff, const int *scratch,
                           const int *cnt, const int *emap, const int *hoff_out, int *pins_out,
                           int *deg, const int *ts = nullptr) {
    lb_runs(
        hoff, E, P,
        [&](int e, int a, int b) {
            const int ee = Team::ld(emap + e);
            if (ee < 0) return;
            const int base = Team::ld(hoff + e), c = Team::ld(cnt + e), o = Team::ld(hoff_out + ee);
            const int stop = base + c < b ? base + c : b;
            for (int i = a; i < stop; ++i) {
                const int v = Team::ld(scratch + i);
                pins_out[o + (i - base)] = v;
                atomicAdd(deg + v, 1);
            }
        },
        t, ts);
}

// ------------------------------------------------------------------------------- incidence
struct DegIn {
    const int *deg;
    __device__ uint64_t operator()(int64_t v) const { return (uint64_t)deg[v]; }
};
struct DegOut {
    int64_t n;
    int *noff, *cursor;
    int *ts;  // tile starts of the incidence CSR (or null)
    __device__ void operator()(int64_t v, uint64_t pre, uint64_t val) const {
        noff[v] = (int)pre;
        cursor[v] = (int)pre;
        lb_mark_tiles(ts, (int)v, (int64_t)pre, (int64_t)val);
        if (v == n - 1) noff[n] = (int)(pre + val);
    }
};

// Fills the node -> hyperedge incidence: every pin slot takes the next free position of its node
// from claim(v).  Each thread owns kLbItems consecutive slots: it finds their hyperedges with one
// search, then issues all its claims before any store, so the atomics' round trips overlap.  The
// order inside a node's list depends on the atomics' order; every consumer is order-independent.
template <class Team, class Claim>
__device__ void d_fill_adj_with(Team t, int E, int P, const int *hoff, const int *pins, int *nadj,
                                Claim claim, const int *ts = nullptr) {
    lb_schedule(hoff, E, P, ts, t, [&](int j, int n, int s, auto end) {
        int send = end(s);
        int v[kLbItems], e[kLbItems], pos[kLbItems];
#pragma unroll
        for (int k = 0; k < kLbItems; ++k) {
            if (k < n) {
                while (j + k >= send) { ++s; send = end(s); }
                e[k] = s;
                v[k] = Team::ld(pins + j + k);
            }
        }
#pragma unroll
        for (int k = 0; k < kLbItems; ++k)
            if (k < n) pos[k] = claim(v[k]);
#pragma unroll
        for (int k = 0; k < kLbItems; ++k)
            if (k < n) nadj[pos[k]] = e[k];
    });
}

// Incidence fill claiming positions from the global per-node cursor (cursor starts at the node's
// offset).
template <class Team>
__device__ void d_fill_adj(Team t, int E, int P, const int *hoff, const int *pins, int *cursor,
                           int *nadj, const int *ts = nullptr) {
    d_fill_adj_with(t, E, P, hoff, pins, nadj, [&](int v) { return atomicAdd(cursor + v, 1); }, ts);
}

// ------------------------------------------------------------------ Algorithm 1
template <class Team>
__device__ void d_hedge_key(Team t, int E, int policy, const int *hoff, const int *hw,
                            unsigned long long *hkey) {
    for (int e = t.rank(); e < E; e += t.size()) {
        uint32_t deg = (uint32_t)(Team::ld(hoff + e + 1) - Team::ld(hoff + e));
        uint32_t w = hw ? (uint32_t)Team::ld(hw + e) : 1u;
        uint32_t h = mix32((uint32_t)e);
        uint32_t pr = policy_priority(policy, deg, w, h);
        hkey[e] = ((unsigned long long)pr << 32) | h;
    }
}

// Every node takes the incident hyperedge with the smallest key (lexicographic (priority, hash);
// the hash is a bijection so the key also identifies the hyperedge).  Load-balanced over the
// incidence array: per-node partial minima are combined with 64-bit atomicMin, whose result does
// not depend on the order of the atomics.
template <class Team>
// With `warp_min` the last runs of a warp's lanes are combined per node before the atomic (levels
// whose nodes have long incidence lists, where many threads would end on one node).
__device__ void d_match_min(Team t, int N, int P, const int *noff, const int *nadj,
                            const unsigned long long *hkey, unsigned long long *nkey,
                            const int *ts = nullptr, bool warp_min = false) {
    auto visit = [&](int, int e, unsigned long long acc) {
        unsigned long long k = Team::ld(hkey + e);
        return k < acc ? k : acc;
    };
    auto flush = [&](int v, unsigned long long acc) {
        if (acc != ~0ull) atomicMin(nkey + v, acc);
    };
    if (warp_min)
        lb_reduce_items<unsigned long long>(noff, N, P, nadj, ~0ull, cooperative_groups::less<unsigned long long>(),
                                            visit, flush, t, ts);
    else
        lb_for_each_items<unsigned long long>(noff, N, P, nadj, ~0ull, visit, flush, t, ts);
}

// match[v] from the winning key; sizes and weights of the matched sets S(e) (integer atomics).
template <class Team>
__device__ void d_match_set(Team t, int N, const unsigned long long *nkey, const int *nw, int *match,
                            int *ssize, int *sweight) {
    for (int v = t.rank(); v < N; v += t.size()) {
        unsigned long long k = Team::ld(nkey + v);
        int m = k == ~0ull ? -1 : (int)unmix32((uint32_t)k);
        match[v] = m;
        if (m >= 0) {
            atomicAdd(&ssize[m], 1);
            atomicAdd(&sweight[m], Team::ld(nw + v));
        }
    }
}

// ------------------------------------------------------------------ Algorithm 2
// Second loop, for every singleton set S(e) = {u}: the lightest step-1 merged node among e's
// pins, as the key (merged weight << 32 | group id), minimum over e's pins.  Load-balanced over
// all pins; hyperedges that are not singleton sets are skipped.
template <class Team>
__device__ void d_single_best(Team t, int E, int P, const int *hoff, const int *pins,
                              const int *match, const int *ssize, const int *sweight,
                              unsigned long long *best, const int *ts = nullptr) {
    lb_for_each_items<unsigned long long>(
        hoff, E, P, pins, ~0ull,
        [&](int e, int u, unsigned long long acc) {
            if (Team::ld(ssize + e) != 1) return acc;
            int mv = Team::ld(match + u);
            if (mv >= 0 && Team::ld(ssize + mv) >= 2) {
                unsigned long long k = ((unsigned long long)(unsigned)Team::ld(sweight + mv) << 32) | (unsigned)mv;
                acc = k < acc ? k : acc;
            }
            return acc;
        },
        [&](int e, unsigned long long acc) {
            if (acc != ~0ull) atomicMin(best + e, acc);
        },
        t, ts);
}

// grp[v] = matched hyperedge of v's final group, or -1 when v stays alone; rep[g] receives the
// smallest member of group g.
template <class Team>
__device__ void d_group(Team t, int N, const int *match, const int *ssize,
                        const unsigned long long *best, int *grp, unsigned *rep) {
    for (int u = t.rank(); u < N; u += t.size()) {
        int m = Team::ld(match + u);
        int g = -1;
        if (m >= 0) {
            if (Team::ld(ssize + m) >= 2) g = m;
            else {
                unsigned long long b = Team::ld(best + m);
                if (b != ~0ull) g = (int)(b & 0xffffffffu);
            }
        }
        grp[u] = g;
        if (g >= 0) atomicMin(&rep[g], (unsigned)u);
    }
}

// Coarse ids: 1 for the smallest member of every group (and every node left alone), scanned.
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

template <class Team>
__device__ void d_cmap(Team t, int N, const int *grp, const int *gcid, const int *nw, int *cmap,
                       int *cw) {
    for (int v = t.rank(); v < N; v += t.size()) {
        int g = Team::ld(grp + v);
        int c = g >= 0 ? Team::ld(gcid + g) : cmap[v];
        cmap[v] = c;
        atomicAdd(&cw[c], Team::ld(nw + v));
    }
}

}  // namespace bp
