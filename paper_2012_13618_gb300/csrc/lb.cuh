// Load-balanced segmented loops over a CSR (offsets off[0..nseg], items [0, total)).
//
// Every thread owns kLbItems consecutive items, finds the segment of its first item and walks
// forward.  Per-segment partial results are flushed with one atomic per segment run, so a
// segment with 100,000 items costs the same per item as one with 2 items, and the result does
// not depend on the schedule when the combining operation is an integer sum or minimum.
//
// Two schedules.  With a tile-start table (the CSRs of the hierarchy's levels), a warp takes a
// warp tile of kWarpTile items, reads the tile's segment range with two loads and its lanes
// search that short range in cached global memory -- no block barriers.  Without one (input
// CSRs; the one-block batch path), a block takes a tile of blockDim * kLbItems items, warps 0
// and 1 find its segment range with a 32-way warp search, and the offsets are staged in shared
// memory for the threads' searches.
#pragma once

#include <cooperative_groups.h>
#include <cooperative_groups/reduce.h>

#include "common.cuh"

namespace bp {

constexpr int kLbBlock = 256;
// Items per thread: 4 (one 16-byte load).  A same-box A/B on the 1M-node bisection: 8 items took
// 2.571 ms, 4 items 2.481, 2 items 2.588 -- the gathers of these loops are latency-bound, and a
// shorter per-thread run puts twice the warps on them.
constexpr int kLbItems = 4;
constexpr int kLbTile = kLbBlock * kLbItems;
constexpr int kWarpTile = 32 * kLbItems;

constexpr int kLbStage = 2048;      // segment offsets of one block tile staged in shared memory
constexpr int kTsGran = kWarpTile;  // tile-start tables hold the segment of every item t * kTsGran

// Tile-start table: ts[t] = the segment holding item t * kTsGran, for every such item < total.
// Written while the CSR offsets are produced, by the thread that owns segment `seg` (items
// [a, a + len)).
__device__ __forceinline__ void lb_mark_tiles(int *ts, int seg, int64_t a, int64_t len) {
    if (!ts || len <= 0) return;
    for (int64_t t = (a + kTsGran - 1) / kTsGran; t * kTsGran < a + len; ++t) ts[t] = seg;
}

// Largest s in [lo, hi] with off[s] <= j (the non-empty segment holding item j).
template <class Team = GridTeam>
__device__ __forceinline__ int lb_seg(const int *off, int j, int lo, int hi) {
    while (lo < hi) {
        int m = (lo + hi + 1) >> 1;
        if (Team::ld(off + m) <= j) lo = m;
        else hi = m - 1;
    }
    return lo;
}

// The same search by the 32 lanes of a warp together (off[lo] <= j): every round probes 32
// evenly spaced offsets and keeps the stretch between the last probe <= j and the first probe
// > j, so R candidates take about log32(R) dependent loads instead of log2(R).  All lanes call
// it with the same arguments and all get the result.
template <class Team = GridTeam>
__device__ __forceinline__ int lb_seg_warp(const int *off, int j, int lo, int hi) {
    const int lane = threadIdx.x & 31;
    while (hi - lo >= 32) {
        const int step = (hi - lo + 31) / 32;
        const int q = min(lo + (lane + 1) * step, hi);
        const unsigned below = __ballot_sync(0xffffffffu, Team::ld(off + q) <= j);
        const int k = __popc(below);  // probes are ascending, so the true ones come first
        const int nlo = k == 0 ? lo : min(lo + k * step, hi);
        const int nhi = k == 32 ? hi : min(lo + (k + 1) * step, hi) - 1;
        lo = nlo;
        hi = nhi;
    }
    const int q = lo + 1 + lane;
    const unsigned below = __ballot_sync(0xffffffffu, q <= hi && Team::ld(off + q) <= j);
    return lo + __popc(below);
}

// Shared staging buffer of the block schedule (one per kernel).
__device__ __forceinline__ int *lb_stage() {
    __shared__ int buf[kLbStage + 2];
    return buf;
}

// Calls fn(j, n, s, end) for every run of n <= kLbItems consecutive items [j, j + n) owned by
// this thread, s = the segment of item j and end(x) = off[x + 1] for the segments of the run's
// tile.  fn must not use block-wide barriers or warp-collective operations.
template <class Fn, class Team = GridTeam>
__device__ __forceinline__ void lb_schedule(const int *off, int nseg, int total, const int *ts,
                                            Team t, Fn fn) {
    if (ts) {
        const int lane = threadIdx.x & 31;
        const int64_t tiles = ((int64_t)total + kWarpTile - 1) / kWarpTile;
        auto end = [&](int x) { return Team::ld(off + x + 1); };
        for (int64_t w = t.warp(); w < tiles; w += t.warps()) {
            const int j0 = (int)(w * kWarpTile);
            const int j1 = (int)(w * kWarpTile + kWarpTile < total ? w * kWarpTile + kWarpTile : total);
            const int j = j0 + lane * kLbItems;
            if (j >= j1) continue;
            const int s0 = Team::ld(ts + w);
            const int s1 = j1 < total ? Team::ld(ts + w + 1) : nseg - 1;
            fn(j, j1 - j < kLbItems ? j1 - j : kLbItems, lb_seg<Team>(off, j, s0, s1), end);
        }
        return;
    }
    __shared__ int s_rng[2];
    int *st = lb_stage();
    const int tile = blockDim.x * kLbItems;
    for (int64_t t0 = (int64_t)t.block() * tile; t0 < total; t0 += (int64_t)t.blocks() * tile) {
        const int j0 = (int)t0;
        const int j1 = (int)(t0 + tile < total ? t0 + tile : total);
        __syncthreads();  // the previous tile is done with the stage
        const int w = threadIdx.x >> 5;
        if (w < 2) {
            const int x = lb_seg_warp<Team>(off, w == 0 ? j0 : j1 - 1, 0, nseg - 1);
            if ((threadIdx.x & 31) == 0) s_rng[w] = x;
        }
        __syncthreads();
        const int s0 = s_rng[0], s1 = s_rng[1];
        const int cnt = s1 - s0 + 2;
        const bool staged = cnt <= kLbStage + 2;
        if (staged)
            for (int i = threadIdx.x; i < cnt; i += blockDim.x) st[i] = Team::ld(off + s0 + i);
        __syncthreads();
        const int j = j0 + threadIdx.x * kLbItems;
        if (j >= j1) continue;
        int s;
        if (staged) {
            int lo = 0, hi = s1 - s0;
            while (lo < hi) {
                int m = (lo + hi + 1) >> 1;
                if (st[m] <= j) lo = m;
                else hi = m - 1;
            }
            s = s0 + lo;
        } else {
            s = lb_seg<Team>(off, j, s0, s1);
        }
        auto end = [&](int x) { return staged ? st[x - s0 + 1] : Team::ld(off + x + 1); };
        fn(j, j1 - j < kLbItems ? j1 - j : kLbItems, s, end);
    }
}

// Segmented reduction over a CSR for a visit that reads one int per item: items[j] is loaded
// for all of the thread's slots up front (one 16-byte load when its kLbItems slots are in range
// and aligned); visit(seg, items[j], acc) folds it in and flush(seg, acc) ends every segment run
// of the thread.  `init` is the identity of the combine operation.
template <class Acc, class Visit, class Flush, class Team = GridTeam>
__device__ __forceinline__ void lb_for_each_items(const int *off, int nseg, int total, const int *items,
                                                  Acc init, Visit visit, Flush flush, Team t = Team(),
                                                  const int *ts = nullptr) {
    static_assert(kLbItems == 4, "one int4 load per thread");
    lb_schedule(off, nseg, total, ts, t, [&](int j, int n, int s, auto end) {
        int it[kLbItems];
        if (n == kLbItems && ((reinterpret_cast<uintptr_t>(items + j) & 15) == 0)) {
            const int4 a = Team::ld(reinterpret_cast<const int4 *>(items + j));
            it[0] = a.x; it[1] = a.y; it[2] = a.z; it[3] = a.w;
        } else {
#pragma unroll
            for (int k = 0; k < kLbItems; ++k) it[k] = k < n ? Team::ld(items + j + k) : 0;
        }
        int send = end(s);
        Acc acc = init;
#pragma unroll
        for (int k = 0; k < kLbItems; ++k) {
            if (k < n) {
                while (j + k >= send) {  // next non-empty segment
                    flush(s, acc);
                    acc = init;
                    ++s;
                    send = end(s);
                }
                acc = visit(s, it[k], acc);
            }
        }
        flush(s, acc);
    });
}

// The same reduction where the last run of every thread is first combined (op, a cooperative
// groups operator such as plus or less) with the last runs of the lanes that end in the same
// segment, so a segment spanning many threads (a coarse node's long incidence list) takes one
// atomic per warp instead of one per thread.
template <class Acc, class Op, class Visit, class Flush, class Team = GridTeam>
__device__ __forceinline__ void lb_reduce_items(const int *off, int nseg, int total, const int *items,
                                                Acc init, Op op, Visit visit, Flush flush,
                                                Team t = Team(), const int *ts = nullptr) {
    static_assert(kLbItems == 4, "one int4 load per thread");
    lb_schedule(off, nseg, total, ts, t, [&](int j, int n, int s, auto end) {
        int it[kLbItems];
        if (n == kLbItems && ((reinterpret_cast<uintptr_t>(items + j) & 15) == 0)) {
            const int4 a = Team::ld(reinterpret_cast<const int4 *>(items + j));
            it[0] = a.x; it[1] = a.y; it[2] = a.z; it[3] = a.w;
        } else {
#pragma unroll
            for (int k = 0; k < kLbItems; ++k) it[k] = k < n ? Team::ld(items + j + k) : 0;
        }
        int send = end(s);
        Acc acc = init;
#pragma unroll
        for (int k = 0; k < kLbItems; ++k) {
            if (k < n) {
                while (j + k >= send) {  // next non-empty segment
                    if (acc != init) flush(s, acc);
                    acc = init;
                    ++s;
                    send = end(s);
                }
                acc = visit(s, it[k], acc);
            }
        }
        namespace cg = cooperative_groups;
        const cg::coalesced_group lanes = cg::coalesced_threads();
        const cg::coalesced_group same = cg::labeled_partition(lanes, s);
        const Acc r = cg::reduce(same, acc, op);
        if (same.thread_rank() == 0 && r != init) flush(s, r);
    });
}

// Calls fn(s, a, b) for every maximal run [a, b) of this thread's items that lies in segment s,
// in item order (per-segment values can then be loaded once per run).
template <class Fn, class Team = GridTeam>
__device__ __forceinline__ void lb_runs(const int *off, int nseg, int total, Fn fn, Team t = Team(),
                                        const int *ts = nullptr) {
    lb_schedule(off, nseg, total, ts, t, [&](int j, int n, int s, auto end) {
        const int je = j + n;
        while (j < je) {
            const int send = end(s);
            const int b = send < je ? send : je;
            if (b > j) fn(s, j, b);
            j = b > j ? b : j;
            ++s;
        }
    });
}

inline int lb_grid(int64_t total, int cap = 152 * 8) {
    int64_t b = (total + kLbTile - 1) / kLbTile;
    if (b < 1) b = 1;
    return (int)(b < cap ? b : cap);
}

}  // namespace bp
