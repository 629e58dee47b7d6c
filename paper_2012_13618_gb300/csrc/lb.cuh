// Load-balanced segmented reductions over a CSR (offsets off[0..nseg], items [0, total)).
//
// A block owns kLbTile consecutive items; each thread owns kLbItems consecutive items of that
// tile, finds the segment of its first item by binary search inside the block's segment range
// and walks forward.  Per-segment partial results are flushed with one atomic per segment run,
// so a segment with 100,000 items costs the same per item as one with 2 items, and the result
// does not depend on the schedule when the combining operation is an integer sum or minimum.
#pragma once

#include "common.cuh"

namespace bp {

constexpr int kLbBlock = 256;
constexpr int kLbItems = 8;
constexpr int kLbTile = kLbBlock * kLbItems;

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

// Visits the items of this thread in order as (segment, item index) and calls
// flush(segment, acc) whenever the segment changes and at the end.  `init` is the identity of
// the combine operation; visit(seg, item, acc) folds one item into acc.  A tile is
// blockDim.x * kLbItems items; the team's blocks take tiles in turn.
template <class Acc, class Visit, class Flush, class Team = GridTeam>
__device__ __forceinline__ void lb_for_each(const int *off, int nseg, int total, Acc init,
                                            Visit visit, Flush flush, Team t = Team()) {
    __shared__ int s_rng[2];
    const int tile = blockDim.x * kLbItems;
    for (int64_t t0 = (int64_t)t.block() * tile; t0 < total; t0 += (int64_t)t.blocks() * tile) {
        const int j0 = (int)t0;
        const int j1 = (int)(t0 + tile < total ? t0 + tile : total);
        __syncthreads();
        if (threadIdx.x == 0) s_rng[0] = lb_seg<Team>(off, j0, 0, nseg - 1);
        if (threadIdx.x == 32) s_rng[1] = lb_seg<Team>(off, j1 - 1, 0, nseg - 1);
        __syncthreads();
        int j = j0 + threadIdx.x * kLbItems;
        if (j >= j1) continue;
        const int je = j + kLbItems < j1 ? j + kLbItems : j1;
        int s = lb_seg<Team>(off, j, s_rng[0], s_rng[1]);
        int send = Team::ld(off + s + 1);
        Acc acc = init;
        for (; j < je; ++j) {
            while (j >= send) {  // next non-empty segment
                flush(s, acc);
                acc = init;
                ++s;
                send = Team::ld(off + s + 1);
            }
            acc = visit(s, j, acc);
        }
        flush(s, acc);
    }
}

// As lb_for_each, for a visit that reads one int per item: items[j] is loaded for all of the
// thread's slots up front (two 16-byte loads when its kLbItems slots are in range and aligned),
// and visit(seg, items[j], acc) folds it in.
template <class Acc, class Visit, class Flush, class Team = GridTeam>
__device__ __forceinline__ void lb_for_each_items(const int *off, int nseg, int total, const int *items,
                                                  Acc init, Visit visit, Flush flush, Team t = Team()) {
    static_assert(kLbItems == 8, "two int4 loads per thread");
    __shared__ int s_rng[2];
    const int tile = blockDim.x * kLbItems;
    for (int64_t t0 = (int64_t)t.block() * tile; t0 < total; t0 += (int64_t)t.blocks() * tile) {
        const int j0 = (int)t0;
        const int j1 = (int)(t0 + tile < total ? t0 + tile : total);
        __syncthreads();
        if (threadIdx.x == 0) s_rng[0] = lb_seg<Team>(off, j0, 0, nseg - 1);
        if (threadIdx.x == 32) s_rng[1] = lb_seg<Team>(off, j1 - 1, 0, nseg - 1);
        __syncthreads();
        const int j = j0 + threadIdx.x * kLbItems;
        if (j >= j1) continue;
        const int n = j1 - j < kLbItems ? j1 - j : kLbItems;
        int it[kLbItems];
        if (n == kLbItems && ((reinterpret_cast<uintptr_t>(items + j) & 15) == 0)) {
            const int4 a = Team::ld(reinterpret_cast<const int4 *>(items + j));
            const int4 b = Team::ld(reinterpret_cast<const int4 *>(items + j) + 1);
            it[0] = a.x; it[1] = a.y; it[2] = a.z; it[3] = a.w;
            it[4] = b.x; it[5] = b.y; it[6] = b.z; it[7] = b.w;
        } else {
#pragma unroll
            for (int k = 0; k < kLbItems; ++k) it[k] = k < n ? Team::ld(items + j + k) : 0;
        }
        int s = lb_seg<Team>(off, j, s_rng[0], s_rng[1]);
        int send = Team::ld(off + s + 1);
        Acc acc = init;
#pragma unroll
        for (int k = 0; k < kLbItems; ++k) {
            if (k < n) {
                while (j + k >= send) {  // next non-empty segment
                    flush(s, acc);
                    acc = init;
                    ++s;
                    send = Team::ld(off + s + 1);
                }
                acc = visit(s, it[k], acc);
            }
        }
        flush(s, acc);
    }
}

// Calls fn(s, a, b) for every maximal run [a, b) of this thread's items that lies in segment s,
// in item order (per-segment values can then be loaded once per run).
template <class Fn, class Team = GridTeam>
__device__ __forceinline__ void lb_runs(const int *off, int nseg, int total, Fn fn, Team t = Team()) {
    __shared__ int s_rng[2];
    const int tile = blockDim.x * kLbItems;
    for (int64_t t0 = (int64_t)t.block() * tile; t0 < total; t0 += (int64_t)t.blocks() * tile) {
        const int j0 = (int)t0;
        const int j1 = (int)(t0 + tile < total ? t0 + tile : total);
        __syncthreads();
        if (threadIdx.x == 0) s_rng[0] = lb_seg<Team>(off, j0, 0, nseg - 1);
        if (threadIdx.x == 32) s_rng[1] = lb_seg<Team>(off, j1 - 1, 0, nseg - 1);
        __syncthreads();
        int j = j0 + threadIdx.x * kLbItems;
        if (j >= j1) continue;
        const int je = j + kLbItems < j1 ? j + kLbItems : j1;
        int s = lb_seg<Team>(off, j, s_rng[0], s_rng[1]);
        while (j < je) {
            const int send = Team::ld(off + s + 1);
            const int b = send < je ? send : je;
            if (b > j) fn(s, j, b);
            j = b > j ? b : j;
            ++s;
        }
    }
}

inline int lb_grid(int64_t total, int cap = 152 * 8) {
    int64_t b = (total + kLbTile - 1) / kLbTile;
    if (b < 1) b = 1;
    return (int)(b < cap ? b : cap);
}

}  // namespace bp
