// The coarse tail of a bisection run as one thread-block-cluster launch (tail.cu): arguments,
// limits, and the arena layout of the coarse levels it builds, which the host mirrors to expose
// those levels as views.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include "refine_dev.cuh"

namespace bp {

constexpr int kTailThreads = 512;         // threads per block of the cluster
constexpr int kTailNodes = 12288;         // largest level (nodes) the tail can start from
constexpr int64_t kTailMaxPins = 4'000'000;  // ... and pins (its shared-memory chunk table)
// Default start: the first level of at most this many pins.  A sweep of the start on the 1M-node
// netlist (graph replay, one GB300) measured 2.694 ms per bisection from 70K pins, 2.73 ms from
// 170K, 2.86 ms from 420K and 3.17 ms from 800K, against 2.68-2.72 ms with the grid path alone:
// above ~70K pins the grid's 152 SMs outrun one cluster; below it the tail removes ~50 launches
// and, in the eager first call, the host round trips of the small levels.
constexpr int64_t kTailStartPins = 70'000;
constexpr int kTailMaxLevels = 64;        // coarse levels one tail may build
constexpr int kTailMaxCluster = 16;
constexpr int kTailChunk = 2048;          // chunk boundaries of a level every this many pins
constexpr int kTailMaxChunks = 510;       // chunks one block may own (shared-memory table)

// Chunks of a level with P pins: chunk c holds the hyperedges whose first pin lies in
// [c * kTailChunk, (c + 1) * kTailChunk); K = ceil(P / kTailChunk).
__host__ __device__ inline int tail_chunks(int P) { return (P + kTailChunk - 1) / kTailChunk; }

struct TailArgs {
    // the starting level (normalised CSR and node weights; its cmap / matching are written)
    int N, E, P;
    const int *hoff, *pins, *hw, *nw;
    int *cmap, *match;
    int policy, max_new, iters, m0, m;
    long long limit0, limit1;
    char *arena;  // coarse levels, tail_layout() one after another
    size_t arena_cap;
    // scratch: per hyperedge of the starting level (sizes and weights of the matched sets, group
    // representatives, staged offsets and weights of contracted hyperedges, work lists of 2E),
    // per pin (2P: staged coarse pins, then distinct pins of wide hyperedges at fine offsets),
    // per node, the starting level's chunk table and the blocks' compaction totals
    int *e_ssize, *e_sweight;
    unsigned *e_rep;
    int *e_soff, *e_shw, *e_list, *p_stage, *n_grp;
    int *ce0, *cp0;  // chunk table of the starting level (tail_chunks(P) + 1 entries each)
    long long *xchg;
    int *sizes;  // {N', E', P'} of every new level (max_new triples; zero past the last)
    int *info;   // [0] new levels built, [1] MiB of arena a run needed but did not have,
                 // [2] algorithmic KiB the launch moved
    uint8_t *side_out;  // bisection of the starting level
    RState *gst;        // the handle's refinement state: warn of the starting level's rebalance
    uint32_t *status;
    unsigned long long *trace;  // diagnostics (BIPART_TAIL_TRACE, eager calls): phase time stamps
};

constexpr int kTailTraceMax = 8192;

// Byte offsets of one coarse level's arrays in the arena (64-byte aligned; every array is
// followed by at least 16 bytes of slack so aligned 16-byte loads may run past its end).
struct TailLayout {
    size_t nw, cmap, match, ce, cp, hoff, hw, pins, end;
};

__host__ __device__ inline size_t tail_round(size_t bytes) { return (bytes + 16 + 63) & ~size_t(63); }

__host__ __device__ inline TailLayout tail_layout(size_t base, int N, int E, int P, bool weighted) {
    TailLayout t;
    size_t o = base;
    const size_t n = (size_t)(N > 0 ? N : 1), e = (size_t)(E > 0 ? E : 1), p = (size_t)(P > 0 ? P : 1);
    const size_t k = (size_t)tail_chunks(P) + 1;
    t.nw = o;    o += tail_round(4 * n);
    t.cmap = o;  o += tail_round(4 * n);
    t.match = o; o += tail_round(4 * n);
    t.ce = o;    o += tail_round(4 * k);
    t.cp = o;    o += tail_round(4 * k);
    t.hoff = o;  o += tail_round(4 * ((size_t)E + 1));
    t.hw = o;    if (weighted) o += tail_round(4 * e);
    t.pins = o;  o += tail_round(4 * p);
    t.end = o;
    return t;
}

}  // namespace bp
