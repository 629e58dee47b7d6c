// Single-pass device-wide exclusive scan (decoupled look-back, Merrill & Garland 2016) over
// 62-bit unsigned values produced on the fly by an input functor and consumed by an output
// functor.  Callers pack two counters into one value (high field << 31 | low field) when both
// stay below 2^31; the sum then never carries between fields.
//
// Tile states are 64-bit words: bits 62-63 hold the flag (0 = not ready, 1 = tile aggregate,
// 2 = inclusive prefix) and bits 0-61 the value, so one aligned store publishes both.  Tiles take
// their index from an atomic counter in launch order, so every tile only waits on tiles that
// already run; each wait is bounded by kSpinLimit polls and reports DEV_TIMEOUT on expiry.
#pragma once

#include "common.cuh"
#include "internal.h"

namespace bp {

// Grid scans: tiles of 2048 items, two per thread of a 1024-thread block (a same-box A/B on the
// 1M-node bisection: 256 x 8 took 2.652 ms, 512 x 4 2.568, 512 x 2 2.555, 1024 x 2 2.548 -- more
// warps to cover each tile's loads and look-back, shorter per-thread runs).
constexpr int kScanBlock = 1024;
constexpr int kScanItems = 2;
constexpr int kScanTile = kScanBlock * kScanItems;
// One-block scans (block_scan_items) keep eight items per thread: there the block's own loop, not
// the look-back, is the cost.
constexpr int kBlockScanItems = 8;
constexpr uint64_t kScanValMask = (1ull << 62) - 1;
constexpr uint64_t kFlagAgg = 1ull << 62;
constexpr uint64_t kFlagPre = 2ull << 62;
constexpr int kLookR = 4;  // predecessors per lane in one look-back round

// `state` points at [tile counter, unused, tile status words ...], all zero at launch; the
// counter wraps back to zero with the last ticket.  `other` is the other half of the stream's
// scan state: its first `other_dirty` tile states, left by the previous multi-tile scan, are
// cleared here for the next one.  A single-tile scan touches neither.
template <class In, class Out>
__global__ void __launch_bounds__(kScanBlock)
k_scan(int64_t n, In in, Out out, unsigned long long *state, unsigned long long *other,
       int64_t other_dirty, uint32_t *status) {
    __shared__ uint64_t s_val[kScanTile];
    __shared__ uint64_t s_pre[kScanTile];
    __shared__ uint64_t red[33];
    __shared__ uint32_t s_tile;
    __shared__ uint64_t s_prefix;
    unsigned long long *tiles = state + 2;

    // a single-tile scan has no predecessor: it neither takes a ticket nor touches the state
    const bool solo = gridDim.x == 1;
    if (threadIdx.x == 0)
        s_tile = solo ? 0u : atomicInc(reinterpret_cast<unsigned *>(state), gridDim.x - 1u);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < other_dirty;
         i += (int64_t)gridDim.x * blockDim.x)
        other[2 + i] = 0ull;
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t base = tile * kScanTile;

#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k * kScanBlock + threadIdx.x;
        s_val[k * kScanBlock + threadIdx.x] = i < n ? (uint64_t)in(i) : 0ull;
    }
    __syncthreads();
    uint64_t loc[kScanItems];
    uint64_t sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        loc[k] = s_val[threadIdx.x * kScanItems + k];
        sum += loc[k];
    }
    uint64_t total;
    uint64_t excl = block_exclusive_scan<uint64_t>(sum, red, &total);

    if (solo) {
        if (threadIdx.x == 0) s_prefix = 0;
    } else if (threadIdx.x < 32) {
        // warp 0 looks back over its predecessors 32 * kLookR at a time: it adds aggregates up to
        // the nearest tile that already holds its inclusive prefix
        const int lane = threadIdx.x;
        uint64_t prefix = 0;
        if (tile == 0) {
            if (lane == 0) atomicExch(&tiles[0], (unsigned long long)(kFlagPre | (total & kScanValMask)));
        } else {
            if (lane == 0) atomicExch(&tiles[tile], (unsigned long long)(kFlagAgg | (total & kScanValMask)));
            // each lane reads kLookR consecutive predecessors: one round covers 32 * kLookR tiles
            int64_t j = tile - 1;
            for (;;) {
                uint64_t st[kLookR];
                bool bad = false, inc_here = false;
#pragma unroll
                for (int r = 0; r < kLookR; ++r) {
                    const int64_t idx = j - (int64_t)lane * kLookR - r;
                    st[r] = kFlagPre;  // before tile 0: an inclusive prefix of 0
                    if (idx >= 0) {
                        int spins = 0;
                        for (;;) {
                            st[r] = *((volatile unsigned long long *)&tiles[idx]);
                            if ((st[r] >> 62) != 0) break;
                            if (++spins > kSpinLimit) break;
                            if (spins > 64) __nanosleep(64);
                        }
                    }
                    bad |= (st[r] >> 62) == 0;
                    inc_here |= (st[r] >> 62) == 2;
                }
                if (__ballot_sync(0xffffffffu, bad)) {  // a predecessor never published
                    if (lane == 0) record_error(status, DEV_TIMEOUT);
                    break;
                }
                const unsigned inc = __ballot_sync(0xffffffffu, inc_here);
                const int stop_lane = inc ? __ffs(inc) - 1 : 32;  // lane holding the nearest inclusive
                uint64_t v = 0;
                bool stopped = false;
#pragma unroll
                for (int r = 0; r < kLookR; ++r) {
                    if (lane < stop_lane || (lane == stop_lane && !stopped)) v += st[r] & kScanValMask;
                    if (lane == stop_lane && (st[r] >> 62) == 2) stopped = true;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                prefix += v;
                if (inc) break;
                j -= 32 * kLookR;
            }
            if (lane == 0)
                atomicExch(&tiles[tile], (unsigned long long)(kFlagPre | ((prefix + total) & kScanValMask)));
        }
        if (lane == 0) s_prefix = prefix;
    }
    __syncthreads();
    uint64_t run = s_prefix + excl;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        s_pre[threadIdx.x * kScanItems + k] = run;
        run += loc[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k * kScanBlock + threadIdx.x;
        if (i < n) out(i, s_pre[k * kScanBlock + threadIdx.x], s_val[k * kScanBlock + threadIdx.x]);
    }
}

// Exclusive scan over n items by one block: chunks of blockDim * kBlockScanItems items, each thread
// owning kBlockScanItems consecutive ones; out(i, prefix, value) after all in() of the chunk.  Used
// where a whole phase runs in one block (small levels; the persistent batch kernel).
template <class In, class Out>
__device__ void block_scan_items(int64_t n, In in, Out out) {
    __shared__ uint64_t red[33];
    uint64_t carry = 0;
    const int64_t chunk = (int64_t)blockDim.x * kBlockScanItems;
    for (int64_t base = 0; base < n; base += chunk) {
        const int64_t i0 = base + (int64_t)threadIdx.x * kBlockScanItems;
        uint64_t v[kBlockScanItems], sum = 0;
#pragma unroll
        for (int k = 0; k < kBlockScanItems; ++k) {
            v[k] = i0 + k < n ? (uint64_t)in(i0 + k) : 0ull;
            sum += v[k];
        }
        uint64_t total;
        uint64_t run = carry + block_exclusive_scan<uint64_t>(sum, red, &total);
#pragma unroll
        for (int k = 0; k < kBlockScanItems; ++k) {
            if (i0 + k < n) out(i0 + k, run, v[k]);
            run += v[k];
        }
        carry += total;
        __syncthreads();
    }
}

// Launches the scan on `s` with the stream's scan state `ss` (single-tile scans use none).
template <class In, class Out>
void scan(int64_t n, In in, Out out, ScanState &ss, uint32_t *status, cudaStream_t s) {
    if (n <= 0) return;
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 1) {
        k_scan<In, Out><<<1, kScanBlock, 0, s>>>(n, in, out, nullptr, nullptr, 0, status);
        BP_LAUNCH();
        return;
    }
    unsigned long long *b = ss.halves(tiles, s);
    const int c = ss.clean, o = c ^ 1;
    k_scan<In, Out><<<(unsigned)tiles, kScanBlock, 0, s>>>(n, in, out, b + (size_t)c * ss.half_words,
                                                             b + (size_t)o * ss.half_words, ss.dirty[o], status);
    BP_LAUNCH();
    ss.dirty[c] = tiles;
    ss.dirty[o] = 0;
    ss.clean = o;
}

}  // namespace bp
