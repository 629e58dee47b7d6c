// Cut evaluation that allocates no device memory (bipart_cut_noalloc in include/bipart.h).
//
// Who needs it: callers that cannot call cudaMalloc at the point where they want a cut -- for
// example a host application that hands all of HBM to its own memory pool up front, so any
// allocation by a library fails or breaks the pool's accounting, or a latency-critical loop that
// cannot afford the device-wide synchronisation an allocation may imply.  They pass the
// hypergraph, the partition and the output slot in device memory they already own; the only
// scratch is the fixed-size array below, which is part of this library's device image.
//
// Scratch: g_cut_scratch holds, per call, a small header (completion counter, error flag), the
// per-block partial sums of the final reduction and lambda_e for every hyperedge.  It is sized
// for at most kCutNoAllocMaxHedges hyperedges (16 MiB plus 33 KiB on every GPU that loads the
// library, held until the process exits).  Every call uses the same array: calls that overlap
// on the GPU (different streams, or different host threads on the same device) race on it and
// must be serialised by the caller.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"

namespace bp {
namespace {

constexpr int kCutNoAllocMaxHedges = 1 << 22;  // 4,194,304 hyperedges
constexpr int kCutNoAllocMaxParts = 64;
constexpr int kNaBlock = 256;
constexpr int kNaMaxBlocks = 1024;
// layout in 8-byte words: [0] counter, [1] error flag, [64 .. 64+kNaMaxBlocks) partials,
// then kCutNoAllocMaxHedges int32 lambda values
constexpr size_t kNaHeaderWords = 64;
constexpr size_t kNaWords = kNaHeaderWords + kNaMaxBlocks + kCutNoAllocMaxHedges / 2;

static __device__ __align__(256) unsigned long long g_cut_scratch[kNaWords];

constexpr int kMaxDevices = 64;
std::mutex g_na_mu;
unsigned long long *g_na_ptr[kMaxDevices] = {};

// lambda_e = number of distinct parts among the pins of e (0 for an empty hyperedge); a pin
// outside [0, N), a part outside [0, k) or a hyperedge weight below 1 raises the error flag
// instead of being used.  Hyperedges of degree <= 32 take one thread; larger ones are handled by
// the whole warp with a shuffle OR reduction of the part masks.
__global__ void __launch_bounds__(kNaBlock)
k_na_lambda(int N, int E, const int *__restrict__ hoff, const int *__restrict__ pins,
            const int *__restrict__ hw, const int *__restrict__ parts, int k,
            unsigned long long *__restrict__ scratch) {
    int *lambda = reinterpret_cast<int *>(scratch + kNaHeaderWords + kNaMaxBlocks);
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    bool bad = false;
    for (int e0 = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; e0 < E; e0 += warps * 32) {
        int e = e0 + lane;
        int a = 0, d = 0;
        if (e < E) {
            a = hoff[e];
            d = hoff[e + 1] - a;
            if (hw && hw[e] < 1) bad = true;
        }
        bool small = e < E && d <= 32;
        if (small) {
            unsigned long long m = 0;
            for (int i = 0; i < d; ++i) {
                int v = pins[a + i];
                int p = (v >= 0 && v < N) ? parts[v] : -1;
                if (p < 0 || p >= k) bad = true;
                else m |= 1ull << p;
            }
            lambda[e] = __popcll(m);
        }
        unsigned big = __ballot_sync(0xffffffffu, e < E && !small);
        while (big) {
            int src = __ffs(big) - 1;
            big &= big - 1;
            int eb = e0 + src;
            int ab = hoff[eb], db = hoff[eb + 1] - ab;
            unsigned long long m = 0;
            for (int i = lane; i < db; i += 32) {
                int v = pins[ab + i];
                int p = (v >= 0 && v < N) ? parts[v] : -1;
                if (p < 0 || p >= k) bad = true;
                else m |= 1ull << p;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m |= __shfl_xor_sync(0xffffffffu, m, o);
            if (lane == 0) lambda[eb] = __popcll(m);
        }
    }
    if (bad) atomicOr(&scratch[1], 1ull);
}

// cut = sum_e w_e * max(lambda_e - 1, 0): per-block partials in the scratch, then the last block
// to finish adds them in block order (a fixed order, so the sum is reproducible) and writes the
// caller's output (-1 when a pin, a part or a weight was out of range).
__global__ void __launch_bounds__(kNaBlock)
k_na_reduce(int E, const int *__restrict__ hw, unsigned long long *__restrict__ scratch,
            long long *__restrict__ out) {
    __shared__ unsigned long long red[33];
    __shared__ bool last;
    const int *lambda = reinterpret_cast<const int *>(scratch + kNaHeaderWords + kNaMaxBlocks);
    unsigned long long *partials = scratch + kNaHeaderWords;
    unsigned long long s = 0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
        int l = lambda[e];
        if (l > 1) s += (unsigned long long)(hw ? hw[e] : 1) * (unsigned long long)(l - 1);
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = s;
        __threadfence();
        last = atomicAdd(&scratch[0], 1ull) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    unsigned long long t = 0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
        t += *((volatile unsigned long long *)&partials[b]);
    t = block_sum(t, red);
    if (threadIdx.x == 0) {
        bool bad = *((volatile unsigned long long *)&scratch[1]) != 0;
        *out = bad ? -1ll : (long long)t;
    }
}

}  // namespace
}  // namespace bp

using namespace bp;

// The first call on a device looks up the scratch array's device address with that device
// current (cudaGetSymbolAddress); later calls on the device reuse it.  Make that first call
// before any stream capture begins.
extern "C" int bipart_cut_noalloc(int32_t num_nodes, int32_t num_hedges,
                                  const int32_t *d_hedge_offsets, const int32_t *d_hedge_pins,
                                  const int32_t *d_hedge_weights, const int32_t *d_parts,
                                  int32_t k, int64_t *d_cut, void *stream) {
    if (num_nodes < 0 || num_hedges < 0) {
        set_error("bipart_cut_noalloc: negative size");
        return BIPART_ERR_INVALID_ARG;
    }
    if (num_hedges > kCutNoAllocMaxHedges) {
        set_error("bipart_cut_noalloc: " + std::to_string(num_hedges) +
                  " hyperedges exceed the fixed scratch limit of " +
                  std::to_string(kCutNoAllocMaxHedges));
        return BIPART_ERR_INVALID_ARG;
    }
    if (k < 1 || k > kCutNoAllocMaxParts) {
        set_error("bipart_cut_noalloc: k must be in [1, 64]");
        return BIPART_ERR_INVALID_ARG;
    }
    if (!d_cut || (num_hedges > 0 && (!d_hedge_offsets || !d_hedge_pins || !d_parts))) {
        set_error("bipart_cut_noalloc: NULL argument");
        return BIPART_ERR_INVALID_ARG;
    }
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        set_error(std::string("bipart_cut_noalloc: no usable device: ") + cudaGetErrorString(err));
        return BIPART_ERR_CUDA;
    }
    unsigned long long *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (!g_na_ptr[dev]) {
            void *p = nullptr;
            err = cudaGetSymbolAddress(&p, g_cut_scratch);
            if (err != cudaSuccess || !p) {
                set_error(std::string("bipart_cut_noalloc: cudaGetSymbolAddress failed: ") +
                          cudaGetErrorString(err));
                return BIPART_ERR_CUDA;
            }
            g_na_ptr[dev] = static_cast<unsigned long long *>(p);
        }
        scratch = g_na_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    // counter and error flag must start at zero; the rest is fully overwritten
    err = cudaMemsetAsync(scratch, 0, 2 * sizeof(unsigned long long), s);
    if (err != cudaSuccess) {
        set_error(std::string("bipart_cut_noalloc: ") + cudaGetErrorString(err));
        return BIPART_ERR_CUDA;
    }
    int grid = num_hedges > 0 ? (num_hedges + kNaBlock - 1) / kNaBlock : 1;
    if (grid > kNaMaxBlocks) grid = kNaMaxBlocks;
    if (num_hedges > 0) {
        k_na_lambda<<<grid, kNaBlock, 0, s>>>(num_nodes, num_hedges, d_hedge_offsets, d_hedge_pins,
                                              d_hedge_weights, d_parts, k, scratch);
        note_launch();
    }
    k_na_reduce<<<grid, kNaBlock, 0, s>>>(num_hedges, d_hedge_weights, scratch,
                                          reinterpret_cast<long long *>(d_cut));
    note_launch();
    err = cudaGetLastError();
    if (err != cudaSuccess) {
        set_error(std::string("bipart_cut_noalloc: launch failed: ") + cudaGetErrorString(err));
        return BIPART_ERR_CUDA;
    }
    return BIPART_OK;
}
