// Shared device helpers of the sm_103a path: error plumbing, the matching hash, warp/block
// reductions and the bounded spin-wait used by every cross-block handshake.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>

#include "bipart.h"

namespace bp {

// Status word shared by kernels that can fail at run time (bounded waits, size overflows).
enum DevErr : uint32_t { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_OVERFLOW = 2, DEV_PLAN_MISMATCH = 4 };

// Spin limit of every device-side wait: after this many polls the waiting thread records
// DEV_TIMEOUT in the status word and carries on with a defined (wrong) value, so the kernel
// always terminates and the host reports BIPART_ERR_TIMEOUT.
constexpr int kSpinLimit = 1 << 22;

void set_error(const std::string &msg);

struct Fail {
    int code;
    std::string msg;
};

#define BP_CUDA(call)                                                                       \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            throw ::bp::Fail{BIPART_ERR_CUDA, std::string(#call) + ": " +                    \
                                                  cudaGetErrorString(e_)};                  \
    } while (0)

void note_launch();

#define BP_LAUNCH()                                                                         \
    do {                                                                                    \
        ::bp::note_launch();                                                                \
        cudaError_t e_ = cudaGetLastError();                                                \
        if (e_ != cudaSuccess)                                                              \
            throw ::bp::Fail{BIPART_ERR_CUDA, std::string("kernel launch at ") + __FILE__ + \
                                                  ":" + std::to_string(__LINE__) + ": " +   \
                                                  cudaGetErrorString(e_)};                  \
    } while (0)

// Matching hash (reading of Algorithm 1's hash(hedge.id)): the 32-bit finaliser of
// MurmurHash3 (Appleby), a bijection of 32-bit integers, so (priority, hash) is unique per
// hyperedge and the three atomicMin passes of Algorithm 1 collapse into one 64-bit minimum.
__host__ __device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x85ebca6bu;
    x ^= x >> 13;
    x *= 0xc2b2ae35u;
    x ^= x >> 16;
    return x;
}

// Multiplicative inverse of an odd 32-bit constant modulo 2^32 (Newton iteration).
constexpr uint32_t inv_odd32(uint32_t c) {
    uint32_t x = c;  // correct to 3 bits for odd c; each step doubles the correct bits
    for (int i = 0; i < 5; ++i) x *= 2u - c * x;
    return x;
}

// Inverse of mix32: undoes each xorshift and multiplication in reverse order, so the matched
// hyperedge can be read back from the low half of a winning (priority, hash) key.
__host__ __device__ __forceinline__ uint32_t unmix32(uint32_t x) {
    constexpr uint32_t i2 = inv_odd32(0xc2b2ae35u), i1 = inv_odd32(0x85ebca6bu);
    x ^= x >> 16;
    x *= i2;
    x ^= (x >> 13) ^ (x >> 26);
    x *= i1;
    x ^= x >> 16;
    return x;
}

// Table 1 priorities as a "smaller is preferred" 32-bit value.
__host__ __device__ __forceinline__ uint32_t policy_priority(int policy, uint32_t deg,
                                                             uint32_t w, uint32_t hash) {
    switch (policy) {
        case BIPART_POLICY_LDH: return deg;
        case BIPART_POLICY_HDH: return 0xFFFFFFFFu - deg;
        case BIPART_POLICY_LWD: return w;
        case BIPART_POLICY_HWD: return 0xFFFFFFFFu - w;
        default: return hash;
    }
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <class T>
__device__ __forceinline__ T warp_min(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u < v ? u : v;
    }
    return v;
}

template <class T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u > v ? u : v;
    }
    return v;
}

// Inclusive warp scan.
template <class T>
__device__ __forceinline__ T warp_inclusive_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Block-wide sum; `red` must hold >= 32 entries; all threads receive the total.
template <class T>
__device__ __forceinline__ T block_sum(T v, T *red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    T t = lane < nw ? red[lane] : T(0);
    if (wid == 0) t = warp_sum(t);
    if (threadIdx.x == 0) red[0] = t;
    __syncthreads();
    T r = red[0];
    __syncthreads();
    return r;
}

// Block-wide exclusive scan; returns this thread's exclusive prefix, total in *total.
template <class T>
__device__ __forceinline__ T block_exclusive_scan(T v, T *red, T *total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    T inc = warp_inclusive_scan(v);
    __syncthreads();
    if (lane == 31 || threadIdx.x == blockDim.x - 1) red[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        T t = lane < nw ? red[lane] : T(0);
        T ti = warp_inclusive_scan(t);
        if (lane < nw) red[lane] = ti - t;
        if (lane == nw - 1) red[32] = ti;
    }
    __syncthreads();
    T r = red[wid] + inc - v;
    *total = red[32];
    __syncthreads();
    return r;
}

__device__ __forceinline__ void record_error(uint32_t *status, uint32_t code) {
    if (status) atomicOr(status, code);
}

// True in the block of a grid launch that arrives here last, which also puts `counter` back to
// zero for the next launch.  Every block's global writes before the call are visible to that
// block (fence, then one counter atomic per block); it should read them through L2 (__ldcg).
__device__ __forceinline__ bool last_block(unsigned *counter) {
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned t = atomicAdd(counter, 1u);
        s_last = t == gridDim.x - 1;
        if (s_last) {
            *counter = 0u;
            __threadfence();
        }
    }
    __syncthreads();
    return s_last != 0;
}

inline int ceil_div_i(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Teams: the threads that share one phase of the algorithm.  GridTeam = every thread of a kernel
// launch (phases are separate launches); CtaTeam = one thread block that runs a whole instance
// (phases separated by __syncthreads).  ld() is the load used for data written by an earlier
// phase: the read-only path within a kernel launch, a coherent load inside a persistent block.
struct GridTeam {
    __device__ __forceinline__ int rank() const { return blockIdx.x * blockDim.x + threadIdx.x; }
    __device__ __forceinline__ int size() const { return gridDim.x * blockDim.x; }
    __device__ __forceinline__ int block() const { return blockIdx.x; }
    __device__ __forceinline__ int blocks() const { return gridDim.x; }
    __device__ __forceinline__ int warp() const { return rank() >> 5; }
    __device__ __forceinline__ int warps() const { return size() >> 5; }
    template <class T>
    __device__ __forceinline__ static T ld(const T *p) { return __ldg(p); }
};

// The blocks [b0, b0 + nb) of a grid launch, as a team of their own (a launch that runs two
// independent phases on disjoint sets of blocks).
struct SubGridTeam {
    int b0, nb;
    __device__ __forceinline__ int block() const { return blockIdx.x - b0; }
    __device__ __forceinline__ int blocks() const { return nb; }
    __device__ __forceinline__ int rank() const { return block() * blockDim.x + threadIdx.x; }
    __device__ __forceinline__ int size() const { return nb * blockDim.x; }
    __device__ __forceinline__ int warp() const { return rank() >> 5; }
    __device__ __forceinline__ int warps() const { return size() >> 5; }
    template <class T>
    __device__ __forceinline__ static T ld(const T *p) { return __ldg(p); }
};

struct CtaTeam {
    __device__ __forceinline__ int rank() const { return threadIdx.x; }
    __device__ __forceinline__ int size() const { return blockDim.x; }
    __device__ __forceinline__ int block() const { return 0; }
    __device__ __forceinline__ int blocks() const { return 1; }
    __device__ __forceinline__ int warp() const { return threadIdx.x >> 5; }
    __device__ __forceinline__ int warps() const { return blockDim.x >> 5; }
    template <class T>
    __device__ __forceinline__ static T ld(const T *p) { return *p; }
};

}  // namespace bp
