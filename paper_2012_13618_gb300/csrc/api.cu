// C ABI of the library (include/bipart.h): handle life cycle, input validation, the multilevel
// driver of Sec. 3.4 and the nested k-way recursion of Algorithm 6 (Sec. 3.5).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <exception>
#include <functional>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unistd.h>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "lb.cuh"
#include "scan.cuh"

namespace bp {

namespace {
thread_local std::string g_last_error;
std::mutex g_alloc_mu;  // guards the three below (set by bipart_set_allocator)
bipart_alloc_fn g_alloc = nullptr;
bipart_free_fn g_free = nullptr;
void *g_alloc_ctx = nullptr;
constexpr int kBlock = 256;
constexpr size_t kSmallBytes = 64 * 1024;

// Host threads that bisect the subgraphs of a recursion-tree level: 8, or $BIPART_KWAY_LANES.
int default_lanes() {
    static const int n = []() {
        const char *e = std::getenv("BIPART_KWAY_LANES");
        const int v = e ? std::atoi(e) : 0;
        return v >= 1 && v <= 64 ? v : 8;
    }();
    return n;
}

inline int grid_for(int64_t n, int per_block = kBlock, int cap = 152 * 16) {
    int64_t b = (n + per_block - 1) / per_block;
    if (b < 1) b = 1;
    return (int)std::min<int64_t>(b, cap);
}
}  // namespace

void set_error(const std::string &msg) { g_last_error = msg; }

thread_local bipart_graph *tl_graph = nullptr;   // handle of the entry point running
thread_local bool tl_capturing = false;

// Sets the handle whose buffers the current entry point (re)allocates.
struct HandleScope {
    bipart_graph *prev;
    explicit HandleScope(bipart_graph *g) : prev(tl_graph) { tl_graph = g; }
    ~HandleScope() { tl_graph = prev; }
};

void note_realloc() {
    if (tl_graph) tl_graph->gen++;
}

void *dev_alloc(size_t bytes, cudaStream_t s, AllocTag *tag) {
    if (tl_capturing) return nullptr;  // no allocation may happen inside a captured plan
    bipart_alloc_fn alloc;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        alloc = g_alloc;
        tag->free_fn = g_free;
        tag->ctx = g_alloc_ctx;
    }
    if (alloc) {
        if (tl_graph) tl_graph->ext_alloc = true;
        return alloc(tag->ctx, bytes, (void *)s);
    }
    tag->free_fn = nullptr;
    void *p = nullptr;
    cudaMemPool_t pool = lib_pool();
    const cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, s) : cudaMallocAsync(&p, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

// The library's own stream-ordered memory pool on the current device: freed memory stays
// reserved in it for the next allocation (no release threshold), instead of going back to the
// driver at every synchronisation as the device's default pool does.  Null if it cannot be made
// (the default pool is used then).
cudaMemPool_t lib_pool() {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    static bool tried[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (!tried[dev]) {
        tried[dev] = true;
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
            pools[dev] = pool;
        } else {
            cudaGetLastError();
        }
    }
    return pools[dev];
}

void lib_pool_trim() {
    if (cudaMemPool_t pool = lib_pool()) {
        cudaDeviceSynchronize();
        cudaMemPoolTrimTo(pool, 0);
    }
}

// Set on the thread that releases destroyed handles: their buffers are freed on its own stream
// (the handle's stream belongs to the caller, who may destroy it once bipart_destroy returns).
thread_local cudaStream_t tl_free_stream = nullptr;

void dev_free(void *p, size_t bytes, cudaStream_t s, const AllocTag &tag) {
    if (!p) return;
    if (tl_free_stream) s = tl_free_stream;
    if (tag.free_fn) tag.free_fn(tag.ctx, p, bytes, (void *)s);
    else cudaFreeAsync(p, s);
}

void zero_fill(void *p, size_t bytes, cudaStream_t s) { BP_CUDA(cudaMemsetAsync(p, 0, bytes, s)); }

// Pinned 4 KB host blocks for the small device-to-host reads of a handle, kept in a process-wide
// pool: pinning and unpinning memory costs far more than a short-lived handle's whole run.
namespace {
std::mutex g_pinned_mu;
std::vector<uint32_t *> g_pinned_free;
}  // namespace

uint32_t *pinned_take() {
    {
        std::lock_guard<std::mutex> lk(g_pinned_mu);
        if (!g_pinned_free.empty()) {
            uint32_t *p = g_pinned_free.back();
            g_pinned_free.pop_back();
            return p;
        }
    }
    void *p = nullptr;
    BP_CUDA(cudaMallocHost(&p, 4096));
    return static_cast<uint32_t *>(p);
}

void pinned_release(uint32_t *p) {
    std::lock_guard<std::mutex> lk(g_pinned_mu);
    g_pinned_free.push_back(p);
}

uint32_t *dev_status(bipart_graph *g) { return g->w.status.as<uint32_t>(); }

void sync(bipart_graph *g) {
    if (g->ex.capturing) return;
    BP_CUDA(cudaStreamSynchronize(g->stream));
}

// Reads the device status word on the handle's own stream (pinned staging), so concurrent
// handles on other streams are never serialised by it.
uint32_t read_status_word(bipart_graph *g) {
    BP_CUDA(cudaMemcpyAsync(g->w.host_small + 1023, dev_status(g), sizeof(uint32_t),
                            cudaMemcpyDeviceToHost, g->stream));
    BP_CUDA(cudaStreamSynchronize(g->stream));
    return g->w.host_small[1023];
}

void raise_status(uint32_t st) {
    if (st & DEV_TIMEOUT) throw Fail{BIPART_ERR_TIMEOUT, "a bounded device-side wait expired"};
    if (st & DEV_OVERFLOW) throw Fail{BIPART_ERR_OOM, "a device-side size limit was exceeded"};
}

void check_status(bipart_graph *g) {
    if (g->ex.capturing) return;
    raise_status(read_status_word(g));
}

// ------------------------------------------------------------------------- plans and conditionals
__global__ void k_expect(const int *d, int v, uint32_t *status) {
    if (threadIdx.x == 0 && *d != v) atomicOr(status, (uint32_t)DEV_PLAN_MISMATCH);
}

constexpr int kMaxChecks = 96;
struct Checks {
    int n;
    int slot[kMaxChecks];
    int32_t value[kMaxChecks];
};

__global__ void k_expect_all(const int32_t *base, Checks c, uint32_t *status) {
    for (int i = threadIdx.x; i < c.n; i += blockDim.x)
        if (base[c.slot[i]] != c.value[i]) atomicOr(status, (uint32_t)DEV_PLAN_MISMATCH);
}

// Per-level size slots in the small scratch, after the selection state.
constexpr int kSlotBase = 6144;   // int index (24 KB into the 64 KB scratch)
constexpr int kSlotLevels = 2048;

int32_t *level_sizes(bipart_graph *g, int idx) {
    int32_t *small = g->w.small.as<int32_t>();
    return idx < kSlotLevels - 1 ? small + kSlotBase + 3 * idx : small + 8;
}

// The last slot triple is kept for the cluster tail's level count, arena check and bytes.
int32_t *tail_info_slot(bipart_graph *g) {
    return g->w.small.as<int32_t>() + kSlotBase + 3 * (kSlotLevels - 1);
}

void read_i32s(bipart_graph *g, int n, const int32_t *const *d, int32_t *v) {
    Exec &ex = g->ex;
    if (ex.capturing) {
        for (int i = 0; i < n; ++i) v[i] = read_i32(g, d[i]);
        return;
    }
    // the values and the status word in one round trip
    for (int i = 0; i < n; ++i)
        BP_CUDA(cudaMemcpyAsync(g->w.host_small + i, d[i], sizeof(int32_t), cudaMemcpyDeviceToHost, g->stream));
    BP_CUDA(cudaMemcpyAsync(g->w.host_small + 1023, dev_status(g), sizeof(uint32_t), cudaMemcpyDeviceToHost,
                            g->stream));
    sync(g);
    raise_status(g->w.host_small[1023]);
    for (int i = 0; i < n; ++i) {
        v[i] = (int32_t)g->w.host_small[i];
        if (ex.recording) ex.sizes.push_back(v[i]);
    }
}

int32_t read_i32(bipart_graph *g, const int32_t *d) {
    Exec &ex = g->ex;
    if (ex.capturing) {
        if (ex.pos >= ex.sizes.size()) throw Fail{BIPART_ERR_CUDA, "plan capture ran past its recorded sizes"};
        int32_t v = ex.sizes[ex.pos++];
        const int32_t *small = g->w.small.as<int32_t>();
        const ptrdiff_t off = d - small;
        if (off >= kSlotBase && off < kSlotBase + 3 * kSlotLevels) {
            ex.checks.emplace_back((int)off, v);
        } else {
            k_expect<<<1, 32, 0, g->stream>>>(d, v, dev_status(g));
            BP_LAUNCH();
            ex.check_kernels++;
        }
        return v;
    }
    int32_t v;
    read_i32s(g, 1, &d, &v);
    return v;
}

void flush_checks(bipart_graph *g) {
    Exec &ex = g->ex;
    for (size_t i = 0; i < ex.checks.size(); i += kMaxChecks) {
        Checks c{};
        c.n = (int)std::min<size_t>(kMaxChecks, ex.checks.size() - i);
        for (int k = 0; k < c.n; ++k) {
            c.slot[k] = ex.checks[i + k].first;
            c.value[k] = ex.checks[i + k].second;
        }
        ProfScope ps("plan_check", 0.0, g->stream);
        k_expect_all<<<1, 128, 0, g->stream>>>(g->w.small.as<int32_t>(), c, dev_status(g));
        BP_LAUNCH();
        ex.check_kernels++;
    }
    ex.checks.clear();
}

unsigned read_flag(bipart_graph *g, const unsigned *d) {
    BP_CUDA(cudaMemcpyAsync(g->w.host_small, d, sizeof(unsigned), cudaMemcpyDeviceToHost, g->stream));
    sync(g);
    return g->w.host_small[0];
}

// Flag slots in the small scratch, after the level size slots.
constexpr int kFlagBase = kSlotBase + 3 * kSlotLevels;  // int index
constexpr int kFlagSlots = 16384 - kFlagBase;

unsigned *flag_slot(bipart_graph *g) {
    Exec &ex = g->ex;
    if (!ex.capturing) return nullptr;
    if (ex.flag_next >= kFlagSlots) throw Fail{BIPART_ERR_CUDA, "too many control decisions to capture"};
    ex.flag_pending = ex.flag_next++;
    return reinterpret_cast<unsigned *>(g->w.small.as<int32_t>() + kFlagBase + ex.flag_pending);
}

bool device_flag(bipart_graph *g, const unsigned *d_flag) {
    Exec &ex = g->ex;
    if (ex.capturing) {
        if (ex.flag_pos >= ex.flags.size()) throw Fail{BIPART_ERR_CUDA, "plan capture ran past its recorded decisions"};
        if (ex.flag_pending < 0) throw Fail{BIPART_ERR_CUDA, "control decision without a slot"};
        const bool v = ex.flags[ex.flag_pos++] != 0;
        ex.checks.emplace_back(kFlagBase + ex.flag_pending, v ? 1 : 0);
        ex.flag_pending = -1;
        return v;
    }
    const bool v = read_flag(g, d_flag) != 0;
    if (ex.recording) ex.flags.push_back(v ? 1 : 0);
    return v;
}

void Plan::reset() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (Probe &p : probes) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    probes.clear();
    exec = nullptr;
    graph = nullptr;
    valid = false;
}

// ------------------------------------------------------------------------- validation kernels
__global__ void k_validate(int N, int E, int P, const int *__restrict__ hoff,
                           const int *__restrict__ pins, const int *__restrict__ nw,
                           const int *__restrict__ hw, unsigned *__restrict__ bad,
                           unsigned long long *__restrict__ sums) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    unsigned b = 0;
    unsigned long long sn = 0, se = 0;
    if (tid == 0 && hoff && hoff[0] != 0) b |= 1;
    for (int e = tid; e < E; e += nt) {
        if (hoff[e + 1] < hoff[e]) b |= 1;
        if (hw) {
            if (hw[e] < 1) b |= 4;
            se += (unsigned)max(hw[e], 0);
        }
    }
    for (int i = tid; i < P; i += nt)
        if (pins[i] < 0 || pins[i] >= N) b |= 2;
    for (int v = tid; v < N; v += nt) {
        if (nw) {
            if (nw[v] < 1) b |= 4;
            sn += (unsigned)max(nw[v], 0);
        } else {
            sn += 1;
        }
    }
    if (b) atomicOr(bad, b);
    sn = warp_sum(sn);
    se = warp_sum(se);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&sums[0], sn);
        atomicAdd(&sums[1], se);
    }
}

__global__ void k_weight_sum(int N, const int *__restrict__ nw, unsigned long long *out) {
    unsigned long long s = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) s += nw[v];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

// Tile-start table of a hyperedge CSR (the segment holding every kTsGran-th pin).
__global__ void k_mark_tiles(int E, const int *__restrict__ hoff, int *__restrict__ ts) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x)
        lb_mark_tiles(ts, e, hoff[e], hoff[e + 1] - hoff[e]);
}

// Side 0 of a subgraph keeps the part range starting at lo, side 1 takes the one starting at hi.
__global__ void k_side_to_part(int N, const uint8_t *__restrict__ side, const int *__restrict__ l2g,
                               int lo, int hi, int *__restrict__ part) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        int v = l2g ? l2g[i] : i;
        part[v] = side[i] ? hi : lo;
    }
}

// ------------------------------------------------------------------------- subgraph extraction
// Reading of Algorithm 6's subgraphs (net splitting): nodes of part j renumbered in ascending id;
// every hyperedge restricted to them kept when it has >= 2 pins, in ascending id, weight carried.
struct SubNodeIn {
    const int *part;
    int j;
    __device__ uint64_t operator()(int64_t v) const { return part[v] == j ? 1ull : 0ull; }
};
struct SubNodeOut {
    int64_t n;
    const int *nw;
    int *loc, *l2g, *sub_nw, *n_out;
    __device__ void operator()(int64_t v, uint64_t pre, uint64_t val) const {
        if (val) {
            loc[v] = (int)pre;
            l2g[pre] = (int)v;
            sub_nw[pre] = nw[v];
        } else {
            loc[v] = -1;
        }
        if (v == n - 1) *n_out = (int)(pre + val);
    }
};

__global__ void __launch_bounds__(kBlock)
k_sub_count(int E, const int *__restrict__ hoff, const int *__restrict__ pins,
            const int *__restrict__ loc, int *__restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    // hyperedges of degree <= 32: one thread; larger ones: the warp handles them cooperatively
    for (int e0 = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; e0 < E; e0 += warps * 32) {
        int e = e0 + lane;
        int a = 0, d = 0;
        if (e < E) { a = hoff[e]; d = hoff[e + 1] - a; }
        bool small = e < E && d <= 32;
        if (small) {
            int c = 0;
            for (int i = 0; i < d; ++i) c += loc[pins[a + i]] >= 0;
            cnt[e] = c;
        }
        unsigned bigmask = __ballot_sync(0xffffffffu, e < E && !small);
        while (bigmask) {
            int src = __ffs(bigmask) - 1;
            bigmask &= bigmask - 1;
            int eb = e0 + src;
            int ab = hoff[eb], db = hoff[eb + 1] - ab;
            int c = 0;
            for (int i = lane; i < db; i += 32) c += loc[pins[ab + i]] >= 0;
            c = warp_sum(c);
            if (lane == 0) cnt[eb] = c;
        }
    }
}

struct SubEdgeIn {
    const int *cnt;
    __device__ uint64_t operator()(int64_t e) const {
        int c = cnt[e];
        return c >= 2 ? ((1ull << 31) | (uint64_t)c) : 0ull;
    }
};
struct SubEdgeOut {
    int64_t n;
    const int *hw;
    int *hoff_out, *hw_out, *emap, *sizes, *ts;
    __device__ void operator()(int64_t e, uint64_t pre, uint64_t val) const {
        if (val) {
            int ei = (int)(pre >> 31);
            hoff_out[ei] = (int)(pre & 0x7fffffffu);
            lb_mark_tiles(ts, ei, (int64_t)(pre & 0x7fffffffu), (int64_t)(val & 0x7fffffffu));
            if (hw_out) hw_out[ei] = hw[e];
            emap[e] = ei;
        } else {
            emap[e] = -1;
        }
        if (e == n - 1) {
            uint64_t t = pre + val;
            hoff_out[(int)(t >> 31)] = (int)(t & 0x7fffffffu);
            sizes[0] = (int)(t >> 31);
            sizes[1] = (int)(t & 0x7fffffffu);
        }
    }
};

__global__ void __launch_bounds__(kBlock)
k_sub_copy(int E, const int *__restrict__ hoff, const int *__restrict__ pins,
           const int *__restrict__ loc, const int *__restrict__ emap,
           const int *__restrict__ hoff_out, int *__restrict__ pins_out, int *__restrict__ deg) {
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int e0 = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; e0 < E; e0 += warps * 32) {
        int e = e0 + lane;
        int a = 0, d = 0, ee = -1;
        if (e < E) { a = hoff[e]; d = hoff[e + 1] - a; ee = emap[e]; }
        bool small = ee >= 0 && d <= 32;
        if (small) {
            int o = hoff_out[ee];
            for (int i = 0; i < d; ++i) {
                int x = loc[pins[a + i]];
                if (x >= 0) {
                    pins_out[o++] = x;
                    atomicAdd(deg + x, 1);
                }
            }
        }
        unsigned bigmask = __ballot_sync(0xffffffffu, ee >= 0 && d > 32);
        while (bigmask) {
            int src = __ffs(bigmask) - 1;
            bigmask &= bigmask - 1;
            int eb = e0 + src;
            int ab = hoff[eb], db = hoff[eb + 1] - ab;
            int o = hoff_out[emap[eb]];
            for (int i0 = 0; i0 < db; i0 += 32) {
                int i = i0 + lane;
                int x = i < db ? loc[pins[ab + i]] : -1;
                unsigned m = __ballot_sync(0xffffffffu, x >= 0);
                if (x >= 0) {
                    pins_out[o + __popc(m & ((1u << lane) - 1))] = x;
                    atomicAdd(deg + x, 1);
                }
                o += __popc(m);
            }
        }
    }
}

namespace {

// Builds the subgraph of part j of the parent's level 0 as the child's level 0 (node map in the
// child's l2g, weight total in its total_node_weight).  The extraction runs on the parent's stream
// with the parent's scratch, reads the subgraph's sizes back once, and copies into child buffers of
// exactly those sizes (a child keeps its buffers, and so its launch plan, from call to call).
void extract_subgraph(bipart_graph *g, const int *d_part, int j, bipart_graph *kid) {
    cudaStream_t s = g->stream;
    Level &L = g->L0;
    Level &S = kid->L0;
    Work &w = g->w;
    const size_t n1 = (size_t)std::max(L.N, 1), e1 = (size_t)std::max(L.E, 1);
    int *loc = (int *)w.n_c.ensure(sizeof(int) * n1, s);
    int *t_l2g = (int *)g->l2g.ensure(sizeof(int) * n1, s);
    int *t_nw = (int *)w.n_b.ensure(sizeof(int) * n1, s);
    int *t_hoff = (int *)w.e_c.ensure(sizeof(int) * (e1 + 1), s);
    int *t_hw = L.unit_hw ? nullptr : (int *)w.e_d.ensure(sizeof(int) * e1, s);
    int *cnt = (int *)w.e_a.ensure(sizeof(int) * e1, s);
    int *emap = (int *)w.e_b.ensure(sizeof(int) * e1, s);
    int *small = w.small.as<int>();
    unsigned long long *wsum = reinterpret_cast<unsigned long long *>(small + 8);
    BP_CUDA(cudaMemsetAsync(small, 0, 12 * sizeof(int), s));
    scan(L.N, SubNodeIn{d_part, j}, SubNodeOut{L.N, L.nw(), loc, t_l2g, t_nw, small + 4}, w.scan,
         dev_status(g), s);
    if (L.E > 0) {
        int gw = grid_for((int64_t)(L.E + 31) / 32 * 32);
        k_sub_count<<<gw, kBlock, 0, s>>>(L.E, L.hoff(), L.pins(), loc, cnt);
        BP_LAUNCH();
        scan(L.E, SubEdgeIn{cnt}, SubEdgeOut{L.E, L.hw(), t_hoff, t_hw, emap, small + 2, nullptr},
             w.scan, dev_status(g), s);
    }
    BP_CUDA(cudaMemcpyAsync(w.host_small, small, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
    BP_CUDA(cudaMemcpyAsync(w.host_small + 4, small + 4, sizeof(int), cudaMemcpyDeviceToHost, s));
    sync(g);
    check_status(g);
    const int N = L.N > 0 ? (int)w.host_small[4] : 0;
    const int E = L.E > 0 ? (int)w.host_small[2] : 0;
    const int P = L.E > 0 ? (int)w.host_small[3] : 0;
    cudaStream_t ks = kid->stream;
    {
        HandleScope hs(kid);
        S.clear_view();
        S.N = N;
        S.E = E;
        S.P = P;
        S.unit_hw = L.unit_hw;
        kid->l2g.ensure(sizeof(int) * (size_t)std::max(N, 1), ks);
        S.b_nw.ensure(sizeof(int) * (size_t)std::max(N, 1), ks);
        S.b_hoff.ensure(sizeof(int) * ((size_t)E + 1), ks);
        S.b_pins.ensure(sizeof(int) * (size_t)std::max(P, 1), ks);
        S.b_tsh.ensure(sizeof(int) * ((size_t)P / kTsGran + 2), ks);
        if (!S.unit_hw) S.b_hw.ensure(sizeof(int) * (size_t)std::max(E, 1), ks);
        S.b_cmap.ensure(sizeof(int) * (size_t)std::max(N, 1), ks);
        S.b_match.ensure(sizeof(int) * (size_t)std::max(N, 1), ks);
        degree_counters(kid, N);  // sized (the counts come from the parent below)
    }
    // the kid's new buffers were allocated on its stream: the parent's copies wait for them
    cudaEvent_t ev = nullptr;
    BP_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    BP_CUDA(cudaEventRecord(ev, ks));
    BP_CUDA(cudaStreamWaitEvent(s, ev, 0));
    cudaEventDestroy(ev);
    if (N > 0) {
        BP_CUDA(cudaMemcpyAsync(kid->l2g.p, t_l2g, sizeof(int) * (size_t)N, cudaMemcpyDeviceToDevice, s));
        BP_CUDA(cudaMemcpyAsync(S.nw(), t_nw, sizeof(int) * (size_t)N, cudaMemcpyDeviceToDevice, s));
    }
    int *deg = degree_counters(g, N);  // subgraph degrees, counted while its pins are written
    if (E > 0) {
        BP_CUDA(cudaMemcpyAsync(S.hoff(), t_hoff, sizeof(int) * ((size_t)E + 1), cudaMemcpyDeviceToDevice, s));
        if (t_hw) BP_CUDA(cudaMemcpyAsync(S.b_hw.p, t_hw, sizeof(int) * (size_t)E, cudaMemcpyDeviceToDevice, s));
        int gw = grid_for((int64_t)(L.E + 31) / 32 * 32);
        k_sub_copy<<<gw, kBlock, 0, s>>>(L.E, L.hoff(), L.pins(), loc, emap, S.hoff(), S.pins(), deg);
        BP_LAUNCH();
        k_mark_tiles<<<grid_for(E), kBlock, 0, s>>>(E, S.hoff(), S.tsh());
        BP_LAUNCH();
    } else {
        BP_CUDA(cudaMemsetAsync(S.hoff(), 0, sizeof(int), s));
    }
    if (N > 0) BP_CUDA(cudaMemcpyAsync(kid->w.n_a.p, deg, sizeof(int) * (size_t)N, cudaMemcpyDeviceToDevice, s));
    if (N > 0) {
        k_weight_sum<<<grid_for(N), kBlock, 0, s>>>(N, t_nw, wsum);
        BP_LAUNCH();
    }
    BP_CUDA(cudaMemcpyAsync(w.host_small, wsum, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    sync(g);
    unsigned long long W = 0;
    std::memcpy(&W, w.host_small, sizeof(W));
    kid->total_node_weight = (int64_t)W;
}

}  // namespace


namespace {

// Sec. 3.4: coarsen until `levels` levels exist or the node count stops changing (reading C11),
// then initial partition + refinement back to level 0.  Coarse levels live in g->lev; the side
// of level 0 goes to d_side and the status word (level-0 rebalance imbalanced) stays on device.
void bisect_body(bipart_graph *g, Level &L0, const Params &p, int64_t W, uint8_t *d_side, int *nlev) {
    // Counters, histograms and scan tile states are zero at rest (each phase clears what it
    // used); they are cleared once here in case an earlier run stopped midway.
    BP_CUDA(cudaMemsetAsync(g->w.small.p, 0, small_state_bytes(), g->stream));
    g->w.scan.reset(g->stream);
    std::vector<Level *> levels{&L0};
    const int64_t limit[2] = {balance_limit(W, p.m0, p.m, p.e6), balance_limit(W, p.m - p.m0, p.m, p.e6)};
    // Levels are coarsened by the grid kernels until one is small enough for the cluster tail,
    // which then runs the rest of the bisection down to that level in one launch.
    int tail_from = g->allow_tail && tail_eligible(L0, p.levels, p.flags) ? 0 : -1;
    bool init_done = false;  // the next level's key and reset pass already ran
    while (tail_from < 0 && (int)levels.size() - 1 < p.levels) {
        Level &f = *levels.back();
        if (f.E == 0) break;  // with no hyperedge nothing merges: N' == N
        size_t idx = levels.size() - 1;
        if (g->lev.size() <= idx) g->lev.emplace_back(new Level);
        Level &c = *g->lev[idx];
        c.clear_view();
        prof_level('c', (int)idx);
        const int tail_new = p.levels - (int)idx - 1;  // contractions allowed after c
        bool to_tail = false;  // decided by coarsen_level, which then leaves c's incidence out
        init_done = coarsen_level(g, f, c, p.policy, level_sizes(g, (int)idx),
                                  (p.flags & BIPART_FLAG_MERGE_PARALLEL) != 0, init_done,
                                  (int)idx + 1 < p.levels, tail_new, p.flags,
                                  g->allow_tail ? &to_tail : nullptr);
        if (c.N == f.N) break;
        levels.push_back(&c);
        if (to_tail) tail_from = (int)levels.size() - 1;
    }
    g->last_tail_from = tail_from;
    if (tail_from >= 0) {
        // the tail leaves the side of its starting level in side_a, sized for level 0 here so
        // that uncoarsen() finds it in place
        g->w.side_b.ensure((size_t)std::max(L0.N, 1), g->stream);
        uint8_t *sa = (uint8_t *)g->w.side_a.ensure((size_t)std::max(L0.N, 1), g->stream);
        prof_level('t', tail_from);
        run_tail(g, levels, p, limit, sa);
    }
    if (nlev) *nlev = (int)levels.size();
    uncoarsen(g, levels, limit, p.m0, p.m, p.iters, d_side, tail_from);
    prof_level(0, 0);
    if (g->ex.capturing) flush_checks(g);
}

int read_bisect_status(bipart_graph *g) {
    BP_CUDA(cudaMemcpyAsync(g->w.host_small, bisect_status_word(g), sizeof(unsigned),
                            cudaMemcpyDeviceToHost, g->stream));
    sync(g);
    return g->w.host_small[0] ? BIPART_WARN_IMBALANCED : BIPART_OK;
}

// Captures the bisection just run eagerly (its sizes recorded) into a CUDA graph with WHILE / IF
// nodes for the device-driven loops.  Best effort: on any failure the plan stays invalid and the
// next call runs eagerly again.
void capture_plan(bipart_graph *g, const Params &p, uint8_t *d_side, int nlev, int64_t kernels) {
    Plan &pl = g->plan;
    pl.reset();
    Exec &ex = g->ex;
    const uint64_t gen0 = g->gen;
    ex.capturing = true;
    ex.pos = 0;
    ex.flag_pos = 0;
    ex.flag_next = 0;
    ex.flag_pending = -1;
    ex.checks.clear();
    ex.check_kernels = 0;
    tl_capturing = true;
    // the graph is captured on a private stream and launched on the handle's stream, which may
    // be the legacy default stream (not capturable)
    cudaStream_t main = g->stream;
    cudaGraph_t graph = nullptr;
    bool ok = true;
    if (!g->cap_stream && cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        g->cap_stream = nullptr;
        ok = false;
    }
    if (ok && cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) ok = false;
    if (ok) {
        g->stream = g->cap_stream;
        try {
            int n2 = 0;
            bisect_body(g, g->L0, p, g->total_node_weight, d_side, &n2);
            if (n2 != nlev) ok = false;
            pl.scan_clean = g->w.scan.clean;
            pl.scan_dirty[0] = g->w.scan.dirty[0];
            pl.scan_dirty[1] = g->w.scan.dirty[1];
        } catch (...) {
            ok = false;
        }
        g->stream = main;
        if (cudaStreamEndCapture(g->cap_stream, &graph) != cudaSuccess) ok = false;
    }
    ex.capturing = false;
    tl_capturing = false;
    cudaGetLastError();
    if (ok && (ex.pos != ex.sizes.size() || ex.flag_pos != ex.flags.size())) ok = false;
    if (ok && g->gen != gen0) ok = false;
    if (ok && cudaGraphInstantiate(&pl.exec, graph, 0) != cudaSuccess) ok = false;
    cudaGetLastError();
    pl.graph = graph;
    if (!ok) {
        if (std::getenv("BIPART_TIMING")) std::fprintf(stderr, "[bipart] plan capture failed; calls stay eager\n");
        pl.reset();
        return;
    }
    pl.valid = true;
    pl.params = p;
    pl.nlev = nlev;
    pl.gen = g->gen;
    pl.prof_epoch = prof_epoch();
    pl.launches = kernels + ex.check_kernels;
}

bool same_params(const Params &a, const Params &b) {
    return a.policy == b.policy && a.levels == b.levels && a.iters == b.iters && a.e6 == b.e6 &&
           a.m0 == b.m0 && a.m == b.m && a.flags == b.flags;
}

// Bisection of the handle's level 0.  First call with given parameters: eager, recording the
// level sizes.  Second call: captures those launches into a CUDA graph and launches it.  Later
// calls: launch the graph.  A replay whose device-side size checks fail (or a change of buffers
// or of profiling) drops the plan and runs eagerly again.
int bisect_top(bipart_graph *g, const Params &p, uint8_t *d_side, int *nlev) {
    Plan &pl = g->plan;
    Exec &ex = g->ex;
    g->last_replayed = false;
    // The cluster tail shortens an eager run (it replaces the small levels' host round trips),
    // while a captured plan runs faster with every level on the grid.  So the first eager run of a
    // parameter set may take the tail; the next one runs every level on the grid and is the
    // recording a plan is captured from.
    const bool have_rec = ex.rec_valid && same_params(ex.rec_params, p) && ex.rec_gen == g->gen;
    if (!(pl.valid && same_params(pl.params, p) && pl.gen == g->gen && pl.prof_epoch == prof_epoch())) {
        pl.reset();
        if (have_rec && !ex.rec_tail) {
            g->allow_tail = false;
            capture_plan(g, p, d_side, ex.rec_nlev, ex.rec_kernels);
        }
    }
    if (pl.valid) {
        // BIPART_TIMING: device time of the replay alone, on stderr (diagnostics)
        static const bool timing = std::getenv("BIPART_TIMING") != nullptr;
        cudaEvent_t t0 = nullptr, t1 = nullptr;
        if (timing) {
            cudaEventCreate(&t0);
            cudaEventCreate(&t1);
            cudaEventRecord(t0, g->stream);
        }
        BP_CUDA(cudaGraphLaunch(pl.exec, g->stream));
        g->w.scan.clean = pl.scan_clean;  // the device's scan state after the graph
        g->w.scan.dirty[0] = pl.scan_dirty[0];
        g->w.scan.dirty[1] = pl.scan_dirty[1];
        if (timing) cudaEventRecord(t1, g->stream);
        for (int64_t i = 0; i < pl.launches; ++i) note_launch();
        sync(g);
        if (timing) {
            float ms = 0;
            cudaEventElapsedTime(&ms, t0, t1);
            std::fprintf(stderr, "[bipart] graph replay %.3f ms (%lld launches)\n", ms, (long long)pl.launches);
            cudaEventDestroy(t0);
            cudaEventDestroy(t1);
        }
        const uint32_t st = read_status_word(g);
        if (!(st & DEV_PLAN_MISMATCH)) {
            check_status(g);
            prof_collect(pl.probes);
            *nlev = pl.nlev;
            g->last_replayed = true;
            return read_bisect_status(g);
        }
        // the replayed control flow did not match this run: discard the plan, run eagerly
        BP_CUDA(cudaMemsetAsync(dev_status(g), 0, sizeof(uint32_t), g->stream));
        pl.reset();
        ex.rec_valid = false;
    }
    g->allow_tail = !have_rec;
    ex.recording = true;
    ex.sizes.clear();
    ex.flags.clear();
    const int64_t k0 = bipart_kernel_launches();
    try {
        bisect_body(g, g->L0, p, g->total_node_weight, d_side, nlev);
    } catch (...) {
        ex.recording = false;
        throw;
    }
    ex.recording = false;
    const int64_t kernels = bipart_kernel_launches() - k0;
    int st = read_bisect_status(g);
    check_status(g);
    ex.rec_valid = true;
    ex.rec_params = p;
    ex.rec_gen = g->gen;
    ex.rec_nlev = *nlev;
    ex.rec_kernels = kernels;
    ex.rec_tail = g->last_tail_from >= 0;
    return st;
}

// Sec. 3.4 without the coarsening: Algorithm 3 on the coarsest kept level, then refinement and
// rebalancing back to level 0 with `iters` iterations and imbalance e6, on the hierarchy the
// handle's last k = 2 bisection built (its levels are kept).  Coarsening depends on neither
// quantity, so the result equals a full bisection with them.  Runs eagerly.
int refine_kept(bipart_graph *g, int64_t e6, int32_t iters, int *d_parts) {
    if (!g->hier.valid) throw Fail{BIPART_ERR_INVALID_ARG, "no k = 2 hierarchy kept (partition with k = 2 first)"};
    Params p = g->hier.params;
    p.e6 = e6;
    p.iters = iters;
    Level &L0 = g->L0;
    if (L0.N == 0) return BIPART_OK;
    cudaStream_t s = g->stream;
    BP_CUDA(cudaMemsetAsync(dev_status(g), 0, sizeof(uint32_t), s));
    BP_CUDA(cudaMemsetAsync(g->w.small.p, 0, small_state_bytes(), s));
    g->w.scan.reset(s);
    const int tail_from = g->hier.tail_from;
    // the grid levels (the tail rebuilds its own from its starting level, identically)
    const int grid_levels = tail_from >= 0 ? tail_from + 1 : g->hier.nlev;
    std::vector<Level *> levels{&L0};
    for (int l = 1; l < grid_levels; ++l) levels.push_back(g->lev[(size_t)l - 1].get());
    const int64_t W = g->total_node_weight;
    const int64_t limit[2] = {balance_limit(W, p.m0, p.m, p.e6), balance_limit(W, p.m - p.m0, p.m, p.e6)};
    uint8_t *d_side = (uint8_t *)g->side_out.ensure((size_t)L0.N, s);
    if (tail_from >= 0) {
        g->w.side_b.ensure((size_t)std::max(L0.N, 1), s);
        uint8_t *sa = (uint8_t *)g->w.side_a.ensure((size_t)std::max(L0.N, 1), s);
        run_tail(g, levels, p, limit, sa);
    }
    if ((int)levels.size() != g->hier.nlev) throw Fail{BIPART_ERR_CUDA, "kept hierarchy changed size"};
    uncoarsen(g, levels, limit, p.m0, p.m, p.iters, d_side, tail_from);
    int st = read_bisect_status(g);
    k_side_to_part<<<grid_for(L0.N), kBlock, 0, s>>>(L0.N, d_side, nullptr, 0, p.m0, d_parts);
    BP_LAUNCH();
    sync(g);
    check_status(g);
    return st;
}

// Nested k-way (Algorithm 6; readings C16, G1-G2 for any k): the subgraph owning the parts
// [lo, lo + m) is bisected with side 0 meant for ceil(m / 2) of them; its nodes carry lo as
// their part until their range holds one part.  Ranges of one tree level are bisected one after
// another, each as its own subgraph.
int partition_device(bipart_graph *g, const Params &p, int *d_parts) {
    cudaStream_t s = g->stream;
    Level &L = g->L0;
    g->hier.valid = false;
    if (L.N == 0) return BIPART_OK;
    if (p.k == 1) {
        BP_CUDA(cudaMemsetAsync(d_parts, 0, sizeof(int) * (size_t)L.N, s));
        return BIPART_OK;
    }
    uint8_t *d_side = (uint8_t *)g->side_out.ensure((size_t)L.N, s);
    BP_CUDA(cudaMemsetAsync(dev_status(g), 0, sizeof(uint32_t), s));
    int status = BIPART_OK;
    int nlev = 0;
    Params top = p;
    top.m = p.k;
    top.m0 = (p.k + 1) / 2;
    int st = bisect_top(g, top, d_side, &nlev);
    if (st != BIPART_OK) status = st;
    {
        ProfScope ps("side_to_part", 5.0 * L.N, s);
        k_side_to_part<<<grid_for(L.N), kBlock, 0, s>>>(L.N, d_side, nullptr, 0, top.m0, d_parts);
        BP_LAUNCH();
    }
    if (p.k == 2) {
        g->hier.nlev = nlev;
        g->hier.valid = true;
        g->hier.tail_from = g->last_tail_from;
        g->hier.params = top;
        sync(g);
        return status;
    }
    const int lanes = g->kid_lanes > 0 ? g->kid_lanes : default_lanes();
    if (lanes == 1 && g->lean) {
        // the coarse levels of the top bisection are not needed any more: their memory goes before
        // the subgraphs take theirs (and the top bisection's plan, which points into them)
        sync(g);
        g->plan.reset();
        g->ex.rec_valid = false;
        g->lev.clear();
        g->gen++;
    }
    int *pa = (int *)g->part_a.ensure(sizeof(int) * (size_t)L.N, s);
    BP_CUDA(cudaMemcpyAsync(pa, d_parts, sizeof(int) * (size_t)L.N, cudaMemcpyDeviceToDevice, s));
    // The subgraphs of each recursion-tree level: extracted one after another on this stream, then
    // bisected at the same time, each by the child workspace of its place in the tree (its own
    // stream, level store and launch plan; a result depends only on its subgraph).  With one lane
    // a single child workspace bisects every subgraph in turn on this stream (the memory of one
    // subgraph at a time; no launch plans are kept for them).
    const bool single = lanes == 1;
    std::vector<std::pair<int32_t, int32_t>> ranges{{0, top.m0}, {top.m0, p.k - top.m0}};
    size_t kid_base = 0;
    while (!ranges.empty()) {
        std::vector<std::pair<int32_t, int32_t>> next, jobs;
        for (const auto &r : ranges) {
            if (r.second < 2) continue;
            jobs.push_back(r);
            const int32_t m0 = (r.second + 1) / 2;
            next.emplace_back(r.first, m0);
            next.emplace_back(r.first + m0, r.second - m0);
        }
        if (jobs.empty()) break;
        while (g->kids.size() < (single ? 1 : kid_base + jobs.size())) {
            if (single) {  // one after another on this handle's stream
                g->kids.emplace_back(graph_new(s));
                g->kids.back()->kid_own_stream = false;
                continue;
            }
            cudaStream_t ks = nullptr;
            BP_CUDA(cudaStreamCreateWithFlags(&ks, cudaStreamNonBlocking));
            g->kids.emplace_back(graph_new(ks));
        }
        auto kid_of = [&](size_t i) { return g->kids[single ? 0 : kid_base + i].get(); };
        auto extract = [&](size_t i) {
            bipart_graph *kid = kid_of(i);
            if (single || !kid->kid_stamp_valid || kid->kid_stamp.k != p.k || !same_params(kid->kid_stamp, p)) {
                // another tree (or another input): the child's subgraph changes, so its plan goes
                kid->plan.reset();
                kid->ex.rec_valid = false;
                kid->kid_stamp = p;
                kid->kid_stamp_valid = true;
            }
            extract_subgraph(g, pa, jobs[i].first, kid);
            // the subgraph is in place once the parent's stream gets here
            BP_CUDA(cudaEventRecord(g->kid_ready, s));
        };
        if (!single)
            for (size_t i = 0; i < jobs.size(); ++i) extract(i);
        std::vector<int> st(jobs.size(), BIPART_OK);
        std::vector<Fail> errs(jobs.size(), Fail{BIPART_OK, ""});
        auto job = [&](int i) {
            bipart_graph *kid = kid_of((size_t)i);
            try {
                HandleScope hs(kid);
                const int32_t lo = jobs[(size_t)i].first, m = jobs[(size_t)i].second;
                Params q = p;
                q.m = m;
                q.m0 = (m + 1) / 2;
                BP_CUDA(cudaStreamWaitEvent(kid->stream, g->kid_ready, 0));
                build_incidence(kid, kid->L0);
                if (kid->L0.N > 0) {
                    uint8_t *ds = (uint8_t *)kid->side_out.ensure((size_t)kid->L0.N, kid->stream);
                    int nl = 0;
                    st[(size_t)i] = bisect_top(kid, q, ds, &nl);
                    k_side_to_part<<<grid_for(kid->L0.N), kBlock, 0, kid->stream>>>(
                        kid->L0.N, ds, kid->l2g.as<int>(), lo, lo + q.m0, d_parts);
                    BP_LAUNCH();
                }
                BP_CUDA(cudaEventRecord(kid->kid_done, kid->stream));
            } catch (const Fail &e) {
                errs[(size_t)i] = e;
                cudaEventRecord(kid->kid_done, kid->stream);
            }
        };
        if (single) {
            for (int i = 0; i < (int)jobs.size(); ++i) {
                extract((size_t)i);
                job(i);
                if (errs[(size_t)i].code != BIPART_OK) throw errs[(size_t)i];
            }
        } else if (jobs.size() == 1) {
            job(0);
        } else {
            if (!g->lanes) g->lanes.reset(new Lanes(lanes));
            g->lanes->run((int)jobs.size(), job);
        }
        for (size_t i = 0; i < jobs.size(); ++i) {
            BP_CUDA(cudaStreamWaitEvent(s, kid_of(i)->kid_done, 0));
            if (errs[i].code != BIPART_OK) throw errs[i];
            if (st[i] != BIPART_OK) status = st[i];
        }
        kid_base += jobs.size();
        if (!next.empty())
            BP_CUDA(cudaMemcpyAsync(pa, d_parts, sizeof(int) * (size_t)L.N, cudaMemcpyDeviceToDevice, s));
        ranges.swap(next);
    }
    sync(g);
    return status;
}

}  // namespace

void validate_params(int32_t k, double eps, int32_t policy, int32_t levels, int32_t iters) {
    if (k < 1) throw Fail{BIPART_ERR_INVALID_ARG, "k must be >= 1"};
    if (!(eps >= 0.0 && eps <= 1000.0)) throw Fail{BIPART_ERR_INVALID_ARG, "epsilon must be in [0, 1000]"};
    if (policy < BIPART_POLICY_LDH || policy > BIPART_POLICY_RAND) throw Fail{BIPART_ERR_INVALID_ARG, "unknown policy"};
    if (levels < 0) throw Fail{BIPART_ERR_INVALID_ARG, "levels must be >= 0"};
    if (iters < 0) throw Fail{BIPART_ERR_INVALID_ARG, "refine_iters must be >= 0"};
}

namespace {

// Base-10^9 digits, least significant first: enough for the powers compared below.
using Digits = std::vector<uint64_t>;

void mul_small(Digits &a, uint64_t f) {
    uint64_t carry = 0;
    for (uint64_t &d : a) {
        const unsigned __int128 t = (unsigned __int128)d * f + carry;
        d = (uint64_t)(t % 1000000000u);
        carry = (uint64_t)(t / 1000000000u);
    }
    while (carry) {
        a.push_back(carry % 1000000000u);
        carry /= 1000000000u;
    }
}

bool less_equal(const Digits &a, const Digits &b) {
    if (a.size() != b.size()) return a.size() < b.size();
    for (size_t i = a.size(); i-- > 0;)
        if (a[i] != b[i]) return a[i] < b[i];
    return true;
}

}  // namespace

// Reading G3: the imbalance every bisection of a k-way partition may use so that the L =
// ceil(log2 k) nested allowances multiply to at most 1 + e: the largest x <= e6 (millionths)
// with (10^6 + x)^L <= (10^6 + e6) * 10^(6 (L - 1)), compared exactly.
int64_t adaptive_e6(int64_t e6, int32_t k) {
    int L = 0;
    while ((int64_t(1) << L) < k) ++L;
    if (L <= 1) return e6;
    Digits bound{1};
    mul_small(bound, (uint64_t)(1000000 + e6));
    for (int i = 1; i < L; ++i) mul_small(bound, 1000000u);
    int64_t lo = 0, hi = e6;
    while (lo < hi) {
        const int64_t x = hi - (hi - lo) / 2;
        Digits pw{1};
        for (int i = 0; i < L; ++i) mul_small(pw, (uint64_t)(1000000 + x));
        if (less_equal(pw, bound)) lo = x;
        else hi = x - 1;
    }
    return lo;
}

Params make_params(int32_t k, double eps, int32_t policy, int32_t levels, int32_t iters,
                   int32_t flags) {
    validate_params(k, eps, policy, levels, iters);
    if (flags & ~(BIPART_FLAG_ADAPTIVE_EPS | BIPART_FLAG_MERGE_PARALLEL))
        throw Fail{BIPART_ERR_INVALID_ARG, "unknown flags"};
    Params p;
    p.k = k;
    p.eps = eps;
    p.policy = policy;
    p.levels = levels;
    p.iters = iters;
    p.flags = flags;
    const int64_t e6 = llround(eps * 1e6);
    p.e6 = (flags & BIPART_FLAG_ADAPTIVE_EPS) ? adaptive_e6(e6, k) : e6;
    p.m0 = 1;
    p.m = 2;
    return p;
}

namespace {

// A fixed set of host worker threads for the long validation loops, started on first use so
// that creating a handle does not pay for thread starts.  One job runs at a time; the calling
// thread works on it too.  A forked child (which inherits no threads) starts a pool of its own;
// pools live until the process exits.
class HostPool {
public:
    static HostPool &get() {
        static std::mutex m;
        static HostPool *pool = nullptr;
        static pid_t owner = 0;
        std::lock_guard<std::mutex> lk(m);
        if (!pool || owner != getpid()) {
            pool = new HostPool();
            owner = getpid();
        }
        return *pool;
    }
    // fn(i) for every i in [0, n), shared out to the workers; returns when all have finished.
    void run(int n, const std::function<void(int)> &fn) {
        std::lock_guard<std::mutex> one_job(run_m_);
        {
            std::lock_guard<std::mutex> lk(m_);
            job_ = &fn;
            n_ = n;
            next_.store(0);
            pending_ = (int)workers_.size();
            ++gen_;
        }
        cv_.notify_all();
        work(fn, n);
        std::unique_lock<std::mutex> lk(m_);
        done_.wait(lk, [&] { return pending_ == 0; });
        job_ = nullptr;
    }

private:
    std::mutex run_m_, m_;
    std::condition_variable cv_, done_;
    const std::function<void(int)> *job_ = nullptr;
    int n_ = 0, pending_ = 0;
    uint64_t gen_ = 0;
    std::atomic<int> next_{0};
    std::vector<std::thread> workers_;

    HostPool() {
        const int hw = (int)std::thread::hardware_concurrency();
        const int T = std::max(1, std::min(hw, 16)) - 1;
        for (int i = 0; i < T; ++i) workers_.emplace_back([this] { loop(); });
    }
    void work(const std::function<void(int)> &fn, int n) {
        for (int i; (i = next_.fetch_add(1)) < n;) fn(i);
    }
    void loop() {
        uint64_t seen = 0;
        std::unique_lock<std::mutex> lk(m_);
        for (;;) {
            cv_.wait(lk, [&] { return gen_ != seen; });
            seen = gen_;
            const std::function<void(int)> *job = job_;
            const int n = n_;
            lk.unlock();
            work(*job, n);
            lk.lock();
            if (--pending_ == 0) done_.notify_one();
        }
    }
};

constexpr int64_t kHostChunk = 1 << 18;
constexpr int64_t kHostBlock = 4096;

// First i in [lo, hi) with bad(i), checked a block at a time with a branch-free OR (a loop the
// compiler vectorises); the exact index is searched only inside a failing block.
template <class Bad>
int64_t first_bad(int64_t lo, int64_t hi, Bad bad) {
    for (int64_t b0 = lo; b0 < hi; b0 += kHostBlock) {
        const int64_t b1 = std::min(hi, b0 + kHostBlock);
        unsigned any = 0;
        for (int64_t i = b0; i < b1; ++i) any |= bad(i) ? 1u : 0u;
        if (any)
            for (int64_t i = b0; i < b1; ++i)
                if (bad(i)) return i;
    }
    return -1;
}

}  // namespace

// Host-side validation of a CSR given in host memory.  The four arrays (offsets, pins, node and
// hyperedge weights) are cut into chunks of kHostChunk entries that all run as ONE job on the host
// pool; each chunk keeps its first offending index (and its weight sum), and the error reported is
// the one a sequential pass would meet first: offsets, then pins, then node weights, hyperedge
// weights and the weight sums.  hedge_pins is read up to hoff[E] entries, its documented length.
// Returns the total node weight.
int64_t validate_host_csr(int32_t N, int32_t E, const int32_t *hoff, const int32_t *pins,
                          const int32_t *nw, const int32_t *hw) {
    if (N < 0 || E < 0) throw Fail{BIPART_ERR_INVALID_ARG, "negative size"};
    if (E > 0 && !hoff) throw Fail{BIPART_ERR_INVALID_ARG, "hedge_offsets is NULL"};
    if (hoff && hoff[0] != 0) throw Fail{BIPART_ERR_INVALID_CSR, "hedge_offsets[0] != 0"};
    const int32_t P = E > 0 ? hoff[E] : 0;  // a negative total fails the offsets check
    const bool pins_null = P > 0 && !pins;
    enum { kOff, kPins, kNw, kHw, kArrays };
    const int64_t len[kArrays] = {E, pins_null ? 0 : std::max(P, 0), nw ? N : 0, hw ? E : 0};
    int64_t first_task[kArrays + 1];
    first_task[0] = 0;
    for (int a = 0; a < kArrays; ++a) first_task[a + 1] = first_task[a] + (len[a] + kHostChunk - 1) / kHostChunk;
    const int tasks = (int)first_task[kArrays];
    std::vector<int64_t> first((size_t)tasks, -1), sum((size_t)tasks, 0);
    auto body = [&](int t) {
        int a = 0;
        while (t >= first_task[a + 1]) ++a;
        const int64_t lo = (t - first_task[a]) * kHostChunk, hi = std::min(len[a], lo + kHostChunk);
        if (a == kOff) {
            first[(size_t)t] = first_bad(lo, hi, [&](int64_t e) { return hoff[e + 1] < hoff[e]; });
        } else if (a == kPins) {
            first[(size_t)t] = first_bad(lo, hi, [&](int64_t i) { return (uint32_t)pins[i] >= (uint32_t)N; });
        } else {
            const int32_t *w = a == kNw ? nw : hw;
            int64_t acc = 0;
            for (int64_t i = lo; i < hi; ++i) acc += w[i];
            sum[(size_t)t] = acc;
            first[(size_t)t] = first_bad(lo, hi, [&](int64_t i) { return (uint32_t)w[i] - 1u >= 0x7fffffffu; });
        }
    };
    if (tasks <= 1) {
        for (int t = 0; t < tasks; ++t) body(t);
    } else {
        HostPool::get().run(tasks, body);
    }
    auto first_of = [&](int a) {
        for (int64_t t = first_task[a]; t < first_task[a + 1]; ++t)
            if (first[(size_t)t] >= 0) return first[(size_t)t];
        return int64_t(-1);
    };
    auto sum_of = [&](int a) {
        int64_t acc = 0;
        for (int64_t t = first_task[a]; t < first_task[a + 1]; ++t) acc += sum[(size_t)t];
        return acc;
    };
    int64_t bad = first_of(kOff);
    if (bad >= 0) throw Fail{BIPART_ERR_INVALID_CSR, "hedge_offsets not non-decreasing at " + std::to_string(bad)};
    if (pins_null) throw Fail{BIPART_ERR_INVALID_ARG, "hedge_pins is NULL"};
    bad = first_of(kPins);
    if (bad >= 0) throw Fail{BIPART_ERR_INVALID_CSR, "pin " + std::to_string(bad) + " out of range"};
    if (nw && first_of(kNw) >= 0) throw Fail{BIPART_ERR_INVALID_CSR, "node weight < 1"};
    if (hw && first_of(kHw) >= 0) throw Fail{BIPART_ERR_INVALID_CSR, "hyperedge weight < 1"};
    const int64_t sn = nw ? sum_of(kNw) : N, se = hw ? sum_of(kHw) : 0;
    if (sn >= (int64_t(1) << 31) || se >= (int64_t(1) << 31))
        throw Fail{BIPART_ERR_INVALID_CSR, "weight sum must stay below 2^31"};
    return sn;
}

}  // namespace bp

bipart_graph::~bipart_graph() {
    lanes.reset();
    kids.clear();
    plan.reset();
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (kid_ready) cudaEventDestroy(kid_ready);
    if (kid_done) cudaEventDestroy(kid_done);
    if (w.host_small) bp::pinned_release(w.host_small);
    w.host_small = nullptr;
}

void bp::KidDel::operator()(bipart_graph *g) const {
    cudaStream_t s = g->kid_own_stream ? g->stream : nullptr;
    delete g;
    if (s) cudaStreamDestroy(s);
}

namespace bp {
namespace {

bipart_graph *new_graph(cudaStream_t s) {
    std::unique_ptr<bipart_graph> g(new bipart_graph);
    BP_CUDA(cudaGetDevice(&g->device));
    g->stream = s;
    g->w.status.ensure(64, s);
    g->w.small.ensure(kSmallBytes, s);
    BP_CUDA(cudaMemsetAsync(g->w.status.p, 0, 64, s));
    g->w.host_small = pinned_take();
    BP_CUDA(cudaEventCreateWithFlags(&g->kid_ready, cudaEventDisableTiming));
    BP_CUDA(cudaEventCreateWithFlags(&g->kid_done, cudaEventDisableTiming));
    refine_init();
    coarsen_init();
    return g.release();
}

// Level 0 of a validated CSR of P pins and total node weight W (both known from the validation).
void finish_create(bipart_graph *g, int32_t N, int32_t E, int32_t P, int64_t W, const int *d_hoff,
                   const int *d_pins, const int *d_nw, const int *d_hw) {
    build_level0(g, g->L0, N, E, P, d_hoff, d_pins, d_nw, d_hw);
    g->total_node_weight = W;
    sync(g);
    check_status(g);
}

// Device-side check of a CSR already on the device: bit 0 malformed offsets, bit 1 a pin out of
// range, bit 2 a weight below 1, bit 3 a weight sum of 2^31 or more; also the node-weight total.
// Every loop of the check is bounded by N, E and P, so it is safe on any content (hoff may be null
// when E = 0).
struct DevCheck {
    unsigned bad = 0;
    int64_t node_weight = 0;
};

DevCheck device_check(bipart_graph *g, int32_t N, int32_t E, int32_t P, const int *hoff, const int *pins,
                      const int *nw, const int *hw) {
    cudaStream_t s = g->stream;
    unsigned *bad = reinterpret_cast<unsigned *>(g->w.small.as<char>() + 48 * 1024);
    unsigned long long *sums = reinterpret_cast<unsigned long long *>(g->w.small.as<char>() + 48 * 1024 + 16);
    BP_CUDA(cudaMemsetAsync(bad, 0, 64, s));
    if (E > 0 || N > 0) {
        k_validate<<<grid_for(std::max<int64_t>({(int64_t)N, (int64_t)E, (int64_t)P})), kBlock, 0, s>>>(
            N, E, P, E > 0 ? hoff : nullptr, pins, nw, hw, bad, sums);
        BP_LAUNCH();
    }
    BP_CUDA(cudaMemcpyAsync(g->w.host_small, bad, 64, cudaMemcpyDeviceToHost, s));
    sync(g);
    DevCheck r;
    r.bad = g->w.host_small[0];
    unsigned long long hs[2];
    std::memcpy(hs, g->w.host_small + 4, sizeof(hs));
    if (hs[0] >= (1ull << 31) || hs[1] >= (1ull << 31)) r.bad |= 8;
    r.node_weight = (int64_t)hs[0];
    return r;
}

}  // namespace

// Workspace for the executor: a handle on its own stream with no hypergraph loaded yet.
bipart_graph *graph_new(cudaStream_t s) { return new_graph(s); }

// Destroyed handles released on a background thread, one stream of its own per device.
namespace {
struct Releaser {
    std::mutex mu;
    std::condition_variable cv;
    std::deque<bipart_graph *> q;
    cudaStream_t streams[64] = {};
    Releaser() { std::thread([this]() { loop(); }).detach(); }
    void loop() {
        for (;;) {
            bipart_graph *g = nullptr;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv.wait(lk, [&]() { return !q.empty(); });
                g = q.front();
                q.pop_front();
            }
            const int dev = g->device;
            if (dev >= 0 && dev < 64 && cudaSetDevice(dev) == cudaSuccess) {
                if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess)
                    streams[dev] = nullptr;
                tl_free_stream = streams[dev];
            }
            cudaGetLastError();
            delete g;
            tl_free_stream = nullptr;
        }
    }
};
}  // namespace

bool release_later(bipart_graph *g) {
    static Releaser *r = new Releaser;  // never destroyed: handles pending at exit go with the process
    if (g->device < 0 || g->device >= 64) return false;
    {
        std::lock_guard<std::mutex> lk(r->mu);
        r->q.push_back(g);
    }
    r->cv.notify_one();
    return true;
}

// Loads a host CSR into an existing handle, reusing its buffers (validated first).
void graph_load_host(bipart_graph *g, int32_t N, int32_t E, const int32_t *hoff, const int32_t *pins,
                     const int32_t *nw, const int32_t *hw) {
    HandleScope hs(g);
    const int64_t W = validate_host_csr(N, E, hoff, pins, nw, hw);
    cudaStream_t s = g->stream;
    const int32_t P = E > 0 ? hoff[E] : 0;
    int *d_hoff = (int *)g->in_hoff.ensure(sizeof(int) * ((size_t)E + 1), s);
    int *d_pins = (int *)g->in_pins.ensure(sizeof(int) * (size_t)std::max(P, 1), s);
    int *d_nw = nw ? (int *)g->in_nw.ensure(sizeof(int) * (size_t)std::max(N, 1), s) : nullptr;
    int *d_hw = hw ? (int *)g->in_hw.ensure(sizeof(int) * (size_t)std::max(E, 1), s) : nullptr;
    if (E > 0) BP_CUDA(cudaMemcpyAsync(d_hoff, hoff, sizeof(int) * ((size_t)E + 1), cudaMemcpyHostToDevice, s));
    if (P > 0) BP_CUDA(cudaMemcpyAsync(d_pins, pins, sizeof(int) * (size_t)P, cudaMemcpyHostToDevice, s));
    if (d_nw && N > 0) BP_CUDA(cudaMemcpyAsync(d_nw, nw, sizeof(int) * (size_t)N, cudaMemcpyHostToDevice, s));
    if (d_hw && E > 0) BP_CUDA(cudaMemcpyAsync(d_hw, hw, sizeof(int) * (size_t)E, cudaMemcpyHostToDevice, s));
    g->plan.reset();
    g->ex.rec_valid = false;
    g->hier.valid = false;
    g->gen++;
    for (auto &kid : g->kids) kid->kid_stamp_valid = false;  // new input: new subgraphs
    finish_create(g, N, E, P, W, E > 0 ? d_hoff : nullptr, d_pins, d_nw, d_hw);
}

// Partitions the loaded hypergraph into host memory (blocking on the handle's stream).
int graph_partition_host(bipart_graph *g, const Params &p, int32_t *out) {
    HandleScope hs(g);
    const int32_t N = g->L0.N;
    int *d = (int *)g->part_b.ensure(sizeof(int) * (size_t)std::max(N, 1), g->stream);
    int st = partition_device(g, p, d);
    if (N > 0) BP_CUDA(cudaMemcpyAsync(out, d, sizeof(int) * (size_t)N, cudaMemcpyDeviceToHost, g->stream));
    sync(g);
    check_status(g);
    return st;
}

namespace {

template <class F>
int guard(F &&f) {
    try {
        return f();
    } catch (const Fail &e) {
        set_error(e.msg);
        return e.code;
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed");
        return BIPART_ERR_OOM;
    } catch (...) {
        set_error("unexpected exception");
        return BIPART_ERR_CUDA;
    }
}

}  // namespace

}  // namespace bp

using namespace bp;

extern "C" {

int bipart_set_allocator(bipart_alloc_fn alloc, bipart_free_fn free_fn, void *ctx) {
    if ((alloc == nullptr) != (free_fn == nullptr)) {
        set_error("alloc and free must both be set or both be NULL");
        return BIPART_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc = alloc;
    g_free = free_fn;
    g_alloc_ctx = ctx;
    return BIPART_OK;
}

const char *bipart_last_error(void) { return g_last_error.c_str(); }

int bipart_create(int32_t num_nodes, int32_t num_hedges, const int32_t *hedge_offsets,
                  const int32_t *hedge_pins, const int32_t *node_weights,
                  const int32_t *hedge_weights, void *stream, bipart_handle *out) {
    return guard([&]() {
        if (!out) throw Fail{BIPART_ERR_INVALID_ARG, "out is NULL"};
        *out = nullptr;
        const int32_t E = num_hedges, N = num_nodes;
        // what the copies depend on is checked here; the copied arrays are then checked on the
        // device by a kernel whose loops are bounded by N, E and P, and no other kernel reads
        // them before it has passed.  The host pass runs only when that check fails (it names
        // the first offending entry, as a sequential pass would) or when no device work is
        // possible (its CSR error outranks the device error).
        if (N < 0 || E < 0) throw Fail{BIPART_ERR_INVALID_ARG, "negative size"};
        if (E > 0 && !hedge_offsets) throw Fail{BIPART_ERR_INVALID_ARG, "hedge_offsets is NULL"};
        if (hedge_offsets && hedge_offsets[0] != 0) throw Fail{BIPART_ERR_INVALID_CSR, "hedge_offsets[0] != 0"};
        const int32_t P = E > 0 ? hedge_offsets[E] : 0;
        if (P < 0) throw Fail{BIPART_ERR_INVALID_CSR, "hedge_offsets[E] < 0"};
        if (P > 0 && !hedge_pins) throw Fail{BIPART_ERR_INVALID_ARG, "hedge_pins is NULL"};
        auto host_check = [&] { validate_host_csr(N, E, hedge_offsets, hedge_pins, node_weights, hedge_weights); };
        cudaStream_t s = (cudaStream_t)stream;
        std::unique_ptr<bipart_graph> g;
        Buf b_hoff, b_pins, b_nw, b_hw;
        int *d_hoff = nullptr, *d_pins = nullptr, *d_nw = nullptr, *d_hw = nullptr;
        DevCheck chk;
        try {
            g.reset(new_graph(s));
            d_hoff = (int *)b_hoff.ensure(sizeof(int) * ((size_t)E + 1), s);
            d_pins = (int *)b_pins.ensure(sizeof(int) * (size_t)std::max(P, 1), s);
            d_nw = node_weights ? (int *)b_nw.ensure(sizeof(int) * (size_t)std::max(N, 1), s) : nullptr;
            d_hw = hedge_weights ? (int *)b_hw.ensure(sizeof(int) * (size_t)std::max(E, 1), s) : nullptr;
            if (E > 0) BP_CUDA(cudaMemcpyAsync(d_hoff, hedge_offsets, sizeof(int) * ((size_t)E + 1), cudaMemcpyHostToDevice, s));
            if (P > 0) BP_CUDA(cudaMemcpyAsync(d_pins, hedge_pins, sizeof(int) * (size_t)P, cudaMemcpyHostToDevice, s));
            if (d_nw && N > 0) BP_CUDA(cudaMemcpyAsync(d_nw, node_weights, sizeof(int) * (size_t)N, cudaMemcpyHostToDevice, s));
            if (d_hw && E > 0) BP_CUDA(cudaMemcpyAsync(d_hw, hedge_weights, sizeof(int) * (size_t)E, cudaMemcpyHostToDevice, s));
            chk = device_check(g.get(), N, E, P, d_hoff, d_pins, d_nw, d_hw);
        } catch (...) {
            host_check();  // a CSR error outranks the device error
            throw;
        }
        if (chk.bad) {
            host_check();
            throw Fail{BIPART_ERR_INVALID_CSR, "malformed CSR (device check)"};
        }
        finish_create(g.get(), N, E, P, chk.node_weight, E > 0 ? d_hoff : nullptr, d_pins, d_nw, d_hw);
        *out = g.release();
        return BIPART_OK;
    });
}

int bipart_create_device(int32_t num_nodes, int32_t num_hedges, const int32_t *hedge_offsets,
                         const int32_t *hedge_pins, const int32_t *node_weights,
                         const int32_t *hedge_weights, void *stream, bipart_handle *out) {
    return guard([&]() {
        if (!out) throw Fail{BIPART_ERR_INVALID_ARG, "out is NULL"};
        *out = nullptr;
        if (num_nodes < 0 || num_hedges < 0) throw Fail{BIPART_ERR_INVALID_ARG, "negative size"};
        if (num_hedges > 0 && !hedge_offsets) throw Fail{BIPART_ERR_INVALID_ARG, "hedge_offsets is NULL"};
        cudaStream_t s = (cudaStream_t)stream;
        std::unique_ptr<bipart_graph> g(new_graph(s));
        const int32_t E = num_hedges, N = num_nodes;
        int32_t P = 0;
        if (E > 0) {
            BP_CUDA(cudaMemcpyAsync(g->w.host_small, hedge_offsets + E, sizeof(int), cudaMemcpyDeviceToHost, s));
            sync(g.get());
            P = (int32_t)g->w.host_small[0];
            if (P < 0) throw Fail{BIPART_ERR_INVALID_CSR, "hedge_offsets[E] < 0"};
            if (P > 0 && !hedge_pins) throw Fail{BIPART_ERR_INVALID_ARG, "hedge_pins is NULL"};
        }
        const DevCheck chk = device_check(g.get(), N, E, P, hedge_offsets, hedge_pins, node_weights, hedge_weights);
        if (chk.bad & 1) throw Fail{BIPART_ERR_INVALID_CSR, "hedge_offsets malformed"};
        if (chk.bad & 2) throw Fail{BIPART_ERR_INVALID_CSR, "pin out of range"};
        if (chk.bad & 4) throw Fail{BIPART_ERR_INVALID_CSR, "weight < 1"};
        if (chk.bad & 8) throw Fail{BIPART_ERR_INVALID_CSR, "weight sum must stay below 2^31"};
        finish_create(g.get(), N, E, P, chk.node_weight, hedge_offsets, hedge_pins, node_weights, hedge_weights);
        *out = g.release();
        return BIPART_OK;
    });
}

int bipart_set_stream(bipart_handle h, void *stream) {
    if (!h) { set_error("handle is NULL"); return BIPART_ERR_INVALID_ARG; }
    return guard([&]() {
        BP_CUDA(cudaStreamSynchronize(h->stream));
        h->stream = (cudaStream_t)stream;
        return BIPART_OK;
    });
}

namespace {

int partition_to_device(bipart_handle h, const Params &p, int32_t *d_out_parts) {
    if (!d_out_parts && h->L0.N > 0) throw Fail{BIPART_ERR_INVALID_ARG, "out_parts is NULL"};
    int st = partition_device(h, p, d_out_parts);
    check_status(h);
    return st;
}

int partition_to_host(bipart_handle h, const Params &p, int32_t *out_parts) {
    const int32_t N = h->L0.N;
    if (!out_parts && N > 0) throw Fail{BIPART_ERR_INVALID_ARG, "out_parts is NULL"};
    int *d = (int *)h->part_b.ensure(sizeof(int) * (size_t)std::max(N, 1), h->stream);
    int st = partition_device(h, p, d);
    if (N > 0) BP_CUDA(cudaMemcpyAsync(out_parts, d, sizeof(int) * (size_t)N, cudaMemcpyDeviceToHost, h->stream));
    sync(h);
    check_status(h);
    return st;
}

}  // namespace

int bipart_partition_device(bipart_handle h, int32_t k, double epsilon, int32_t policy,
                            int32_t levels, int32_t refine_iters, int32_t *d_out_parts) {
    if (!h) { set_error("handle is NULL"); return BIPART_ERR_INVALID_ARG; }
    HandleScope hs(h);
    return guard([&]() {
        return partition_to_device(h, make_params(k, epsilon, policy, levels, refine_iters, 0), d_out_parts);
    });
}

int bipart_partition(bipart_handle h, int32_t k, double epsilon, int32_t policy, int32_t levels,
                     int32_t refine_iters, int32_t *out_parts) {
    if (!h) { set_error("handle is NULL"); return BIPART_ERR_INVALID_ARG; }
    HandleScope hs(h);
    return guard([&]() {
        return partition_to_host(h, make_params(k, epsilon, policy, levels, refine_iters, 0), out_parts);
    });
}

int bipart_partition_ex(bipart_handle h, const bipart_params *params, int32_t *out_parts) {
    if (!h || !params) { set_error("NULL argument"); return BIPART_ERR_INVALID_ARG; }
    HandleScope hs(h);
    return guard([&]() {
        const bipart_params &q = *params;
        return partition_to_host(h, make_params(q.k, q.epsilon, q.policy, q.levels, q.refine_iters, q.flags),
                                 out_parts);
    });
}

int bipart_partition_device_ex(bipart_handle h, const bipart_params *params, int32_t *d_out_parts) {
    if (!h || !params) { set_error("NULL argument"); return BIPART_ERR_INVALID_ARG; }
    HandleScope hs(h);
    return guard([&]() {
        const bipart_params &q = *params;
        return partition_to_device(h, make_params(q.k, q.epsilon, q.policy, q.levels, q.refine_iters, q.flags),
                                   d_out_parts);
    });
}

int bipart_refine_kept(bipart_handle h, double epsilon, int32_t refine_iters, int32_t *out_parts) {
    if (!h || (!out_parts && h->L0.N > 0)) { set_error("NULL argument"); return BIPART_ERR_INVALID_ARG; }
    HandleScope hs(h);
    return guard([&]() {
        if (!h->hier.valid) throw Fail{BIPART_ERR_INVALID_ARG, "no k = 2 hierarchy kept (partition with k = 2 first)"};
        const Params &q = h->hier.params;
        const Params p = make_params(2, epsilon, q.policy, q.levels, refine_iters, q.flags);
        const int32_t N = h->L0.N;
        int *d = (int *)h->part_b.ensure(sizeof(int) * (size_t)std::max(N, 1), h->stream);
        const int st = refine_kept(h, p.e6, p.iters, d);
        if (N > 0) BP_CUDA(cudaMemcpyAsync(out_parts, d, sizeof(int) * (size_t)N, cudaMemcpyDeviceToHost, h->stream));
        sync(h);
        return st;
    });
}

int bipart_plan_active(bipart_handle h, int32_t *active) {
    if (!h || !active) { set_error("NULL argument"); return BIPART_ERR_INVALID_ARG; }
    *active = h->last_replayed ? 1 : 0;
    return BIPART_OK;
}

int bipart_num_levels(bipart_handle h, int32_t *num_levels) {
    if (!h || !num_levels) { set_error("NULL argument"); return BIPART_ERR_INVALID_ARG; }
    if (!h->hier.valid) { set_error("no k = 2 hierarchy kept"); return BIPART_ERR_INVALID_ARG; }
    *num_levels = h->hier.nlev;
    return BIPART_OK;
}

__global__ void k_fill_i32(int n, int val, int *a) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = val;
}

int bipart_get_level(bipart_handle h, int32_t level, int32_t *N, int32_t *E, int32_t *P,
                     int32_t *hoff, int32_t *pins, int32_t *node_weights, int32_t *hedge_weights,
                     int32_t *cmap, int32_t *match) {
    if (!h) { set_error("handle is NULL"); return BIPART_ERR_INVALID_ARG; }
    return guard([&]() {
        int nlev = h->hier.valid ? h->hier.nlev : 1;
        if (level < 0 || level >= nlev) throw Fail{BIPART_ERR_INVALID_ARG, "level out of range"};
        Level &L = level == 0 ? h->L0 : *h->lev[level - 1];
        cudaStream_t s = h->stream;
        if (N) *N = L.N;
        if (E) *E = L.E;
        if (P) *P = L.P;
        if (hoff) BP_CUDA(cudaMemcpyAsync(hoff, L.hoff(), sizeof(int) * ((size_t)L.E + 1), cudaMemcpyDeviceToHost, s));
        if (pins && L.P > 0) BP_CUDA(cudaMemcpyAsync(pins, L.pins(), sizeof(int) * (size_t)L.P, cudaMemcpyDeviceToHost, s));
        if (node_weights && L.N > 0) BP_CUDA(cudaMemcpyAsync(node_weights, L.nw(), sizeof(int) * (size_t)L.N, cudaMemcpyDeviceToHost, s));
        bool coarsest = level == nlev - 1;
        if (cmap && L.N > 0) {
            if (coarsest) std::fill(cmap, cmap + L.N, -1);
            else BP_CUDA(cudaMemcpyAsync(cmap, L.cmap(), sizeof(int) * (size_t)L.N, cudaMemcpyDeviceToHost, s));
        }
        if (match && L.N > 0) {
            if (coarsest) std::fill(match, match + L.N, -1);
            else BP_CUDA(cudaMemcpyAsync(match, L.match(), sizeof(int) * (size_t)L.N, cudaMemcpyDeviceToHost, s));
        }
        if (hedge_weights && L.E > 0) {
            if (L.unit_hw) std::fill(hedge_weights, hedge_weights + L.E, 1);
            else BP_CUDA(cudaMemcpyAsync(hedge_weights, L.hw(), sizeof(int) * (size_t)L.E, cudaMemcpyDeviceToHost, s));
        }
        sync(h);
        return BIPART_OK;
    });
}

int bipart_sizes(bipart_handle h, int32_t *N, int32_t *E, int32_t *P) {
    if (!h) { set_error("handle is NULL"); return BIPART_ERR_INVALID_ARG; }
    if (N) *N = h->L0.N;
    if (E) *E = h->L0.E;
    if (P) *P = h->L0.P;
    return BIPART_OK;
}

void bipart_destroy(bipart_handle h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    bool ext = h->ext_alloc;
    for (const auto &k : h->kids) ext |= k->ext_alloc;
    // A handle whose buffers all came from the library's own allocator is released by a
    // background thread (its work has finished: freeing ~150 buffers costs the caller ~0.3 ms);
    // one that used an allocator hook is released here, where that hook expects to be called.
    if (!ext && release_later(h)) return;
    delete h;
}

}  // extern "C"

// Cut evaluation reuses the sorted-unique kernels: lambda_e = number of distinct parts of e.
namespace bp {
void distinct_counts(bipart_graph *g, Level &L, const int *d_map, int *cnt);
}

__global__ void k_cut_sum(int E, const int *__restrict__ cnt, const int *__restrict__ hw,
                          unsigned long long *out) {
    unsigned long long s = 0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x)
        s += (unsigned long long)(hw ? hw[e] : 1) * (unsigned long long)(cnt[e] - 1);
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

extern "C" int bipart_cut(bipart_handle h, const int32_t *parts, int64_t *cut) {
    if (!h || !cut || (!parts && h->L0.N > 0)) { set_error("NULL argument"); return BIPART_ERR_INVALID_ARG; }
    HandleScope hs(h);
    return guard([&]() {
        Level &L = h->L0;
        cudaStream_t s = h->stream;
        *cut = 0;
        if (L.E == 0) return BIPART_OK;
        int *d = (int *)h->part_b.ensure(sizeof(int) * (size_t)std::max(L.N, 1), s);
        BP_CUDA(cudaMemcpyAsync(d, parts, sizeof(int) * (size_t)L.N, cudaMemcpyHostToDevice, s));
        int *cnt = (int *)h->w.e_a.ensure(sizeof(int) * (size_t)L.E, s);
        distinct_counts(h, L, d, cnt);
        unsigned long long *acc = reinterpret_cast<unsigned long long *>(h->w.small.as<char>() + 48 * 1024 + 128);
        BP_CUDA(cudaMemsetAsync(acc, 0, sizeof(unsigned long long), s));
        k_cut_sum<<<grid_for(L.E), kBlock, 0, s>>>(L.E, cnt, L.hw(), acc);
        BP_LAUNCH();
        unsigned long long r = 0;
        BP_CUDA(cudaMemcpyAsync(h->w.host_small, acc, sizeof(r), cudaMemcpyDeviceToHost, s));
        sync(h);
        std::memcpy(&r, h->w.host_small, sizeof(r));
        *cut = (int64_t)r;
        return BIPART_OK;
    });
}

// ------------------------------------------------------------------------- diagnostics
#include <atomic>
#include <map>
#include <mutex>

namespace bp {
namespace {
std::atomic<long long> g_launches{0};
struct ProfRec {
    std::string name;
    double bytes;
    cudaEvent_t a, b;
    cudaStream_t s;
};
struct ProfTot {
    long long launches = 0;
    double ms = 0, bytes = 0;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
bool g_prof_levels = false;  // totals keyed by kernel and level (profile mode 2)
int g_prof_epoch = 0;
std::string g_prof_only;
std::vector<ProfRec> g_prof_pending;
std::vector<cudaEvent_t> g_prof_pool;
std::map<std::string, ProfTot> g_prof_tot;

cudaEvent_t prof_event() {
    if (!g_prof_pool.empty()) {
        cudaEvent_t e = g_prof_pool.back();
        g_prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void prof_drain() {
    for (ProfRec &r : g_prof_pending) {
        float ms = 0;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            ProfTot &t = g_prof_tot[r.name];
            t.launches++;
            t.ms += ms;
            t.bytes += r.bytes;
        }
        g_prof_pool.push_back(r.a);
        g_prof_pool.push_back(r.b);
    }
    g_prof_pending.clear();
}
}  // namespace

void note_launch() {
    if (tl_capturing) return;  // captured launches run when the graph is launched
    g_launches.fetch_add(1, std::memory_order_relaxed);
}

int prof_epoch() { return g_prof_epoch; }

void prof_collect(const std::vector<Probe> &probes) {
    if (probes.empty()) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (const Probe &p : probes) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            ProfTot &t = g_prof_tot[p.name];
            t.launches++;
            t.ms += ms;
            t.bytes += p.bytes;
        }
    }
    cudaGetLastError();
}

thread_local char tl_prof_phase = 0;
thread_local int tl_prof_level = 0;

void prof_level(char phase, int level) {
    tl_prof_phase = phase;
    tl_prof_level = level;
}

ProfScope::ProfScope(const char *name_in, double bytes, cudaStream_t s) {
    if (!g_prof_on) return;
    if (!g_prof_only.empty() && g_prof_only != name_in) return;
    std::string tagged;
    if (g_prof_levels && tl_prof_phase) {
        tagged = std::string(name_in) + "@" + tl_prof_phase + std::to_string(tl_prof_level);
    }
    const char *name = tagged.empty() ? name_in : tagged.c_str();
    if (tl_capturing) {
        // inside a captured plan: event record nodes (external records: a plain record during
        // capture only orders work inside the graph), read back after every replay
        bipart_graph *g = tl_graph;
        if (!g) return;
        Probe p{name, bytes, nullptr, nullptr};
        cudaEventCreate(&p.a);
        cudaEventCreate(&p.b);
        cudaEventRecordWithFlags(p.a, s, cudaEventRecordExternal);
        g->plan.probes.push_back(p);
        slot = -2 - (int)(g->plan.probes.size() - 1);
        return;
    }
    std::lock_guard<std::mutex> lk(g_prof_mu);
    // finished records are drained here, never between a scope's end() and its set_bytes()
    if (g_prof_pending.size() > 4096) prof_drain();
    ProfRec r{name, bytes, prof_event(), prof_event(), s};
    cudaEventRecord(r.a, s);
    g_prof_pending.push_back(r);
    slot = (int)g_prof_pending.size() - 1;
}

void ProfScope::set_bytes(double bytes) {
    if (slot <= -2) {
        bipart_graph *g = tl_graph;
        size_t i = (size_t)(-2 - slot);
        if (g && i < g->plan.probes.size()) g->plan.probes[i].bytes = bytes;
        return;
    }
    if (slot < 0) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (slot < (int)g_prof_pending.size()) g_prof_pending[slot].bytes = bytes;
}

void ProfScope::end() {
    if (ended) return;
    ended = true;
    if (slot <= -2) {
        bipart_graph *g = tl_graph;
        size_t i = (size_t)(-2 - slot);
        if (g && i < g->plan.probes.size())
            cudaEventRecordWithFlags(g->plan.probes[i].b, g->stream, cudaEventRecordExternal);
        return;
    }
    if (slot < 0) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (slot < (int)g_prof_pending.size()) cudaEventRecord(g_prof_pending[slot].b, g_prof_pending[slot].s);
}
}  // namespace bp

extern "C" int64_t bipart_kernel_launches(void) { return (int64_t)bp::g_launches.load(); }

extern "C" int bipart_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(bp::g_prof_mu);
    bp::prof_drain();
    bp::g_prof_tot.clear();
    if (bp::g_prof_on != (on != 0) || bp::g_prof_levels != (on == 2))
        bp::g_prof_epoch++;  // plans are recaptured with/without probes
    bp::g_prof_on = on != 0;
    bp::g_prof_levels = on == 2;
    return BIPART_OK;
}

extern "C" int bipart_profile_select(const char *kernel_name) {
    std::lock_guard<std::mutex> lk(bp::g_prof_mu);
    bp::prof_drain();
    bp::g_prof_tot.clear();
    std::string only = kernel_name ? kernel_name : "";
    if (only != bp::g_prof_only) bp::g_prof_epoch++;
    bp::g_prof_only = only;
    return BIPART_OK;
}

extern "C" int bipart_profile_read(int32_t idx, char *name, size_t name_len, int64_t *launches,
                                   double *total_ms, double *total_bytes) {
    std::lock_guard<std::mutex> lk(bp::g_prof_mu);
    bp::prof_drain();
    int n = (int)bp::g_prof_tot.size();
    if (idx < 0) return n;
    if (idx >= n) { bp::set_error("profile index out of range"); return BIPART_ERR_INVALID_ARG; }
    auto it = bp::g_prof_tot.begin();
    std::advance(it, idx);
    if (name && name_len) {
        std::strncpy(name, it->first.c_str(), name_len - 1);
        name[name_len - 1] = 0;
    }
    if (launches) *launches = it->second.launches;
    if (total_ms) *total_ms = it->second.ms;
    if (total_bytes) *total_bytes = it->second.bytes;
    return n;
}
