// Batched partitioning in persistent launches: every thread block takes whole instances from a
// queue (largest first) and runs the complete partition of an instance on its own -- level-0
// normalisation, coarsening (Algorithms 1-2), the initial partition (Algorithm 3), refinement
// and rebalancing (Algorithms 4-5), and for k > 2 the nested bisections of Algorithm 6 with net
// splitting -- with the phases separated by __syncthreads() instead of kernel boundaries.  The
// phase code is the device code the grid kernels run (coarsen_dev.cuh, refine_dev.cuh)
// instantiated for a one-block team, so an instance's result is identical to the single-instance
// path.
//
// Instances go into size buckets by pin count; each bucket runs as its own persistent launch with
// the block shape (threads, blocks per SM) its tuning chose, and the launches of all buckets,
// with the copies out, form one CUDA graph whose branches run at the same time (a bucket that
// runs out of instances frees its SMs for the others); the inputs go in ahead of it, each chunk
// as soon as the host has staged it.  The graph is kept and replayed while
// the batches keep the same shape.  The tuner times every candidate shape on each bucket of a
// given batch and keeps the winners in a JSON file per device.
//
// Each block owns an arena in HBM (sized by the host for the largest instance of its bucket) from
// which it carves the level store and scratch of its current instance with a bump pointer.  An
// instance whose hierarchy does not fit is marked deferred and the host runs it through the
// single-instance path instead.
#include <cuda_runtime.h>
#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "block_dev.cuh"

namespace bp {

// The kernel of each block shape (block_shapes_*.cu).
const void *batch_kernel_256_1();
const void *batch_kernel_256_2();
const void *batch_kernel_256_4();
const void *batch_kernel_512_1();
const void *batch_kernel_512_2();
const void *batch_kernel_1024_1();

// ------------------------------------------------------------------ host side
namespace {

// Candidate block shapes (threads, blocks per SM asked of the compiler's register budget).  The
// selection of Algorithms 3 and 5 needs at least 256 threads.
struct Shape {
    int threads, per_sm;
    const void *(*fn)();
};
const Shape kShapes[] = {
    {256, 1, batch_kernel_256_1}, {256, 2, batch_kernel_256_2}, {256, 4, batch_kernel_256_4},
    {512, 1, batch_kernel_512_1}, {512, 2, batch_kernel_512_2}, {1024, 1, batch_kernel_1024_1},
};
constexpr int kNumShapes = (int)(sizeof(kShapes) / sizeof(kShapes[0]));

// Size buckets by pin count: [0, 16K), [16K, 128K), [128K, 1M), [1M, ...).
constexpr int kBuckets = 4;
const int64_t kBucketEdge[kBuckets - 1] = {16 << 10, 128 << 10, 1 << 20};
// Shapes used before a bucket is tuned on this device.
const int kDefaultShape[kBuckets] = {1, 5, 5, 5};

int bucket_of(int64_t P) {
    int b = 0;
    while (b < kBuckets - 1 && P >= kBucketEdge[b]) ++b;
    return b;
}

// Upper bound of the arena bytes an instance may need (level store over all levels, scratch and,
// for k > 2, the part vector, node maps and one subgraph's level store); instances above the
// arena given to their bucket are deferred by the device.
size_t arena_estimate(int64_t N, int64_t E, int64_t P, int k) {
    const int64_t level0 = 4 * (E + 1) + 4 * E + 4 * P + 4 * N + 4 * (N + 1) + 4 * P + 8 * N + P / 32 + 16;
    const int64_t scratch = E * (4 * 4 + 8) + N * (4 * 3 + 8 + 4 + 4 + 3) + 4 * P + 64 * 1024;
    const int64_t kway = k > 2 ? 16 * N + level0 : 0;
    return (size_t)(scratch + 5 * level0 + kway + (4 << 20));
}

// ---------------------------------------------------------------- tuning table (JSON cache)
// {"version": 1, "devices": {"<name> / <SMs> SMs": {"<bucket>": [threads, per_sm], ...}, ...}}
// A minimal reader for exactly this layout (objects, arrays, strings, integers).
struct JVal {
    enum Kind { NUL, NUM, STR, ARR, OBJ } kind = NUL;
    long long num = 0;
    std::string str;
    std::vector<JVal> arr;
    std::vector<std::pair<std::string, JVal>> obj;
};

struct JParse {
    const char *p, *end;
    bool ok = true;
    void ws() {
        while (p < end && (*p == ' ' || *p == '\n' || *p == '\r' || *p == '\t')) ++p;
    }
    bool lit(char c) {
        ws();
        if (p < end && *p == c) {
            ++p;
            return true;
        }
        return false;
    }
    std::string string() {
        std::string s;
        if (!lit('"')) {
            ok = false;
            return s;
        }
        while (p < end && *p != '"') {
            if (*p == '\\' && p + 1 < end) ++p;
            s.push_back(*p++);
        }
        if (p < end) ++p;
        else ok = false;
        return s;
    }
    JVal value(int depth = 0) {
        JVal v;
        ws();
        if (!ok || p >= end || depth > 8) {
            ok = false;
            return v;
        }
        if (*p == '{') {
            ++p;
            v.kind = JVal::OBJ;
            if (lit('}')) return v;
            do {
                std::string k = string();
                if (!lit(':')) ok = false;
                if (!ok) return v;
                v.obj.emplace_back(k, value(depth + 1));
            } while (ok && lit(','));
            if (!lit('}')) ok = false;
        } else if (*p == '[') {
            ++p;
            v.kind = JVal::ARR;
            if (lit(']')) return v;
            do v.arr.push_back(value(depth + 1));
            while (ok && lit(','));
            if (!lit(']')) ok = false;
        } else if (*p == '"') {
            v.kind = JVal::STR;
            v.str = string();
        } else {
            char *q = nullptr;
            v.num = std::strtoll(p, &q, 10);
            if (q == p) ok = false;
            else {
                v.kind = JVal::NUM;
                p = q;
            }
        }
        return v;
    }
};

std::string tune_path() {
    if (const char *e = std::getenv("BIPART_TUNE_CACHE")) return e;
    std::string dir;
    if (const char *x = std::getenv("XDG_CACHE_HOME")) dir = x;
    else if (const char *h = std::getenv("HOME")) dir = std::string(h) + "/.cache";
    else dir = "/tmp";
    return dir + "/bipart/batch_tune.json";
}

void mkdirs_for(const std::string &path) {
    for (size_t i = 1; i < path.size(); ++i)
        if (path[i] == '/') ::mkdir(path.substr(0, i).c_str(), 0755);
}

// device key -> bucket -> shape index
using TuneTable = std::map<std::string, std::map<int, int>>;

TuneTable read_table(const std::string &path) {
    TuneTable t;
    FILE *f = std::fopen(path.c_str(), "rb");
    if (!f) return t;
    std::string text;
    char buf[4096];
    size_t r;
    while ((r = std::fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, r);
    std::fclose(f);
    JParse jp{text.data(), text.data() + text.size()};
    JVal root = jp.value();
    if (!jp.ok || root.kind != JVal::OBJ) return t;
    for (auto &kv : root.obj) {
        if (kv.first != "devices" || kv.second.kind != JVal::OBJ) continue;
        for (auto &dev : kv.second.obj) {
            if (dev.second.kind != JVal::OBJ) continue;
            for (auto &b : dev.second.obj) {
                const int bucket = std::atoi(b.first.c_str());
                if (bucket < 0 || bucket >= kBuckets || b.second.kind != JVal::ARR || b.second.arr.size() != 2) continue;
                for (int s = 0; s < kNumShapes; ++s)
                    if (kShapes[s].threads == b.second.arr[0].num && kShapes[s].per_sm == b.second.arr[1].num)
                        t[dev.first][bucket] = s;
            }
        }
    }
    return t;
}

void write_table(const std::string &path, const TuneTable &t) {
    mkdirs_for(path);
    const std::string tmp = path + ".tmp" + std::to_string((long long)::getpid());
    FILE *f = std::fopen(tmp.c_str(), "wb");
    if (!f) return;  // a cache that cannot be written only costs a re-tune
    std::fprintf(f, "{\"version\": 1, \"devices\": {");
    bool first_dev = true;
    for (auto &dev : t) {
        std::string name;
        for (char c : dev.first) name += (c == '"' || c == '\\') ? '_' : c;
        std::fprintf(f, "%s\n  \"%s\": {", first_dev ? "" : ",", name.c_str());
        bool first = true;
        for (auto &b : dev.second) {
            std::fprintf(f, "%s\"%d\": [%d, %d]", first ? "" : ", ", b.first, kShapes[b.second].threads,
                         kShapes[b.second].per_sm);
            first = false;
        }
        std::fprintf(f, "}");
        first_dev = false;
    }
    std::fprintf(f, "\n}}\n");
    std::fclose(f);
    std::rename(tmp.c_str(), path.c_str());
}

// ---------------------------------------------------------------- the batch context
// Pinned host memory that only grows.
struct Pinned {
    void *p = nullptr;
    size_t cap = 0;
    void *ensure(size_t bytes) {
        if (bytes == 0) bytes = 16;
        if (bytes > cap) {
            if (p) cudaFreeHost(p);
            p = nullptr;
            cap = 0;
            const size_t c = bytes + bytes / 8 + 4096;
            if (cudaHostAlloc(&p, c, cudaHostAllocDefault) != cudaSuccess) {
                cudaGetLastError();
                p = nullptr;
                throw Fail{BIPART_ERR_OOM, "pinned host allocation of " + std::to_string(c) + " bytes failed"};
            }
            cap = c;
        }
        return p;
    }
    void release() {
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
    }
};

// Byte offsets of the batch's arrays in the staging buffers (host and device alike).
struct Layout {
    size_t inst, order, hoff, pins, nw, hw, in_end;  // inputs
    size_t parts, out_end;                           // outputs (after the inputs)
};

struct BucketRun {
    int shape = 0, blocks = 0, count = 0, first = 0;  // instances order[first, first + count)
    size_t arena = 0, arena_off = 0;
};

struct BatchCtx {
    std::mutex mu;
    int device = -1, sms = 0;
    std::string dev_key;
    cudaStream_t stream = nullptr;
    cudaStream_t branch[kBuckets] = {};
    cudaEvent_t fork = nullptr, join[kBuckets] = {};
    Pinned host;                 // inputs then outputs
    Buf dev, arena, misc;
    std::unique_ptr<Lanes> lanes;
    bool attrs = false;
    int occ[kNumShapes] = {};
    // the table: loaded once, updated by the tuner
    bool table_loaded = false;
    TuneTable table;
    // the last graph and the batch shape it was captured for
    cudaGraphExec_t exec = nullptr;
    std::vector<long long> key;

    void init() {
        int dev_now = 0;
        BP_CUDA(cudaGetDevice(&dev_now));
        if (device == dev_now) return;
        if (device >= 0) throw Fail{BIPART_ERR_INVALID_ARG, "the batch path serves one device per process"};
        device = dev_now;
        BP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
        cudaDeviceProp prop;
        BP_CUDA(cudaGetDeviceProperties(&prop, device));
        dev_key = std::string(prop.name) + " / " + std::to_string(sms) + " SMs";
        BP_CUDA(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
        BP_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        for (int b = 0; b < kBuckets; ++b) {
            BP_CUDA(cudaStreamCreateWithFlags(&branch[b], cudaStreamNonBlocking));
            BP_CUDA(cudaEventCreateWithFlags(&join[b], cudaEventDisableTiming));
        }
        for (int s = 0; s < kNumShapes; ++s) {
            BP_CUDA(cudaFuncSetAttribute(kShapes[s].fn(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes));
            int per = 0;
            BP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kShapes[s].fn(), kShapes[s].threads, kSmemBytes));
            occ[s] = std::max(1, std::min(per, kShapes[s].per_sm));
        }
        lanes.reset(new Lanes(16));
    }
    int shape_for(int bucket) {
        if (!table_loaded) {
            table = read_table(tune_path());
            table_loaded = true;
        }
        auto it = table.find(dev_key);
        if (it != table.end()) {
            auto jt = it->second.find(bucket);
            if (jt != it->second.end()) return jt->second;
        }
        return kDefaultShape[bucket];
    }
    void drop_graph() {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        key.clear();
    }
};

BatchCtx &ctx() {
    static BatchCtx *c = new BatchCtx;  // never destroyed: process exit tears the context down
    return *c;
}

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

// Everything a batch call prepares on the host before the device work.
struct Prepared {
    std::vector<int> order;  // instances by bucket, largest first within a bucket
    BucketRun run[kBuckets];
    Layout lay;
    size_t arena_total = 0;
    std::vector<long long> key;
};

Prepared prepare(BatchCtx &c, std::vector<BInst> &inst, const std::vector<const int32_t *> &nw,
                 const std::vector<const int32_t *> &hw, const int *force_shape) {
    const int n = (int)inst.size();
    Prepared pr;
    int64_t sh = 0, sp = 0, sn = 0, sw = 0, so = 0;
    for (int i = 0; i < n; ++i) {
        BInst &I = inst[i];
        I.hoff = sh;
        I.pins = sp;
        I.nw = nw[i] ? sn : -1;
        I.hw = hw[i] ? sw : -1;
        I.out = so;
        I.status = 0;
        sh += I.E + 1;
        sp += I.P;
        if (nw[i]) sn += I.N;
        if (hw[i]) sw += I.E;
        so += I.N;
    }
    std::vector<std::vector<int>> by(kBuckets);
    for (int i = 0; i < n; ++i) by[bucket_of(inst[i].P)].push_back(i);
    // optional override (tests of the deferral path): arena bytes per block in MiB
    size_t arena_cap = 0;
    if (const char *env = std::getenv("BIPART_BLOCK_ARENA_MB")) {
        long long mb = std::atoll(env);
        if (mb > 0) arena_cap = (size_t)mb << 20;
    }
    for (int b = kBuckets - 1; b >= 0; --b) {
        std::vector<int> &v = by[b];
        std::stable_sort(v.begin(), v.end(), [&](int x, int y) { return inst[x].P > inst[y].P; });
        BucketRun &r = pr.run[b];
        r.first = (int)pr.order.size();
        r.count = (int)v.size();
        pr.order.insert(pr.order.end(), v.begin(), v.end());
        if (v.empty()) continue;
        r.shape = force_shape ? force_shape[b] : c.shape_for(b);
        r.blocks = std::min(r.count, c.sms * c.occ[r.shape]);
        size_t a = 0;
        for (int i : v) a = std::max(a, arena_estimate(inst[i].N, inst[i].E, inst[i].P, inst[i].k));
        if (arena_cap) a = std::min(a, arena_cap);
        r.arena = al256(a);
        r.arena_off = pr.arena_total;
        pr.arena_total += r.arena * (size_t)r.blocks;
    }
    Layout &L = pr.lay;
    L.inst = 0;
    L.order = al256(L.inst + sizeof(BInst) * (size_t)n);
    L.hoff = al256(L.order + sizeof(int) * (size_t)n);
    L.pins = al256(L.hoff + sizeof(int) * (size_t)sh);
    L.nw = al256(L.pins + sizeof(int) * (size_t)sp);
    L.hw = al256(L.nw + sizeof(int) * (size_t)sn);
    L.in_end = al256(L.hw + sizeof(int) * (size_t)sw);
    L.parts = L.in_end;
    L.out_end = al256(L.parts + sizeof(int) * (size_t)so);
    // the graph depends on the sizes, the parameters, the bucket shapes and the buffers
    std::vector<long long> &k = pr.key;
    k.reserve((size_t)n * 9 + 4 * kBuckets + 4);
    k.push_back(n);
    for (const BInst &I : inst) {
        k.push_back(I.N);
        k.push_back(I.E);
        k.push_back(I.P);
        k.push_back(I.k);
        k.push_back(I.policy);
        k.push_back(I.levels);
        k.push_back(I.iters);
        k.push_back(I.e6);
        k.push_back((I.nw >= 0) | ((I.hw >= 0) << 1));
    }
    for (int b = 0; b < kBuckets; ++b) {
        k.push_back(pr.run[b].shape);
        k.push_back(pr.run[b].blocks);
        k.push_back((long long)pr.run[b].arena);
    }
    return pr;
}

// Copies the batch's inputs into the pinned staging buffer on the context's host threads and moves
// them to the device on c.stream: the pieces are staged in chunks of destination offsets, and each
// chunk's copy to the device is queued as soon as the chunk is staged, so the copies run while the
// host stages the next chunks.
void stage_inputs(BatchCtx &c, const Prepared &pr, const std::vector<BInst> &inst,
                  const std::vector<const int32_t *> &hoff, const std::vector<const int32_t *> &pins,
                  const std::vector<const int32_t *> &nw, const std::vector<const int32_t *> &hw) {
    char *h = (char *)c.host.p, *d = (char *)c.dev.p;
    const Layout &L = pr.lay;
    std::memcpy(h + L.inst, inst.data(), sizeof(BInst) * inst.size());
    std::memcpy(h + L.order, pr.order.data(), sizeof(int) * pr.order.size());
    struct Piece {
        size_t off;
        const void *src;
        size_t bytes;
    };
    std::vector<Piece> pieces;
    const size_t kPiece = 4 << 20;
    auto add = [&](size_t off, const int32_t *src, int64_t count) {
        const size_t bytes = sizeof(int32_t) * (size_t)count;
        for (size_t o = 0; o < bytes; o += kPiece) pieces.push_back({off + o, (const char *)src + o, std::min(kPiece, bytes - o)});
    };
    for (size_t i = 0; i < inst.size(); ++i) {
        const BInst &I = inst[i];
        add(L.hoff + sizeof(int) * (size_t)I.hoff, hoff[i], I.E + 1);
        if (I.P > 0) add(L.pins + sizeof(int) * (size_t)I.pins, pins[i], I.P);
        if (I.nw >= 0) add(L.nw + sizeof(int) * (size_t)I.nw, nw[i], I.N);
        if (I.hw >= 0 && I.E > 0) add(L.hw + sizeof(int) * (size_t)I.hw, hw[i], I.E);
    }
    std::sort(pieces.begin(), pieces.end(), [](const Piece &a, const Piece &b) { return a.off < b.off; });
    const size_t kChunk = 256 << 20;
    size_t up = 0;  // [0, up) is queued for the device
    for (size_t j = 0; j < pieces.size();) {
        size_t j1 = j;
        while (j1 < pieces.size() && pieces[j1].off < pieces[j].off + kChunk) ++j1;
        const int tasks = (int)std::min<size_t>(j1 - j, 64);
        c.lanes->run(tasks, [&](int t) {
            for (size_t q = j + (size_t)t; q < j1; q += (size_t)tasks)
                std::memcpy(h + pieces[q].off, pieces[q].src, pieces[q].bytes);
        });
        const size_t hi = j1 < pieces.size() ? pieces[j1].off : L.in_end;
        BP_CUDA(cudaMemcpyAsync(d + up, h + up, hi - up, cudaMemcpyHostToDevice, c.stream));
        up = hi;
        j = j1;
    }
    if (up < L.in_end) BP_CUDA(cudaMemcpyAsync(d + up, h + up, L.in_end - up, cudaMemcpyHostToDevice, c.stream));
}

// Records the batch's device work on c.stream (after the inputs stage_inputs queued): one
// persistent launch per bucket on its own branch, outputs back.  Run eagerly or under capture.
void record(BatchCtx &c, const Prepared &pr, int n) {
    char *h = (char *)c.host.p, *d = (char *)c.dev.p;
    const Layout &L = pr.lay;
    cudaStream_t s = c.stream;
    int *heads = c.misc.as<int>();
    uint32_t *status = reinterpret_cast<uint32_t *>(heads + 16);
    BP_CUDA(cudaMemsetAsync(heads, 0, 256, s));
    BP_CUDA(cudaEventRecord(c.fork, s));
    for (int b = kBuckets - 1; b >= 0; --b) {
        const BucketRun &r = pr.run[b];
        if (r.count == 0) continue;
        cudaStream_t bs = c.branch[b];
        BP_CUDA(cudaStreamWaitEvent(bs, c.fork, 0));
        BArgs a;
        a.inst = reinterpret_cast<BInst *>(d + L.inst);
        a.order = reinterpret_cast<const int *>(d + L.order) + r.first;
        a.n = r.count;
        a.next = heads + b;
        a.hoff = reinterpret_cast<const int *>(d + L.hoff);
        a.pins = reinterpret_cast<const int *>(d + L.pins);
        a.nw = reinterpret_cast<const int *>(d + L.nw);
        a.hw = reinterpret_cast<const int *>(d + L.hw);
        a.parts = reinterpret_cast<int *>(d + L.parts);
        a.arena = c.arena.as<char>() + r.arena_off;
        a.arena_bytes = r.arena;
        a.status = status;
        void *args[] = {&a};
        BP_CUDA(cudaLaunchKernel(kShapes[r.shape].fn(), dim3(r.blocks), dim3(kShapes[r.shape].threads), args,
                                 kSmemBytes, bs));
        BP_LAUNCH();
        BP_CUDA(cudaEventRecord(c.join[b], bs));
        BP_CUDA(cudaStreamWaitEvent(s, c.join[b], 0));
    }
    BP_CUDA(cudaMemcpyAsync(h + L.inst, d + L.inst, sizeof(BInst) * (size_t)n, cudaMemcpyDeviceToHost, s));
    BP_CUDA(cudaMemcpyAsync(h + L.parts, d + L.parts, L.out_end - L.parts, cudaMemcpyDeviceToHost, s));
    BP_CUDA(cudaMemcpyAsync(h + L.out_end, status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
}

// Ensures the context's buffers for a prepared batch (dropping the graph when one moves).
void ensure_buffers(BatchCtx &c, const Prepared &pr) {
    const void *h0 = c.host.p, *d0 = c.dev.p, *a0 = c.arena.p, *m0 = c.misc.p;
    c.host.ensure(pr.lay.out_end + 256);
    c.dev.ensure(pr.lay.out_end, c.stream);
    c.arena.ensure(std::max<size_t>(pr.arena_total, 256), c.stream);
    c.misc.ensure(256, c.stream);
    if (c.host.p != h0 || c.dev.p != d0 || c.arena.p != a0 || c.misc.p != m0) c.drop_graph();
}

// Runs a prepared and staged batch (graph replay when the shape repeats); returns kernel ms when
// timed.
float launch(BatchCtx &c, const Prepared &pr, int n, bool use_graph, bool timed) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (timed) {
        BP_CUDA(cudaEventCreate(&e0));
        BP_CUDA(cudaEventCreate(&e1));
        BP_CUDA(cudaEventRecord(e0, c.stream));
    }
    if (use_graph) {
        if (!c.exec || c.key != pr.key) {
            c.drop_graph();
            cudaGraph_t g = nullptr;
            BP_CUDA(cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal));
            try {
                record(c, pr, n);
            } catch (...) {
                cudaStreamEndCapture(c.stream, &g);
                if (g) cudaGraphDestroy(g);
                cudaGetLastError();
                throw;
            }
            BP_CUDA(cudaStreamEndCapture(c.stream, &g));
            const cudaError_t e = cudaGraphInstantiate(&c.exec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                c.exec = nullptr;
                BP_CUDA(e);
            }
            c.key = pr.key;
        }
        BP_CUDA(cudaGraphLaunch(c.exec, c.stream));
    } else {
        record(c, pr, n);
    }
    float ms = 0.f;
    if (timed) BP_CUDA(cudaEventRecord(e1, c.stream));
    BP_CUDA(cudaStreamSynchronize(c.stream));
    if (timed) {
        cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    uint32_t dst = 0;
    std::memcpy(&dst, (char *)c.host.p + pr.lay.out_end, sizeof(dst));
    if (dst & DEV_TIMEOUT) throw Fail{BIPART_ERR_TIMEOUT, "a bounded device loop expired in the batch kernel"};
    return ms;
}

}  // namespace

bool block_eligible(int64_t N, int64_t E, int64_t P, int k, int levels) {
    (void)E;
    return k >= 1 && k <= kBlockMaxK && levels < kMaxLev && N <= (1 << 18) && P <= (1 << 24);
}

void run_block_batch(std::vector<BInst> &inst, const std::vector<const int32_t *> &hoff,
                     const std::vector<const int32_t *> &pins, const std::vector<const int32_t *> &nw,
                     const std::vector<const int32_t *> &hw, const std::vector<int32_t *> &outs) {
    const int n = (int)inst.size();
    if (n == 0) return;
    BatchCtx &c = ctx();
    std::lock_guard<std::mutex> lk(c.mu);
    c.init();
    const bool timing = std::getenv("BIPART_TIMING") != nullptr;
    auto t0 = std::chrono::steady_clock::now();
    Prepared pr = prepare(c, inst, nw, hw, nullptr);
    ensure_buffers(c, pr);
    auto t1 = std::chrono::steady_clock::now();
    stage_inputs(c, pr, inst, hoff, pins, nw, hw);
    auto t2 = std::chrono::steady_clock::now();
    const bool replay = c.exec && c.key == pr.key;
    const float ms = launch(c, pr, n, true, timing);
    auto t3 = std::chrono::steady_clock::now();
    const char *h = (const char *)c.host.p;
    std::memcpy(inst.data(), h + pr.lay.inst, sizeof(BInst) * (size_t)n);
    const int32_t *parts = reinterpret_cast<const int32_t *>(h + pr.lay.parts);
    const int tasks = std::min(n, 64);
    c.lanes->run(tasks, [&](int t) {
        for (int i = t; i < n; i += tasks)
            if (inst[i].status < kBlkDeferred) std::memcpy(outs[i], parts + inst[i].out, sizeof(int32_t) * (size_t)inst[i].N);
    });
    if (timing) {
        auto t4 = std::chrono::steady_clock::now();
        auto dms = [](auto a, auto b) { return std::chrono::duration<double, std::milli>(b - a).count(); };
        std::fprintf(stderr, "[bipart] block batch: %d instances, graph %s, prepare %.2f ms, staging %.2f ms "
                     "(%.1f MiB), device %.2f ms (events %.2f), copy-out %.2f ms\n", n,
                     replay ? "replayed" : "captured", dms(t0, t1), dms(t1, t2), pr.lay.in_end / 1048576.0,
                     dms(t2, t3), ms, dms(t3, t4));
        for (int b = 0; b < kBuckets; ++b)
            if (pr.run[b].count)
                std::fprintf(stderr, "[bipart]   bucket %d: %d instances, %d blocks x %d threads, arena %.1f MiB/block\n",
                             b, pr.run[b].count, pr.run[b].blocks, kShapes[pr.run[b].shape].threads,
                             pr.run[b].arena / 1048576.0);
    }
}

// Times every candidate shape on each bucket of the batch (kernel time by CUDA events, the best
// of two runs) and records the fastest per bucket, in this process and in the JSON cache.
// chosen[2 b], chosen[2 b + 1] receive bucket b's threads and blocks per SM (0 when the batch has
// no instance in it).
void tune_block_batch(std::vector<BInst> &inst, const std::vector<const int32_t *> &hoff,
                      const std::vector<const int32_t *> &pins, const std::vector<const int32_t *> &nw,
                      const std::vector<const int32_t *> &hw, int32_t *chosen) {
    const int n = (int)inst.size();
    BatchCtx &c = ctx();
    std::lock_guard<std::mutex> lk(c.mu);
    c.init();
    if (!c.table_loaded) {
        c.table = read_table(tune_path());
        c.table_loaded = true;
    }
    std::vector<int> counts(kBuckets, 0);
    for (const BInst &I : inst) counts[bucket_of(I.P)]++;
    const bool verbose = std::getenv("BIPART_TIMING") != nullptr;
    for (int b = 0; b < kBuckets; ++b) {
        if (chosen) chosen[2 * b] = chosen[2 * b + 1] = 0;
        if (counts[b] == 0) continue;
        // this bucket's instances alone
        std::vector<BInst> sub;
        std::vector<const int32_t *> sh, sp, sn, sw;
        for (int i = 0; i < n; ++i)
            if (bucket_of(inst[i].P) == b) {
                sub.push_back(inst[i]);
                sh.push_back(hoff[i]);
                sp.push_back(pins[i]);
                sn.push_back(nw[i]);
                sw.push_back(hw[i]);
            }
        int best = -1;
        float best_ms = 0.f;
        for (int s = 0; s < kNumShapes; ++s) {
            int force[kBuckets];
            for (int q = 0; q < kBuckets; ++q) force[q] = s;
            Prepared pr = prepare(c, sub, sn, sw, force);
            ensure_buffers(c, pr);
            stage_inputs(c, pr, sub, sh, sp, sn, sw);
            float ms = 0.f;
            for (int rep = 0; rep < 2; ++rep) {
                const float t = launch(c, pr, (int)sub.size(), false, true);
                ms = rep == 0 ? t : std::min(ms, t);
            }
            int deferred = 0;
            const BInst *out = reinterpret_cast<const BInst *>((const char *)c.host.p + pr.lay.inst);
            for (size_t i = 0; i < sub.size(); ++i) deferred += out[i].status == kBlkDeferred;
            if (verbose)
                std::fprintf(stderr, "[bipart] tune bucket %d (%zu instances): %d x %d per SM: %.2f ms%s\n", b,
                             sub.size(), kShapes[s].threads, kShapes[s].per_sm, ms,
                             deferred ? " (some deferred: not eligible)" : "");
            if (deferred) continue;
            if (best < 0 || ms < best_ms) {
                best = s;
                best_ms = ms;
            }
        }
        if (best < 0) continue;
        c.table[c.dev_key][b] = best;
        if (chosen) {
            chosen[2 * b] = kShapes[best].threads;
            chosen[2 * b + 1] = kShapes[best].per_sm;
        }
    }
    c.drop_graph();
    write_table(tune_path(), c.table);
}

// Device bytes the batch context needs for these instances (staging copy, outputs and arenas).
size_t block_batch_bytes(std::vector<BInst> inst) {
    if (inst.empty()) return 0;
    BatchCtx &c = ctx();
    std::lock_guard<std::mutex> lk(c.mu);
    c.init();
    std::vector<const int32_t *> nw(inst.size(), nullptr), hw(inst.size(), nullptr);
    for (size_t i = 0; i < inst.size(); ++i) {
        if (inst[i].nw >= 0) nw[i] = reinterpret_cast<const int32_t *>(1);  // only presence counts here
        if (inst[i].hw >= 0) hw[i] = reinterpret_cast<const int32_t *>(1);
    }
    const Prepared pr = prepare(c, inst, nw, hw, nullptr);
    return pr.lay.out_end + std::max<size_t>(pr.arena_total, 256) + 256;
}

// Frees the device buffers and graph of the batch context (the pinned staging stays).
void trim_block_batch() {
    BatchCtx &c = ctx();
    std::lock_guard<std::mutex> lk(c.mu);
    if (c.device < 0) return;
    if (c.stream) cudaStreamSynchronize(c.stream);
    c.drop_graph();
    c.dev.release();
    c.arena.release();
    c.misc.release();
}

// Frees the batch context's buffers and graph (they are kept between calls otherwise).
void release_block_batch() {
    BatchCtx &c = ctx();
    std::lock_guard<std::mutex> lk(c.mu);
    if (c.device < 0) return;
    if (c.stream) cudaStreamSynchronize(c.stream);
    c.drop_graph();
    c.host.release();
    c.dev.release();
    c.arena.release();
    c.misc.release();
}

}  // namespace bp
