// Batched and served partitioning: a native worker pool on one GPU.
//
// Every worker thread owns a private workspace (a handle with its own non-blocking CUDA stream
// and its own level store and scratch, grown to the largest instance it has seen), so any number
// of independent hypergraphs are partitioned concurrently: while one worker waits on its stream,
// the others keep the GPU busy.  A job's result depends only on its own input (the workspaces
// share nothing), so the output of an instance is the same alone, in a batch, or in any mix of
// served requests.
//
// Batch (bipart_partition_batch): all instances queued largest first (longest-processing-time
// order keeps the tail short), then waited for.
// Serving (bipart_server_*): requests arrive at any time; a request is admitted when its
// estimated working set fits the HBM budget next to the requests already running (continuous
// batching: new requests start as soon as memory and a worker are free, smaller ones may pass a
// large one that does not fit yet); each request records its queueing and running time.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace bp {

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
    bipart_instance inst;
    bipart_params params;
    int32_t *out = nullptr;
    int64_t ticket = 0;
    size_t bytes = 0;
    int status = 0;
    bool done = false;
    std::string error;
    Clock::time_point t_submit, t_start, t_end;
    uint64_t sig = 0;  // shape of the input and parameters (sizes only)
    int pref = -1;     // the worker that last ran this shape, whose launch plans fit it
    bool block_ok = false;  // the persistent block path can take it (server micro-batches)
};

// Shape of a request: what a worker's captured launch plans depend on besides the data.
uint64_t job_sig(const bipart_instance &in, const bipart_params &p) {
    const int64_t P = (in.num_hedges > 0 && in.hedge_offsets) ? in.hedge_offsets[in.num_hedges] : 0;
    uint64_t h = 0x9e3779b97f4a7c15ull;
    auto mix = [&](uint64_t v) {
        h ^= v + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
    };
    mix((uint64_t)in.num_nodes);
    mix((uint64_t)in.num_hedges);
    mix((uint64_t)P);
    mix((uint64_t)(in.node_weights != nullptr) | ((uint64_t)(in.hedge_weights != nullptr) << 1));
    mix((uint64_t)p.k);
    uint64_t eb;
    std::memcpy(&eb, &p.epsilon, sizeof(eb));
    mix(eb);
    mix((uint64_t)p.policy);
    mix((uint64_t)p.levels);
    mix((uint64_t)p.refine_iters);
    mix((uint64_t)p.flags);
    return h | 1;
}

// Estimated device working set of one job: level store over all levels (bounded by a few times
// level 0 for the shapes of interest), scratch and the input copy.  Checked against the bytes a
// request's workspace actually allocates (counted through the allocator hooks) on netlist and
// row-net requests with k in {2, 4, 16}.
size_t estimate_bytes(const bipart_instance &in) {
    const size_t N = (size_t)std::max(in.num_nodes, 0), E = (size_t)std::max(in.num_hedges, 0);
    const size_t P = (in.num_hedges > 0 && in.hedge_offsets) ? (size_t)std::max(in.hedge_offsets[in.num_hedges], 0) : 0;
    return 64 * P + 96 * E + 96 * N + (8u << 20);
}


// The persistent block path takes an instance when it fits a block (block_eligible) and does not
// ask for parallel-net merging, which only the grid path implements.
bool block_takes(const bipart_instance &in, const bipart_params &p) {
    const int64_t P = in.num_hedges > 0 ? in.hedge_offsets[in.num_hedges] : 0;
    return in.num_nodes > 0 && block_eligible(in.num_nodes, in.num_hedges, P, p.k, p.levels) &&
           !(p.flags & BIPART_FLAG_MERGE_PARALLEL);
}

// Descriptors and array pointers of the instances idx[] for the block path.
struct BlockSet {
    std::vector<BInst> bi;
    std::vector<const int32_t *> ho, pi, nw, hw;
};

BlockSet block_set(const std::vector<const bipart_instance *> &ins, const std::vector<const bipart_params *> &ps) {
    // instances without hyperedges still need an offsets array of one zero
    static const int32_t zero = 0;
    BlockSet b;
    const size_t n = ins.size();
    b.bi.resize(n);
    b.ho.resize(n);
    b.pi.resize(n);
    b.nw.resize(n);
    b.hw.resize(n);
    for (size_t j = 0; j < n; ++j) {
        const bipart_instance &in = *ins[j];
        const bipart_params &p = *ps[j];
        BInst &d = b.bi[j];
        d.N = in.num_nodes;
        d.E = in.num_hedges;
        d.P = in.num_hedges > 0 ? in.hedge_offsets[in.num_hedges] : 0;
        d.policy = p.policy;
        d.levels = p.levels;
        d.iters = p.refine_iters;
        d.k = p.k;
        d.e6 = make_params(p.k, p.epsilon, p.policy, p.levels, p.refine_iters, p.flags).e6;
        d.status = 0;
        d.nw = in.node_weights ? 0 : -1;  // presence (offsets are assigned by the batch)
        d.hw = in.hedge_weights ? 0 : -1;
        b.ho[j] = in.num_hedges > 0 ? in.hedge_offsets : &zero;
        b.pi[j] = in.hedge_pins;
        b.nw[j] = in.node_weights;
        b.hw[j] = in.hedge_weights;
    }
    return b;
}

BlockSet block_set(const std::vector<int32_t> &idx, const bipart_instance *instances,
                   const bipart_params *params) {
    std::vector<const bipart_instance *> ins;
    std::vector<const bipart_params *> ps;
    for (int32_t i : idx) {
        ins.push_back(instances + i);
        ps.push_back(params + i);
    }
    return block_set(ins, ps);
}

// The checks every instance gets on the host before any of its data is touched: sizes, pointers,
// hedge_offsets[0] and hedge_offsets[E] (the staging and the size buckets rely on them), then its
// parameters.  The CSR content is checked where it is read: by its block in the persistent batch
// kernel (kBlkMalformed, see block_error) or by the worker's creation of its workspace level 0.
void precheck(const bipart_instance &x, const bipart_params &p) {
    if (x.num_nodes < 0 || x.num_hedges < 0) throw Fail{BIPART_ERR_INVALID_ARG, "negative size"};
    if (x.num_hedges > 0 && !x.hedge_offsets) throw Fail{BIPART_ERR_INVALID_ARG, "hedge_offsets is NULL"};
    if (x.hedge_offsets && x.hedge_offsets[0] != 0) throw Fail{BIPART_ERR_INVALID_CSR, "hedge_offsets[0] != 0"};
    const int32_t P = x.num_hedges > 0 ? x.hedge_offsets[x.num_hedges] : 0;
    if (P < 0) throw Fail{BIPART_ERR_INVALID_CSR, "hedge_offsets[E] < 0"};
    if (P > 0 && !x.hedge_pins) throw Fail{BIPART_ERR_INVALID_ARG, "hedge_pins is NULL"};
    make_params(p.k, p.epsilon, p.policy, p.levels, p.refine_iters, p.flags);  // validates
}

// precheck on every instance; st[i] / err[i] record a failure.
void precheck_all(int32_t n, const bipart_instance *instances, const bipart_params *params,
                  std::vector<int32_t> &st, std::vector<std::string> &err) {
    for (int32_t i = 0; i < n; ++i) {
        try {
            precheck(instances[i], params[i]);
        } catch (const Fail &e) {
            st[i] = e.code;
            err[i] = e.msg;
        }
    }
}

// The error of an instance its block found malformed: the host pass over its CSR names the first
// offending entry.
Fail block_error(const bipart_instance &x) {
    try {
        validate_host_csr(x.num_nodes, x.num_hedges, x.hedge_offsets, x.hedge_pins, x.node_weights,
                          x.hedge_weights);
    } catch (const Fail &e) {
        return e;
    }
    return Fail{BIPART_ERR_INVALID_CSR, "malformed CSR (device check)"};
}


class Pool {
   public:
    // kid_lanes: the workspaces' host threads for the subgraphs of a k-way tree level (1: one
    // after another on the worker's stream; 0: the library default).  batching: waiting requests
    // the persistent block path takes are run together as one batch once enough of them queue up.
    Pool(int workers, size_t budget, int kid_lanes, bool batching = false)
        : budget_(budget), kid_lanes_(kid_lanes), batching_(batching) {
        BP_CUDA(cudaGetDevice(&device_));
        if (workers < 1) workers = 1;
        busy_.assign((size_t)workers, 0);
        for (int i = 0; i < workers; ++i) threads_.emplace_back([this, i]() { run(i); });
    }
    int workers() const { return (int)threads_.size(); }

    ~Pool() {
        {
            std::lock_guard<std::mutex> lk(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        for (std::thread &t : threads_) t.join();
    }

    // Queues a job; returns its ticket.  Jobs that fail the host checks (precheck) or are larger
    // than the whole budget are rejected: their ticket is done at once with the error.
    int64_t submit(const bipart_instance &inst, const bipart_params &p, int32_t *out, bool front_by_size) {
        auto j = std::make_shared<Job>();
        j->inst = inst;
        j->params = p;
        j->out = out;
        try {
            precheck(inst, p);
        } catch (const Fail &e) {
            j->status = e.code;
            j->error = e.msg;
            j->done = true;
            j->t_submit = j->t_start = j->t_end = Clock::now();
            std::lock_guard<std::mutex> lk(mu_);
            j->ticket = ++next_ticket_;
            jobs_[j->ticket] = j;
            done_cv_.notify_all();
            return j->ticket;
        }
        j->bytes = estimate_bytes(inst);
        j->sig = job_sig(inst, p);
        j->block_ok = batching_ && block_takes(inst, p) && batch_cost(inst, p) <= kBatchMaxCost;
        j->t_submit = Clock::now();
        std::lock_guard<std::mutex> lk(mu_);
        j->ticket = ++next_ticket_;
        auto last = last_.find(j->sig);
        if (last != last_.end()) j->pref = last->second;
        if (budget_ && j->bytes > budget_) {
            j->status = BIPART_ERR_OOM;
            j->error = "request exceeds the whole HBM budget";
            j->done = true;
            j->t_start = j->t_end = j->t_submit;
            jobs_[j->ticket] = j;
            done_cv_.notify_all();
            return j->ticket;
        }
        jobs_[j->ticket] = j;
        if (front_by_size) {
            auto it = std::find_if(queue_.begin(), queue_.end(),
                                   [&](const std::shared_ptr<Job> &q) { return q->bytes < j->bytes; });
            queue_.insert(it, j);
        } else {
            queue_.push_back(j);
        }
        // a job meant for one worker must reach that worker, not just any sleeping one
        if (j->pref >= 0) cv_.notify_all();
        else cv_.notify_one();
        return j->ticket;
    }

    // Waits for a ticket; timeout_ms < 0 waits forever.  Returns false on timeout.
    bool wait(int64_t ticket, int timeout_ms, std::shared_ptr<Job> *out) {
        std::unique_lock<std::mutex> lk(mu_);
        auto pred = [&]() {
            auto it = jobs_.find(ticket);
            return it == jobs_.end() || it->second->done;
        };
        if (timeout_ms < 0) done_cv_.wait(lk, pred);
        else if (!done_cv_.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) return false;
        auto it = jobs_.find(ticket);
        if (it == jobs_.end()) {
            out->reset();
            return true;
        }
        *out = it->second;
        jobs_.erase(it);
        return true;
    }

   private:
    void run(int me) {
        cudaSetDevice(device_);
        cudaStream_t s = nullptr;
        std::unique_ptr<bipart_graph> ws;
        try {
            BP_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
            ws.reset(graph_new(s));
            ws->kid_lanes = kid_lanes_;
            ws->lean = budget_ != 0;
        } catch (const Fail &) {
            ws.reset();
        }
        auto fresh_workspace = [&]() {
            // under a budget a worker holds device memory only while it runs a request: the
            // workspace is rebuilt empty before the request's share is given back
            try {
                ws.reset();
                ws.reset(graph_new(s));
                ws->kid_lanes = kid_lanes_;
                ws->lean = true;
            } catch (const Fail &) {
                ws.reset();
            }
        };
        auto run_one = [&](Job &j) {
            if (!ws) {
                j.status = BIPART_ERR_CUDA;
                j.error = "worker could not create its workspace";
                return;
            }
            try {
                const bipart_instance &in = j.inst;
                graph_load_host(ws.get(), in.num_nodes, in.num_hedges, in.hedge_offsets, in.hedge_pins,
                                in.node_weights, in.hedge_weights);
                const bipart_params &q = j.params;
                const Params p = make_params(q.k, q.epsilon, q.policy, q.levels, q.refine_iters, q.flags);
                j.status = graph_partition_host(ws.get(), p, j.out);
            } catch (const Fail &e) {
                j.status = e.code;
                j.error = e.msg;
            } catch (...) {
                j.status = BIPART_ERR_CUDA;
                j.error = "unexpected exception";
            }
        };
        for (;;) {
            std::shared_ptr<Job> j;
            std::vector<std::shared_ptr<Job>> batch;
            size_t batch_bytes = 0;
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [&]() { return (stop_ && queue_.empty()) || admissible(me) != queue_.end(); });
                if (stop_ && queue_.empty()) break;
                if (!take_batch(batch, batch_bytes)) {
                    auto it = admissible(me);
                    j = *it;
                    queue_.erase(it);
                    in_flight_ += j->bytes;
                }
                busy_[(size_t)me] = 1;
                // jobs left waiting for this worker may now go to any other
                if (!queue_.empty()) cv_.notify_all();
            }
            if (!batch.empty()) {
                run_batch(batch, run_one);
                if (budget_) {
                    trim_block_batch();
                    if (ws) fresh_workspace();
                }
                {
                    std::lock_guard<std::mutex> lk(mu_);
                    in_flight_ -= batch_bytes;
                    batch_busy_ = false;
                    busy_[(size_t)me] = 0;
                    for (auto &b : batch) b->done = true;
                }
                done_cv_.notify_all();
                cv_.notify_all();
                continue;
            }
            j->t_start = Clock::now();
            run_one(*j);
            j->t_end = Clock::now();
            if (budget_ && ws) fresh_workspace();
            {
                std::lock_guard<std::mutex> lk(mu_);
                in_flight_ -= j->bytes;
                j->done = true;
                busy_[(size_t)me] = 0;
                if (j->status >= 0) last_[j->sig] = me;
            }
            done_cv_.notify_all();
            cv_.notify_all();  // memory was released: more requests may fit now
        }
        ws.reset();
        if (s) cudaStreamDestroy(s);
    }

    // Server micro-batching: once at least kBatchMin waiting requests can run in the persistent
    // block path (a backlog: every worker is busy and requests queue up), a free worker takes up
    // to kBatchMax of them, in queue order, as one batch -- one thread block per request, all in
    // a few launches -- if the batch's device memory fits the budget next to the running jobs.
    // One batch runs at a time.  Called with mu_ held.
    // Only requests of at most kBatchMaxCost pin-bisections (pins x ceil(log2 k)) go into a
    // micro-batch: a batch completes as a whole, so its longest block sets every member's latency,
    // and one block takes about as long on a 256K-pin bisection as the grid path on a 2M-pin one.
    static constexpr int kBatchMin = 8, kBatchMax = 1024;
    static constexpr int64_t kBatchMaxCost = 256 << 10;
    static int64_t batch_cost(const bipart_instance &in, const bipart_params &p) {
        const int64_t P = in.num_hedges > 0 ? in.hedge_offsets[in.num_hedges] : 0;
        int depth = 1;
        while ((int64_t(1) << depth) < p.k) ++depth;
        return P * depth;
    }
    bool take_batch(std::vector<std::shared_ptr<Job>> &out, size_t &bytes) {
        if (!batching_ || batch_busy_) return false;
        std::vector<std::shared_ptr<Job>> cand;
        for (auto &q : queue_)
            if (q->block_ok && (int)cand.size() < kBatchMax) cand.push_back(q);
        if ((int)cand.size() < kBatchMin) return false;
        std::vector<const bipart_instance *> ins;
        std::vector<const bipart_params *> ps;
        for (auto &q : cand) {
            ins.push_back(&q->inst);
            ps.push_back(&q->params);
        }
        size_t need = 0;
        try {
            need = block_batch_bytes(block_set(ins, ps).bi);
        } catch (const Fail &) {
            return false;
        }
        if (budget_ && (need > budget_ || (in_flight_ != 0 && in_flight_ + need > budget_))) return false;
        std::deque<std::shared_ptr<Job>> rest;
        for (auto &q : queue_)
            if (!(q->block_ok && std::find(cand.begin(), cand.end(), q) != cand.end())) rest.push_back(q);
        queue_.swap(rest);
        in_flight_ += need;
        batch_busy_ = true;
        bytes = need;
        batches_ += 1;
        batched_ += (int64_t)cand.size();
        out.swap(cand);
        return true;
    }

   public:
    void stats(int64_t *batches, int64_t *batched) {
        std::lock_guard<std::mutex> lk(mu_);
        if (batches) *batches = batches_;
        if (batched) *batched = batched_;
    }

   private:

    // Runs a micro-batch on this thread; a request the block path defers runs alone here.
    template <class RunOne>
    void run_batch(std::vector<std::shared_ptr<Job>> &batch, RunOne &run_one) {
        const Clock::time_point t0 = Clock::now();
        std::vector<const bipart_instance *> ins;
        std::vector<const bipart_params *> ps;
        std::vector<int32_t *> outs;
        for (auto &b : batch) {
            b->t_start = t0;
            ins.push_back(&b->inst);
            ps.push_back(&b->params);
            outs.push_back(b->out);
        }
        try {
            BlockSet bs = block_set(ins, ps);
            // under a budget the batch holds only what it was admitted for (buffers a larger
            // earlier batch of this process left behind go first)
            if (budget_) trim_block_batch();
            run_block_batch(bs.bi, bs.ho, bs.pi, bs.nw, bs.hw, outs);
            const Clock::time_point t1 = Clock::now();
            for (size_t i = 0; i < batch.size(); ++i) {
                Job &j = *batch[i];
                if (bs.bi[i].status == kBlkDeferred) {
                    run_one(j);
                    j.t_end = Clock::now();
                } else if (bs.bi[i].status == kBlkMalformed) {
                    const Fail e = block_error(j.inst);
                    j.status = e.code;
                    j.error = e.msg;
                    j.t_end = Clock::now();
                } else {
                    j.status = bs.bi[i].status ? BIPART_WARN_IMBALANCED : BIPART_OK;
                    j.t_end = t1;
                }
            }
        } catch (const Fail &e) {
            for (auto &b : batch) {
                b->status = e.code;
                b->error = e.msg;
                b->t_end = Clock::now();
            }
        }
    }

    // First queued job that fits next to the running ones (always the head when nothing runs)
    // and that worker `me` may take: a job whose shape another worker ran last waits for that
    // worker (which can replay its launch plans) unless that worker is busy.
    std::deque<std::shared_ptr<Job>>::iterator admissible(int me) {
        for (auto it = queue_.begin(); it != queue_.end(); ++it) {
            const int pref = (*it)->pref;
            if (pref >= 0 && pref != me && pref < (int)busy_.size() && !busy_[(size_t)pref]) continue;
            if (!budget_ || in_flight_ == 0 || in_flight_ + (*it)->bytes <= budget_) return it;
        }
        return queue_.end();
    }

    int device_ = 0;
    size_t budget_ = 0;
    int kid_lanes_ = 0;
    bool batching_ = false;
    bool batch_busy_ = false;
    int64_t batches_ = 0, batched_ = 0;  // micro-batches run and the requests they held
    size_t in_flight_ = 0;
    bool stop_ = false;
    int64_t next_ticket_ = 0;
    std::mutex mu_;
    std::condition_variable cv_, done_cv_;
    std::deque<std::shared_ptr<Job>> queue_;
    std::unordered_map<int64_t, std::shared_ptr<Job>> jobs_;
    std::vector<char> busy_;
    std::unordered_map<uint64_t, int> last_;  // shape -> worker that ran it last
    std::vector<std::thread> threads_;
};

// The batch call's worker pool, kept between calls (its workspaces keep their level stores and
// launch plans); replaced when a call asks for another worker count.  Never destroyed at exit.
std::mutex g_batch_pool_mu;
std::shared_ptr<Pool> *g_batch_pool = new std::shared_ptr<Pool>();

std::shared_ptr<Pool> batch_pool(int workers) {
    std::lock_guard<std::mutex> lk(g_batch_pool_mu);
    // a batch's pool jobs are the few instances too large for a block: their k-way subgraphs
    // run concurrently
    if (!*g_batch_pool || (*g_batch_pool)->workers() != workers) g_batch_pool->reset(new Pool(workers, 0, 0));
    return *g_batch_pool;
}

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace
}  // namespace bp

struct bipart_server_s {
    std::unique_ptr<bp::Pool> pool;
};

using namespace bp;


// Batch: the instances the persistent block path takes run there (size buckets, one CUDA graph)
// on this thread; the others (and any instance the block path defers) go to the worker pool,
// which runs concurrently.
extern "C" int bipart_partition_batch(int32_t n, const bipart_instance *instances,
                                      const bipart_params *params, int32_t *const *out_parts,
                                      int32_t *statuses, int32_t workers) {
    if (n < 0 || (n > 0 && (!instances || !params || !out_parts))) {
        set_error("bipart_partition_batch: bad arguments");
        return BIPART_ERR_INVALID_ARG;
    }
    if (n == 0) return BIPART_OK;
    try {
        if (workers <= 0) workers = std::min<int32_t>(16, std::max<int32_t>(n, 1));
        std::vector<int32_t> st(n, BIPART_OK);
        std::vector<std::string> err(n);
        precheck_all(n, instances, params, st, err);
        std::vector<int32_t> blk, rest;
        for (int32_t i = 0; i < n; ++i) {
            if (st[i] != BIPART_OK) continue;
            if (block_takes(instances[i], params[i])) blk.push_back(i);
            else rest.push_back(i);
        }
        std::stable_sort(rest.begin(), rest.end(), [&](int32_t a, int32_t b) {
            return estimate_bytes(instances[a]) > estimate_bytes(instances[b]);
        });
        // the worker pool is made only if some valid instance needs it (an all-invalid batch
        // reports its validation errors without touching the GPU)
        std::shared_ptr<Pool> pool_owner;
        auto pool_ref = [&]() -> Pool & {
            if (!pool_owner) pool_owner = batch_pool(workers);
            return *pool_owner;
        };
        std::vector<int64_t> tickets(n, 0);
        for (int32_t i : rest) tickets[i] = pool_ref().submit(instances[i], params[i], out_parts[i], false);
        if (!blk.empty()) {
            BlockSet b = block_set(blk, instances, params);
            std::vector<int32_t *> outs(blk.size());
            for (size_t j = 0; j < blk.size(); ++j) outs[j] = out_parts[blk[j]];
            run_block_batch(b.bi, b.ho, b.pi, b.nw, b.hw, outs);
            for (size_t j = 0; j < blk.size(); ++j) {
                const int32_t i = blk[j];
                if (b.bi[j].status == kBlkDeferred) {  // did not fit the block arena: single-instance path
                    tickets[i] = pool_ref().submit(instances[i], params[i], out_parts[i], false);
                    continue;
                }
                if (b.bi[j].status == kBlkMalformed) {
                    const Fail e = block_error(instances[i]);
                    st[i] = e.code;
                    err[i] = e.msg;
                    continue;
                }
                st[i] = b.bi[j].status ? BIPART_WARN_IMBALANCED : BIPART_OK;
            }
        }
        for (int32_t i = 0; i < n; ++i) {
            if (!tickets[i]) continue;
            std::shared_ptr<Job> j;
            pool_ref().wait(tickets[i], -1, &j);
            st[i] = j ? j->status : BIPART_ERR_CUDA;
            if (j && st[i] < 0) err[i] = j->error;
        }
        int rc = BIPART_OK;
        for (int32_t i = 0; i < n; ++i) {
            if (statuses) statuses[i] = st[i];
            if (st[i] < 0 && rc == BIPART_OK) {
                rc = st[i];
                set_error("instance " + std::to_string(i) + ": " + err[i]);
            }
        }
        return rc;
    } catch (const Fail &e) {
        set_error(e.msg);
        return e.code;
    } catch (...) {
        set_error("bipart_partition_batch: unexpected exception");
        return BIPART_ERR_CUDA;
    }
}

extern "C" int bipart_batch_tune(int32_t n, const bipart_instance *instances, const bipart_params *params,
                                 int32_t *chosen) {
    if (n < 0 || (n > 0 && (!instances || !params))) {
        set_error("bipart_batch_tune: bad arguments");
        return BIPART_ERR_INVALID_ARG;
    }
    try {
        std::vector<int32_t> st(n, BIPART_OK);
        std::vector<std::string> err(n);
        precheck_all(n, instances, params, st, err);
        std::vector<int32_t> blk;
        for (int32_t i = 0; i < n; ++i) {
            if (st[i] != BIPART_OK) {
                set_error("instance " + std::to_string(i) + ": " + err[i]);
                return st[i];
            }
            if (block_takes(instances[i], params[i])) blk.push_back(i);
        }
        if (chosen)
            for (int q = 0; q < 8; ++q) chosen[q] = 0;
        if (blk.empty()) return BIPART_OK;
        BlockSet b = block_set(blk, instances, params);
        tune_block_batch(b.bi, b.ho, b.pi, b.nw, b.hw, chosen);
        return BIPART_OK;
    } catch (const Fail &e) {
        set_error(e.msg);
        return e.code;
    } catch (...) {
        set_error("bipart_batch_tune: unexpected exception");
        return BIPART_ERR_CUDA;
    }
}

extern "C" void bipart_batch_release(void) {
    try {
        release_block_batch();
        std::shared_ptr<Pool> old;
        {
            std::lock_guard<std::mutex> lk(g_batch_pool_mu);
            old.swap(*g_batch_pool);
        }
        old.reset();
        lib_pool_trim();
    } catch (...) {
    }
}

extern "C" int bipart_server_create(size_t hbm_budget_bytes, int32_t workers, bipart_server *out) {
    if (!out) {
        set_error("out is NULL");
        return BIPART_ERR_INVALID_ARG;
    }
    *out = nullptr;
    try {
        std::unique_ptr<bipart_server_s> s(new bipart_server_s);
        // requests run concurrently across workers; each one's k-way subgraphs one after another
        s->pool.reset(new Pool(workers > 0 ? workers : 8, hbm_budget_bytes, 1, true));
        *out = s.release();
        return BIPART_OK;
    } catch (const Fail &e) {
        set_error(e.msg);
        return e.code;
    } catch (...) {
        set_error("bipart_server_create: unexpected exception");
        return BIPART_ERR_CUDA;
    }
}

extern "C" int bipart_server_submit(bipart_server server, const bipart_instance *instance,
                                    const bipart_params *params, int32_t *out_parts,
                                    int64_t *ticket) {
    if (!server || !instance || !params || !ticket || (!out_parts && instance->num_nodes > 0)) {
        set_error("bipart_server_submit: NULL argument");
        return BIPART_ERR_INVALID_ARG;
    }
    *ticket = server->pool->submit(*instance, *params, out_parts, false);
    return BIPART_OK;
}

extern "C" int bipart_server_wait(bipart_server server, int64_t ticket, int32_t timeout_ms,
                                  int32_t *status, double *queue_ms, double *run_ms) {
    if (!server) {
        set_error("server is NULL");
        return BIPART_ERR_INVALID_ARG;
    }
    std::shared_ptr<Job> j;
    if (!server->pool->wait(ticket, timeout_ms, &j)) {
        set_error("bipart_server_wait: timed out");
        return BIPART_ERR_TIMEOUT;
    }
    if (!j) {
        set_error("bipart_server_wait: unknown ticket");
        return BIPART_ERR_INVALID_ARG;
    }
    if (status) *status = j->status;
    if (queue_ms) *queue_ms = ms_between(j->t_submit, j->t_start);
    if (run_ms) *run_ms = ms_between(j->t_start, j->t_end);
    if (j->status < 0) set_error(j->error);
    return BIPART_OK;
}

extern "C" int bipart_server_stats(bipart_server server, int64_t *batches, int64_t *batched_requests) {
    if (!server) {
        set_error("server is NULL");
        return BIPART_ERR_INVALID_ARG;
    }
    server->pool->stats(batches, batched_requests);
    return BIPART_OK;
}

extern "C" void bipart_server_destroy(bipart_server server) { delete server; }
