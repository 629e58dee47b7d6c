// Host-side structures of the sm_103a path: device buffers, the per-level store and the
// per-handle workspace.  Shared by the .cu translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <string>
#include <vector>

#include "bipart.h"
#include "common.cuh"

namespace bp {

// ---------------------------------------------------------------------------------- memory
void *dev_alloc(size_t bytes, cudaStream_t s);
void dev_free(void *p, size_t bytes, cudaStream_t s);

// A growable device buffer (capacity only grows; contents are not preserved on growth).
struct Buf {
    void *p = nullptr;
    size_t cap = 0;
    cudaStream_t s = nullptr;
    Buf() = default;
    Buf(const Buf &) = delete;
    Buf &operator=(const Buf &) = delete;
    ~Buf() { release(); }
    void release() {
        if (p) dev_free(p, cap, s);
        p = nullptr;
        cap = 0;
    }
    void *ensure(size_t bytes, cudaStream_t stream) {
        if (bytes == 0) bytes = 16;
        if (bytes > cap) {
            release();
            s = stream;
            size_t c = bytes + bytes / 8 + 256;
            p = dev_alloc(c, stream);
            if (!p) throw Fail{BIPART_ERR_OOM, "device allocation of " + std::to_string(c) + " bytes failed"};
            cap = c;
        }
        return p;
    }
    template <class T>
    T *as() const { return reinterpret_cast<T *>(p); }
};

// One level of the multilevel hierarchy, resident in HBM.
//   hoff[E+1], pins[P]   hyperedge -> pins CSR, pins ascending within a hyperedge
//   hw[E]                hyperedge weights (nullptr: all 1)
//   nw[N]                node weights
//   noff[N+1], nadj[P]   node -> hyperedges CSR (order within a node unspecified)
//   cmap[N], match[N]    node -> node of the next level; Algorithm 1 matching (when coarser
//                        levels exist)
struct Level {
    int32_t N = 0, E = 0, P = 0;
    bool unit_hw = true;
    Buf b_hoff, b_pins, b_hw, b_nw, b_noff, b_nadj, b_cmap, b_match;
    int32_t *hoff() const { return b_hoff.as<int32_t>(); }
    int32_t *pins() const { return b_pins.as<int32_t>(); }
    int32_t *hw() const { return unit_hw ? nullptr : b_hw.as<int32_t>(); }
    int32_t *nw() const { return b_nw.as<int32_t>(); }
    int32_t *noff() const { return b_noff.as<int32_t>(); }
    int32_t *nadj() const { return b_nadj.as<int32_t>(); }
    int32_t *cmap() const { return b_cmap.as<int32_t>(); }
    int32_t *match() const { return b_match.as<int32_t>(); }
    void reserve(int32_t n, int32_t e, int32_t p, bool unit, cudaStream_t s) {
        N = n; E = e; P = p; unit_hw = unit;
        b_hoff.ensure(sizeof(int32_t) * ((size_t)e + 1), s);
        b_pins.ensure(sizeof(int32_t) * (size_t)p, s);
        if (!unit) b_hw.ensure(sizeof(int32_t) * (size_t)e, s);
        b_nw.ensure(sizeof(int32_t) * (size_t)n, s);
        b_noff.ensure(sizeof(int32_t) * ((size_t)n + 1), s);
        b_nadj.ensure(sizeof(int32_t) * (size_t)p, s);
        b_cmap.ensure(sizeof(int32_t) * (size_t)n, s);
        b_match.ensure(sizeof(int32_t) * (size_t)n, s);
    }
};

// Scratch shared by all levels of one bisection, sized by the largest level seen.
struct Work {
    Buf scan;        // decoupled look-back tile states + tile counter
    Buf status;      // device error word (DevErr bits)
    Buf small;       // small device scalars (counters, totals, selection state)
    Buf e_a, e_b, e_c, e_d;  // per-hyperedge int32 scratch
    Buf e_key;       // per-hyperedge uint64 keys
    Buf n_a, n_b, n_c;       // per-node int32 scratch
    Buf n_key;       // per-node uint64 keys
    Buf p_a;         // per-pin int32 scratch
    Buf side_a, side_b;      // uint8 sides (ping-pong across levels)
    Buf gain;        // int32 gains
    Buf hc;          // int2 per-hyperedge gain contributions
    Buf list;        // node list (rebalance candidates)
    Buf pinned;      // host-pinned mirror of `small`
    uint32_t *host_small = nullptr;
};

struct Params {
    int32_t k;
    double eps;
    int32_t policy;
    int32_t levels;
    int32_t iters;
};

// Result of one bisection kept for parity queries.
struct Hierarchy {
    int32_t nlev = 0;
    bool valid = false;
};

}  // namespace bp

struct bipart_graph {
    int device = 0;
    cudaStream_t stream = nullptr;
    bp::Level L0;                                  // normalised input
    std::vector<std::unique_ptr<bp::Level>> lev;   // coarse levels 1.. of the last bisection
    bp::Hierarchy hier;
    bp::Work w;
    // k-way workspace: subgraph level 0 and its node map
    bp::Level sub0;
    bp::Buf part_a, part_b, l2g;
    int64_t total_node_weight = 0;
};

namespace bp {

// ------------------------------------------------------------------- coarsening (coarsen.cu)
// Builds level 0 from a device CSR (already validated): normalisation + incidence.
void build_level0(bipart_graph *g, Level &L, int32_t N, int32_t E, const int32_t *d_hoff,
                  const int32_t *d_pins, const int32_t *d_nw, const int32_t *d_hw);
// Algorithm 1 + 2 on `f`, producing `c` (sizes read back to the host).
void coarsen_level(bipart_graph *g, Level &f, Level &c, int policy);
// Node -> hyperedge incidence of a level whose hyperedge CSR is complete.
void build_incidence(bipart_graph *g, Level &L);

// -------------------------------------------------------------------- refinement (refine.cu)
// Runs Algorithms 3, 5 (+ rebalance) over the hierarchy; writes side of level 0.
int uncoarsen(bipart_graph *g, std::vector<Level *> &levels, int64_t limit, int32_t iters,
              uint8_t *d_side0);
int64_t balance_limit(int64_t W, double eps);

// ------------------------------------------------------------------------- diagnostics
// Brackets one kernel launch with CUDA events on `s` when profiling is on (see
// bipart_profile_enable); `bytes` is the launch's algorithmic traffic.
struct ProfScope {
    int slot = -1;
    ProfScope(const char *name, double bytes, cudaStream_t s);
    ~ProfScope();
};

// ------------------------------------------------------------------------- misc (api.cu)
uint32_t *dev_status(bipart_graph *g);
void check_status(bipart_graph *g);
void sync(bipart_graph *g);

}  // namespace bp
