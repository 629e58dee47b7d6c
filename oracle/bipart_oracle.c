/*
 * BiPart CPU ORACLE -- test infrastructure only.
 *
 * A plain, slow, sequential C restatement of the deterministic multilevel bisection of
 * Maleki, Agarwal, Burtscher and Pingali, "BiPart: A Parallel and Deterministic Multilevel
 * Hypergraph Partitioner" (PPoPP'21).  Only tests, the package's smoke check and the benchmark's
 * CPU-baseline leg may load it; the CUDA path shares no code, header or table with this file.
 *
 * Every function follows one algorithm of the paper in its order and notation; where the paper
 * is silent the fixed reading is stated at the function (the same readings are written out for
 * the CUDA path as specification, not as shared code):
 *
 *   normalise      input hyperedges -> sorted unique pins, drop < 2 pins (reading C10)
 *   match          Algorithm 1 (Sec. 3.1.1): three min passes; hash = MurmurHash3 fmix32 (C1-C3)
 *   coarsen        Algorithm 2 (Sec. 3.1.2): merge matched sets, attach singletons, contract
 *                  (C4-C9); optionally merge parallel nets of the contracted level (M1)
 *   gains          Algorithm 4 (Sec. 3.2): move gains from per-hyperedge side counts, weighted
 *                  by hyperedge weight (weighted cut, Sec. 1.1)
 *   initial        Algorithm 3 (Sec. 3.2): grow P0 by the top ceil(sqrt n) gains (C14)
 *   refine         Algorithm 5 (Sec. 3.3): gain >= 0 lists, swap the top l_min (C15)
 *   rebalance      Algorithm 5's final step, a variant of Algorithm 3 (C13)
 *   bisect         Sec. 3.4 multilevel driver: levels / stop rule (C11), balance limit (C12)
 *   partition      Algorithm 6 (Sec. 3.5): nested k-way by recursive bisection (C16), extended
 *                  to any k with proportional side targets and an optional per-bisection
 *                  epsilon (readings G1-G3)
 *   cut            Sec. 1.1: sum over hyperedges of w_e (lambda_e - 1) (C17)
 *
 * Pins: every function here is checked by the -m "not gpu" tests against brute force, closed
 * forms and invariants (see tests/test_oracle_*.py).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORC_OK 0
#define ORC_WARN_IMBALANCED 1
#define ORC_ERR_INVALID_ARG (-1)
#define ORC_ERR_OOM (-3)

enum { POL_LDH = 0, POL_HDH = 1, POL_LWD = 2, POL_HWD = 3, POL_RAND = 4 };

/* Refinement admits nodes whose gain is at least this value (Algorithm 5 filters gain >= 0). */
#define REFINE_MIN_GAIN 0

#define ORC_FLAG_ADAPTIVE 1
#define ORC_FLAG_MERGE 2

struct orc_hg;
struct orc_run;
struct orc_hg *orc_coarsen_ex(const struct orc_hg *g, int policy, int merge, int32_t *cmap,
                              int32_t *match_out);
struct orc_run *orc_bisect_ex(const struct orc_hg *g0, int64_t e6, int32_t m0, int32_t m,
                              int merge, int policy, int32_t levels, int32_t iters);
int32_t orc_initial_target(const struct orc_hg *g, uint8_t *side, int32_t m0, int32_t m);
int orc_rebalance2(const struct orc_hg *g, uint8_t *side, int64_t limit0, int64_t limit1,
                   int32_t *rounds_out);
int64_t orc_limit_part(int64_t W, int32_t ms, int32_t m, int64_t e6);
struct orc_run *orc_bisect_target(const struct orc_hg *g0, int64_t e6, int32_t m0, int32_t m,
                                  int policy, int32_t levels, int32_t iters);

typedef struct orc_hg {
    int32_t N, E;
    int32_t *off;   /* E + 1 */
    int32_t *pin;   /* off[E]; pins of e are sorted ascending and unique */
    int32_t *nwt;   /* N node weights (>= 1) */
    int32_t *hwt;   /* E hyperedge weights (>= 1) */
} orc_hg;

static void *xmalloc(size_t n) { return malloc(n ? n : 1); }
static void *xcalloc(size_t n, size_t s) { return calloc(n ? n : 1, s ? s : 1); }

void orc_hg_free(orc_hg *g) {
    if (!g) return;
    free(g->off); free(g->pin); free(g->nwt); free(g->hwt); free(g);
}

static orc_hg *hg_alloc(int32_t N, int32_t E, int64_t P) {
    orc_hg *g = (orc_hg *)xcalloc(1, sizeof(orc_hg));
    g->N = N; g->E = E;
    g->off = (int32_t *)xmalloc(sizeof(int32_t) * ((size_t)E + 1));
    g->pin = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)P);
    g->nwt = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)N);
    g->hwt = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)E);
    return g;
}

int32_t orc_hg_N(const orc_hg *g) { return g->N; }
int32_t orc_hg_E(const orc_hg *g) { return g->E; }
int32_t orc_hg_P(const orc_hg *g) { return g->off[g->E]; }

void orc_hg_copy(const orc_hg *g, int32_t *off, int32_t *pin, int32_t *nwt, int32_t *hwt) {
    if (off) memcpy(off, g->off, sizeof(int32_t) * ((size_t)g->E + 1));
    if (pin) memcpy(pin, g->pin, sizeof(int32_t) * (size_t)g->off[g->E]);
    if (nwt) memcpy(nwt, g->nwt, sizeof(int32_t) * (size_t)g->N);
    if (hwt) memcpy(hwt, g->hwt, sizeof(int32_t) * (size_t)g->E);
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Sort a pin list ascending and drop repeats; returns the distinct count. */
static int32_t sort_unique(int32_t *a, int32_t n) {
    if (n == 0) return 0;
    qsort(a, (size_t)n, sizeof(int32_t), cmp_i32);
    int32_t m = 1;
    for (int32_t i = 1; i < n; i++)
        if (a[i] != a[m - 1]) a[m++] = a[i];
    return m;
}

/* ------------------------------------------------------------------------------------------
 * Reading C10: level 0 is the input with each hyperedge's pins sorted ascending and
 * deduplicated; hyperedges left with fewer than 2 distinct pins are dropped (they can never be
 * cut) and the survivors are renumbered in ascending input order, keeping their weights.
 * NULL weights mean unit weights.  The input is assumed valid (offsets monotone, pins in range).
 * ------------------------------------------------------------------------------------------ */
orc_hg *orc_hg_normalise(int32_t N, int32_t E, const int32_t *off, const int32_t *pins,
                         const int32_t *nwt, const int32_t *hwt) {
    int64_t P = off[E];
    orc_hg *g = hg_alloc(N, E, P);
    for (int32_t v = 0; v < N; v++) g->nwt[v] = nwt ? nwt[v] : 1;
    int32_t *buf = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)(P > 0 ? P : 1));
    int32_t ne = 0, np = 0;
    g->off[0] = 0;
    for (int32_t e = 0; e < E; e++) {
        int32_t d = off[e + 1] - off[e];
        memcpy(buf, pins + off[e], sizeof(int32_t) * (size_t)d);
        int32_t m = sort_unique(buf, d);
        if (m < 2) continue;
        memcpy(g->pin + np, buf, sizeof(int32_t) * (size_t)m);
        np += m;
        g->hwt[ne] = hwt ? hwt[e] : 1;
        g->off[++ne] = np;
    }
    g->E = ne;
    free(buf);
    return g;
}

/* ------------------------------------------------------------------------------------------
 * Reading C1: the hash of Algorithm 1 is the MurmurHash3 32-bit finaliser (fmix32, Appleby),
 * applied to the level-local hyperedge id.  It is a bijection of 32-bit integers, so
 * (priority, hash) is unique per hyperedge.
 * ------------------------------------------------------------------------------------------ */
uint32_t orc_hash(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

/* Reading C2/C4 (Table 1): lower value = higher priority; degree = distinct pins at this level. */
uint32_t orc_priority(const orc_hg *g, int32_t e, int policy) {
    uint32_t deg = (uint32_t)(g->off[e + 1] - g->off[e]);
    uint32_t w = (uint32_t)g->hwt[e];
    switch (policy) {
        case POL_LDH: return deg;
        case POL_HDH: return 0xFFFFFFFFu - deg;
        case POL_LWD: return w;
        case POL_HWD: return 0xFFFFFFFFu - w;
        default:      return orc_hash((uint32_t)e);
    }
}

/* ------------------------------------------------------------------------------------------
 * Algorithm 1 (parallel matching policy), sequentially.  Three passes over the hyperedges:
 *   (1) node.priority = min over incident hyperedges of hedge.priority;
 *   (2) node.rand     = min hedge.rand over incident hyperedges whose priority equals it;
 *   (3) node.hedgeid  = min hedge.id over incident hyperedges with that priority and rand.
 * The third pass also compares the priority (reading C3); with a bijective hash the rand test
 * alone picks the same hyperedge.  Nodes in no hyperedge keep hedgeid = infinity -> -1 (C6).
 * ------------------------------------------------------------------------------------------ */
void orc_match(const orc_hg *g, int policy, int32_t *hedgeid) {
    const uint64_t INF = UINT64_MAX;
    uint64_t *npri = (uint64_t *)xmalloc(sizeof(uint64_t) * (size_t)g->N);
    uint64_t *nrand = (uint64_t *)xmalloc(sizeof(uint64_t) * (size_t)g->N);
    uint64_t *nid = (uint64_t *)xmalloc(sizeof(uint64_t) * (size_t)g->N);
    for (int32_t v = 0; v < g->N; v++) { npri[v] = INF; nrand[v] = INF; nid[v] = INF; }
    for (int32_t e = 0; e < g->E; e++) {
        uint64_t pr = orc_priority(g, e, policy);
        for (int32_t i = g->off[e]; i < g->off[e + 1]; i++) {
            int32_t v = g->pin[i];
            if (pr < npri[v]) npri[v] = pr;
        }
    }
    for (int32_t e = 0; e < g->E; e++) {
        uint64_t pr = orc_priority(g, e, policy), rd = orc_hash((uint32_t)e);
        for (int32_t i = g->off[e]; i < g->off[e + 1]; i++) {
            int32_t v = g->pin[i];
            if (pr == npri[v] && rd < nrand[v]) nrand[v] = rd;
        }
    }
    for (int32_t e = 0; e < g->E; e++) {
        uint64_t pr = orc_priority(g, e, policy), rd = orc_hash((uint32_t)e);
        for (int32_t i = g->off[e]; i < g->off[e + 1]; i++) {
            int32_t v = g->pin[i];
            if (pr == npri[v] && rd == nrand[v] && (uint64_t)e < nid[v]) nid[v] = (uint64_t)e;
        }
    }
    for (int32_t v = 0; v < g->N; v++) hedgeid[v] = nid[v] == INF ? -1 : (int32_t)nid[v];
    free(npri); free(nrand); free(nid);
}

/* ------------------------------------------------------------------------------------------
 * Algorithm 2 (parallel coarsening), sequentially.
 *   S(e) = { v in e : hedgeid(v) = e }.
 *   Step 1: every S(e) with |S(e)| > 1 becomes one merged node (group id e).
 *   Step 2 (reading C7): for S(e) = {u}, the "already merged" nodes of e are those merged in
 *     step 1 (a snapshot: attachments made in step 2 do not count, weights are not updated);
 *     u joins the merged node of smallest weight (sum of its step-1 members' weights), ties to
 *     the smaller group id; with no merged node in e, u stays alone.  Unmatched nodes stay alone.
 *   Step 3 (readings C8, C9): coarse nodes are numbered in ascending order of their smallest
 *     fine member; each fine hyperedge whose pins have more than one distinct parent becomes a
 *     coarse hyperedge (ascending fine id) with sorted unique pins and the same weight.
 * cmap[v] receives the coarse node of fine node v.  The matching is returned in match (N).
 * ------------------------------------------------------------------------------------------ */
/* ------------------------------------------------------------------------------------------
 * Reading M1 (a switch, off by default; the paper never merges hyperedges): parallel nets of a
 * contracted level -- coarse hyperedges with the same sorted pin list -- become the one with the
 * smallest id, which keeps its place and carries the sum of their weights; the others are
 * dropped.  Every cut is unchanged, since identical nets are cut together.
 * ------------------------------------------------------------------------------------------ */
static const orc_hg *g_lists;  /* hyperedges compared by cmp_lists (single-threaded oracle) */

static int cmp_lists(const void *pa, const void *pb) {
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    int32_t da = g_lists->off[a + 1] - g_lists->off[a], db = g_lists->off[b + 1] - g_lists->off[b];
    const int32_t *la = g_lists->pin + g_lists->off[a], *lb = g_lists->pin + g_lists->off[b];
    for (int32_t i = 0; i < da && i < db; i++)
        if (la[i] != lb[i]) return la[i] < lb[i] ? -1 : 1;
    if (da != db) return da < db ? -1 : 1;
    return a < b ? -1 : (a > b ? 1 : 0);
}

static int same_list(const orc_hg *c, int32_t a, int32_t b) {
    int32_t da = c->off[a + 1] - c->off[a], db = c->off[b + 1] - c->off[b];
    if (da != db) return 0;
    return memcmp(c->pin + c->off[a], c->pin + c->off[b], sizeof(int32_t) * (size_t)da) == 0;
}

void orc_merge_parallel(orc_hg *c) {
    int32_t E = c->E;
    if (E < 2) return;
    int32_t *idx = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)E);
    int32_t *rep = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)E);
    int64_t *w = (int64_t *)xcalloc((size_t)E, sizeof(int64_t));
    for (int32_t e = 0; e < E; e++) idx[e] = e;
    g_lists = c;
    qsort(idx, (size_t)E, sizeof(int32_t), cmp_lists);
    for (int32_t i = 0; i < E; i++) {
        /* runs of equal lists are sorted by id: the run's first is the smallest id */
        rep[idx[i]] = (i > 0 && same_list(c, idx[i], idx[i - 1])) ? rep[idx[i - 1]] : idx[i];
    }
    for (int32_t e = 0; e < E; e++) w[rep[e]] += c->hwt[e];
    int32_t ne = 0, np = 0;
    for (int32_t e = 0; e < E; e++) {
        if (rep[e] != e) continue;
        int32_t a = c->off[e], d = c->off[e + 1] - a;
        memmove(c->pin + np, c->pin + a, sizeof(int32_t) * (size_t)d);
        c->hwt[ne] = (int32_t)w[e];
        np += d;
        c->off[++ne] = np;
    }
    c->E = ne;
    free(idx); free(rep); free(w);
}

orc_hg *orc_coarsen(const orc_hg *g, int policy, int32_t *cmap, int32_t *match_out) {
    return orc_coarsen_ex(g, policy, 0, cmap, match_out);
}

/* Algorithm 2, then (with `merge`) reading M1 on the contracted level. */
orc_hg *orc_coarsen_ex(const orc_hg *g, int policy, int merge, int32_t *cmap, int32_t *match_out) {
    int32_t N = g->N, E = g->E;
    int32_t *hedgeid = match_out ? match_out : (int32_t *)xmalloc(sizeof(int32_t) * (size_t)N);
    orc_match(g, policy, hedgeid);

    int32_t *Ssize = (int32_t *)xcalloc((size_t)E, sizeof(int32_t));
    int64_t *mergedw = (int64_t *)xcalloc((size_t)E, sizeof(int64_t));
    /* parent: >= 0 -> the merged node formed from S(parent); -1 - v -> node v on its own */
    int32_t *parent = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)N);
    for (int32_t v = 0; v < N; v++) parent[v] = -1 - v;

    for (int32_t e = 0; e < E; e++)
        for (int32_t i = g->off[e]; i < g->off[e + 1]; i++)
            if (hedgeid[g->pin[i]] == e) Ssize[e]++;

    /* Step 1: merge every S(e) with more than one node. */
    uint8_t *merged = (uint8_t *)xcalloc((size_t)N, 1);
    for (int32_t e = 0; e < E; e++) {
        if (Ssize[e] <= 1) continue;
        for (int32_t i = g->off[e]; i < g->off[e + 1]; i++) {
            int32_t v = g->pin[i];
            if (hedgeid[v] != e) continue;
            parent[v] = e;
            merged[v] = 1;
            mergedw[e] += g->nwt[v];
        }
    }
    /* Step 2: singleton sets join the lightest merged node of their hyperedge. */
    for (int32_t e = 0; e < E; e++) {
        if (Ssize[e] != 1) continue;
        int32_t u = -1, best = -1;
        for (int32_t i = g->off[e]; i < g->off[e + 1]; i++) {
            int32_t v = g->pin[i];
            if (hedgeid[v] == e) u = v;
        }
        for (int32_t i = g->off[e]; i < g->off[e + 1]; i++) {
            int32_t v = g->pin[i];
            if (!merged[v]) continue;
            int32_t gv = parent[v];
            if (best < 0 || mergedw[gv] < mergedw[best] || (mergedw[gv] == mergedw[best] && gv < best))
                best = gv;
        }
        parent[u] = best >= 0 ? best : -1 - u;
    }

    /* Step 3a: coarse node ids, ascending by smallest fine member. */
    int32_t *grp_first = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)(E > 0 ? E : 1));
    for (int32_t e = 0; e < E; e++) grp_first[e] = -1;
    int32_t Nc = 0;
    for (int32_t v = 0; v < N; v++) {
        int32_t p = parent[v];
        if (p < 0) {
            cmap[v] = Nc++;
        } else if (grp_first[p] < 0) {
            grp_first[p] = Nc;
            cmap[v] = Nc++;
        } else {
            cmap[v] = grp_first[p];
        }
    }
    /* Step 3b: coarse hyperedges. */
    int64_t P = g->off[E];
    orc_hg *c = hg_alloc(Nc, E, P);
    for (int32_t k = 0; k < Nc; k++) c->nwt[k] = 0;
    for (int32_t v = 0; v < N; v++) c->nwt[cmap[v]] += g->nwt[v];
    int32_t ne = 0, np = 0;
    c->off[0] = 0;
    for (int32_t e = 0; e < E; e++) {
        int32_t d = g->off[e + 1] - g->off[e];
        int32_t *dst = c->pin + np;
        for (int32_t i = 0; i < d; i++) dst[i] = cmap[g->pin[g->off[e] + i]];
        int32_t m = sort_unique(dst, d);
        if (m < 2) continue;
        np += m;
        c->hwt[ne] = g->hwt[e];
        c->off[++ne] = np;
    }
    c->E = ne;
    if (merge) orc_merge_parallel(c);

    free(grp_first); free(merged); free(parent); free(mergedw); free(Ssize);
    if (!match_out) free(hedgeid);
    return c;
}

/* ------------------------------------------------------------------------------------------
 * Algorithm 4 (move gains).  For each hyperedge, n0 / n1 count its pins in P0 / P1; a pin u on
 * side i gains w_e when it is the only pin of e on side i (moving it uncuts e) and loses w_e when
 * all pins of e are on side i (moving it cuts e).  With unit weights this is Algorithm 4 as
 * printed; with weights it is the change of the weighted cut.
 * ------------------------------------------------------------------------------------------ */
void orc_gains(const orc_hg *g, const uint8_t *side, int32_t *gain) {
    for (int32_t v = 0; v < g->N; v++) gain[v] = 0;
    for (int32_t e = 0; e < g->E; e++) {
        int32_t n[2] = {0, 0}, d = g->off[e + 1] - g->off[e];
        for (int32_t i = g->off[e]; i < g->off[e + 1]; i++) n[side[g->pin[i]]]++;
        for (int32_t i = g->off[e]; i < g->off[e + 1]; i++) {
            int32_t u = g->pin[i];
            int32_t ni = n[side[u]];
            if (ni == 1) gain[u] += g->hwt[e];
            else if (ni == d) gain[u] -= g->hwt[e];
        }
    }
}

/* Node order used by Algorithms 3 and 5: higher gain first, ties to the smaller node id. */
typedef struct { int32_t gain, id, w; } cand_t;
static int cmp_cand(const void *a, const void *b) {
    const cand_t *x = (const cand_t *)a, *y = (const cand_t *)b;
    if (x->gain != y->gain) return x->gain > y->gain ? -1 : 1;
    return (x->id > y->id) - (x->id < y->id);
}

/* ceil(sqrt(n)) in integers (reading C14). */
int64_t orc_ceil_sqrt(int64_t n) {
    if (n <= 0) return 0;
    int64_t r = (int64_t)sqrt((double)n);
    while (r * r > n) r--;
    while ((r + 1) * (r + 1) <= n) r++;
    return r * r == n ? r : r + 1;
}

static void side_weights(const orc_hg *g, const uint8_t *side, int64_t W[2]) {
    W[0] = W[1] = 0;
    for (int32_t v = 0; v < g->N; v++) W[side[v]] += g->nwt[v];
}

/* ------------------------------------------------------------------------------------------
 * Algorithm 3 (initial partitioning) on the coarsest level.  P0 = {}, P1 = V; while P0 is
 * lighter than P1 (by node weight, reading C14), recompute the gains and move the
 * s = ceil(sqrt(n)) nodes of P1 with the highest gains (ties to the smaller id) to P0; the last
 * round may overshoot.  Returns the number of rounds.
 * ------------------------------------------------------------------------------------------ */
int32_t orc_initial(const orc_hg *g, uint8_t *side) { return orc_initial_target(g, side, 1, 2); }

/* Reading G2: with side 0 meant to hold m0 of the m parts of this subgraph, "P0 lighter than P1"
 * becomes "P0 below its share": m * W0 < m0 * W.  For m0 / m = 1 / 2 this is W0 < W1. */
int32_t orc_initial_target(const orc_hg *g, uint8_t *side, int32_t m0, int32_t m) {
    int32_t n = g->N;
    int64_t s = orc_ceil_sqrt(n);
    for (int32_t v = 0; v < n; v++) side[v] = 1;
    int64_t W[2];
    side_weights(g, side, W);
    const int64_t Wt = W[0] + W[1];
    int32_t *gain = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    cand_t *L = (cand_t *)xmalloc(sizeof(cand_t) * (size_t)(n > 0 ? n : 1));
    int32_t rounds = 0;
    while ((int64_t)m * W[0] < (int64_t)m0 * Wt) {
        orc_gains(g, side, gain);
        int32_t m = 0;
        for (int32_t v = 0; v < n; v++)
            if (side[v] == 1) { L[m].gain = gain[v]; L[m].id = v; L[m].w = g->nwt[v]; m++; }
        qsort(L, (size_t)m, sizeof(cand_t), cmp_cand);
        int64_t take = s < m ? s : m;
        for (int64_t i = 0; i < take; i++) {
            side[L[i].id] = 0;
            W[0] += L[i].w;
            W[1] -= L[i].w;
        }
        rounds++;
    }
    free(gain); free(L);
    return rounds;
}

/* ------------------------------------------------------------------------------------------
 * Algorithm 5, one refinement iteration: gains; L_i = nodes of P_i with gain >= 0 (reading C15);
 * both lists in (gain desc, id asc) order; the first l_min = min(|L0|, |L1|) of each list swap
 * sides at once (gains are not updated in between).  Returns l_min.
 * ------------------------------------------------------------------------------------------ */
int32_t orc_refine_iter(const orc_hg *g, uint8_t *side) {
    int32_t n = g->N;
    int32_t *gain = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)n);
    cand_t *L0 = (cand_t *)xmalloc(sizeof(cand_t) * (size_t)n);
    cand_t *L1 = (cand_t *)xmalloc(sizeof(cand_t) * (size_t)n);
    orc_gains(g, side, gain);
    int32_t m0 = 0, m1 = 0;
    for (int32_t v = 0; v < n; v++) {
        if (gain[v] < REFINE_MIN_GAIN) continue;
        cand_t c = {gain[v], v, g->nwt[v]};
        if (side[v] == 0) L0[m0++] = c; else L1[m1++] = c;
    }
    qsort(L0, (size_t)m0, sizeof(cand_t), cmp_cand);
    qsort(L1, (size_t)m1, sizeof(cand_t), cmp_cand);
    int32_t lmin = m0 < m1 ? m0 : m1;
    for (int32_t i = 0; i < lmin; i++) { side[L0[i].id] = 1; side[L1[i].id] = 0; }
    free(gain); free(L0); free(L1);
    return lmin;
}

/* ------------------------------------------------------------------------------------------
 * Reading C12: the weight limit of one side of a bisection with total weight W and imbalance
 * eps is max(ceil(W/2), floor(W * (10^6 + e) / (2 * 10^6))), e = llround(eps * 10^6).
 * ------------------------------------------------------------------------------------------ */
int64_t orc_limit(int64_t W, double eps) {
    int64_t e6 = llround(eps * 1e6);
    int64_t a = (W + 1) / 2;
    int64_t b = (W * (1000000 + e6)) / 2000000;
    return a > b ? a : b;
}

/* Reading G2: the limit of a side meant to hold ms of the m parts of a subgraph of weight W, with
 * imbalance e6 millionths: max(ceil(W ms / m), floor(W ms (10^6 + e6) / (m 10^6))).  For
 * ms / m = 1 / 2 this is orc_limit.  Exact in 128-bit integers. */
int64_t orc_limit_part(int64_t W, int32_t ms, int32_t m, int64_t e6) {
    __int128 num = (__int128)W * ms;
    int64_t a = (int64_t)((num + m - 1) / m);
    int64_t b = (int64_t)(num * (1000000 + e6) / ((__int128)m * 1000000));
    return a > b ? a : b;
}

/* Reading G3: the per-bisection imbalance when every bisection on the way to k parts may use
 * the same allowance: the largest x in [0, e6] with (10^6 + x)^L <= (10^6 + e6) (10^6)^(L-1),
 * L = ceil(log2 k), i.e. floor(10^6 ((1 + eps)^(1/L) - 1)) without floating point.  L <= 1
 * returns e6.  The powers are compared exactly in base-2^32 integers. */
#define BIG_LIMBS 40
typedef struct { uint32_t d[BIG_LIMBS]; } big_t;

static void big_set(big_t *a, uint32_t v) { memset(a, 0, sizeof(*a)); a->d[0] = v; }

static void big_mul(big_t *a, uint32_t v) {
    uint64_t carry = 0;
    for (int i = 0; i < BIG_LIMBS; i++) {
        uint64_t t = (uint64_t)a->d[i] * v + carry;
        a->d[i] = (uint32_t)t;
        carry = t >> 32;
    }
}

static int big_cmp(const big_t *a, const big_t *b) {
    for (int i = BIG_LIMBS - 1; i >= 0; i--) {
        if (a->d[i] != b->d[i]) return a->d[i] < b->d[i] ? -1 : 1;
    }
    return 0;
}

static int32_t ceil_log2(int64_t k) {
    int32_t L = 0;
    while (((int64_t)1 << L) < k) L++;
    return L;
}

int64_t orc_adaptive_e6(int64_t e6, int32_t k) {
    int32_t L = ceil_log2(k);
    if (L <= 1) return e6;
    big_t rhs;
    big_set(&rhs, (uint32_t)(1000000 + e6));
    for (int32_t i = 1; i < L; i++) big_mul(&rhs, 1000000u);
    int64_t lo = 0, hi = e6;  /* lo satisfies the bound; find the largest that does */
    while (lo < hi) {
        int64_t mid = lo + (hi - lo + 1) / 2;
        big_t lhs;
        big_set(&lhs, 1);
        for (int32_t i = 0; i < L; i++) big_mul(&lhs, (uint32_t)(1000000 + mid));
        if (big_cmp(&lhs, &rhs) <= 0) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

/* ------------------------------------------------------------------------------------------
 * Algorithm 5, final step (reading C13, "a variant of Algorithm 3"): while the heavier side H
 * exceeds the limit, recompute the gains; the candidates are the nodes of H whose weight fits in
 * room = limit - W(other side), in (gain desc, id asc) order; move the shortest prefix whose
 * weight reaches need = W(H) - limit, stopping early at s = ceil(sqrt(n)) nodes or when the next
 * node would exceed room.  Returns ORC_OK when balanced, ORC_WARN_IMBALANCED when no candidate
 * is left while H is still too heavy.
 * ------------------------------------------------------------------------------------------ */
int orc_rebalance(const orc_hg *g, uint8_t *side, int64_t limit, int32_t *rounds_out) {
    return orc_rebalance2(g, side, limit, limit, rounds_out);
}

/* Reading G2: the same with a limit per side (side s may hold up to limit_s); room and need are
 * taken against the limits of the light and the heavy side. */
int orc_rebalance2(const orc_hg *g, uint8_t *side, int64_t limit0, int64_t limit1, int32_t *rounds_out) {
    const int64_t lim[2] = {limit0, limit1};
    int32_t n = g->N;
    int64_t s = orc_ceil_sqrt(n);
    int32_t *gain = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    cand_t *L = (cand_t *)xmalloc(sizeof(cand_t) * (size_t)(n > 0 ? n : 1));
    int status = ORC_OK, rounds = 0;
    for (;;) {
        int64_t W[2];
        side_weights(g, side, W);
        int H;
        if (W[0] > lim[0]) H = 0;
        else if (W[1] > lim[1]) H = 1;
        else break;
        int64_t room = lim[1 - H] - W[1 - H], need = W[H] - lim[H];
        orc_gains(g, side, gain);
        int32_t m = 0;
        for (int32_t v = 0; v < n; v++)
            if (side[v] == H && g->nwt[v] <= room) { L[m].gain = gain[v]; L[m].id = v; L[m].w = g->nwt[v]; m++; }
        if (m == 0) { status = ORC_WARN_IMBALANCED; break; }
        qsort(L, (size_t)m, sizeof(cand_t), cmp_cand);
        int64_t moved = 0, cnt = 0;
        for (int32_t i = 0; i < m && cnt < s; i++) {
            if (moved + L[i].w > room) break;
            side[L[i].id] = (uint8_t)(1 - H);
            moved += L[i].w;
            cnt++;
            if (moved >= need) break;
        }
        rounds++;
    }
    if (rounds_out) *rounds_out = rounds;
    free(gain); free(L);
    return status;
}

/* ------------------------------------------------------------------------------------------
 * Sec. 3.4 multilevel bisection.  Coarsen with Algorithm 2 until `levels` coarse levels exist
 * or a contraction leaves the node count unchanged (reading C11; that coarse level is
 * discarded); Algorithm 3 on the coarsest level; then from the coarsest level to the input:
 * project (Algorithm 5's initialisation, except at the coarsest level), `iters` refinement
 * iterations, rebalance against the limit of reading C12.
 * ------------------------------------------------------------------------------------------ */
typedef struct orc_run {
    int32_t nlev;          /* number of levels including level 0 */
    orc_hg **lev;          /* lev[0] is the (borrowed) input */
    int32_t **cmap;        /* cmap[l]: level l -> level l+1, for l < nlev - 1 */
    int32_t **match;       /* Algorithm 1 result at level l, for l < nlev - 1 */
    uint8_t *side;         /* final bisection of level 0 */
    int32_t init_rounds;
    int status;            /* ORC_OK or ORC_WARN_IMBALANCED (of the level-0 rebalance) */
    int64_t limit;
} orc_run;

orc_run *orc_bisect(const orc_hg *g0, double eps, int policy, int32_t levels, int32_t iters) {
    return orc_bisect_target(g0, llround(eps * 1e6), 1, 2, policy, levels, iters);
}

/* The same bisection with side 0 meant to hold m0 of m parts (reading G2) and the imbalance given
 * in millionths.  m0 / m = 1 / 2 is orc_bisect. */
orc_run *orc_bisect_target(const orc_hg *g0, int64_t e6, int32_t m0, int32_t m, int policy,
                           int32_t levels, int32_t iters) {
    return orc_bisect_ex(g0, e6, m0, m, 0, policy, levels, iters);
}

/* The same with `merge` (reading M1) applied to every contracted level. */
orc_run *orc_bisect_ex(const orc_hg *g0, int64_t e6, int32_t m0, int32_t m, int merge, int policy,
                       int32_t levels, int32_t iters) {
    orc_run *r = (orc_run *)xcalloc(1, sizeof(orc_run));
    int32_t cap = levels + 1;
    r->lev = (orc_hg **)xcalloc((size_t)cap, sizeof(orc_hg *));
    r->cmap = (int32_t **)xcalloc((size_t)cap, sizeof(int32_t *));
    r->match = (int32_t **)xcalloc((size_t)cap, sizeof(int32_t *));
    r->lev[0] = (orc_hg *)g0;
    r->nlev = 1;
    while (r->nlev - 1 < levels) {
        const orc_hg *f = r->lev[r->nlev - 1];
        int32_t *cm = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)(f->N > 0 ? f->N : 1));
        int32_t *mt = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)(f->N > 0 ? f->N : 1));
        orc_hg *c = orc_coarsen_ex(f, policy, merge, cm, mt);
        if (c->N == f->N) { orc_hg_free(c); free(cm); free(mt); break; }
        r->cmap[r->nlev - 1] = cm;
        r->match[r->nlev - 1] = mt;
        r->lev[r->nlev++] = c;
    }
    int64_t W = 0;
    for (int32_t v = 0; v < g0->N; v++) W += g0->nwt[v];
    r->limit = orc_limit_part(W, m0, m, e6);
    const int64_t limit1 = orc_limit_part(W, m - m0, m, e6);

    int32_t L = r->nlev - 1;
    uint8_t *side = (uint8_t *)xmalloc((size_t)(r->lev[L]->N > 0 ? r->lev[L]->N : 1));
    r->init_rounds = orc_initial_target(r->lev[L], side, m0, m);
    int status = ORC_OK;
    for (int32_t l = L; l >= 0; l--) {
        const orc_hg *g = r->lev[l];
        if (l < L) {
            uint8_t *fine = (uint8_t *)xmalloc((size_t)(g->N > 0 ? g->N : 1));
            for (int32_t v = 0; v < g->N; v++) fine[v] = side[r->cmap[l][v]];
            free(side);
            side = fine;
        }
        for (int32_t it = 0; it < iters; it++) orc_refine_iter(g, side);
        status = orc_rebalance2(g, side, r->limit, limit1, NULL);
    }
    r->side = side;
    r->status = status;
    return r;
}

int32_t orc_run_nlev(const orc_run *r) { return r->nlev; }
const orc_hg *orc_run_level(const orc_run *r, int32_t l) { return r->lev[l]; }
void orc_run_cmap(const orc_run *r, int32_t l, int32_t *out) {
    memcpy(out, r->cmap[l], sizeof(int32_t) * (size_t)r->lev[l]->N);
}
void orc_run_match(const orc_run *r, int32_t l, int32_t *out) {
    memcpy(out, r->match[l], sizeof(int32_t) * (size_t)r->lev[l]->N);
}
void orc_run_side(const orc_run *r, uint8_t *out) { memcpy(out, r->side, (size_t)r->lev[0]->N); }
int orc_run_status(const orc_run *r) { return r->status; }
int32_t orc_run_init_rounds(const orc_run *r) { return r->init_rounds; }
int64_t orc_run_limit(const orc_run *r) { return r->limit; }

void orc_run_free(orc_run *r) {
    if (!r) return;
    for (int32_t l = 1; l < r->nlev; l++) orc_hg_free(r->lev[l]);
    for (int32_t l = 0; l < r->nlev; l++) { free(r->cmap[l]); free(r->match[l]); }
    free(r->lev); free(r->cmap); free(r->match); free(r->side); free(r);
}

/* ------------------------------------------------------------------------------------------
 * Sec. 1.1 cut: sum over hyperedges of w_e * (lambda_e - 1), lambda_e = number of distinct parts
 * among e's pins (reading C17: over the hyperedges of the graph given).
 * ------------------------------------------------------------------------------------------ */
int64_t orc_cut(const orc_hg *g, const int32_t *part) {
    int64_t cut = 0;
    int32_t maxd = 0;
    for (int32_t e = 0; e < g->E; e++)
        if (g->off[e + 1] - g->off[e] > maxd) maxd = g->off[e + 1] - g->off[e];
    int32_t *buf = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)(maxd > 0 ? maxd : 1));
    for (int32_t e = 0; e < g->E; e++) {
        int32_t d = g->off[e + 1] - g->off[e];
        for (int32_t i = 0; i < d; i++) buf[i] = part[g->pin[g->off[e] + i]];
        int32_t lambda = sort_unique(buf, d);
        cut += (int64_t)g->hwt[e] * (lambda - 1);
    }
    free(buf);
    return cut;
}

/* Second way for a bisection: a hyperedge counts iff it has pins on both sides. */
int64_t orc_cut_bisection(const orc_hg *g, const uint8_t *side) {
    int64_t cut = 0;
    for (int32_t e = 0; e < g->E; e++) {
        int32_t n0 = 0, n1 = 0;
        for (int32_t i = g->off[e]; i < g->off[e + 1]; i++) {
            if (side[g->pin[i]]) n1++; else n0++;
        }
        if (n0 > 0 && n1 > 0) cut += g->hwt[e];
    }
    return cut;
}

/* ------------------------------------------------------------------------------------------
 * Reading C16: the subgraph of part j holds the nodes with part j, renumbered in ascending id,
 * and every hyperedge restricted to them that keeps at least 2 pins (net splitting), in
 * ascending hyperedge id, with weights carried.
 * ------------------------------------------------------------------------------------------ */
orc_hg *orc_subgraph(const orc_hg *g, const int32_t *part, int32_t j, int32_t *local_to_global) {
    int32_t *loc = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)(g->N > 0 ? g->N : 1));
    int32_t n = 0;
    for (int32_t v = 0; v < g->N; v++) {
        if (part[v] == j) { loc[v] = n; if (local_to_global) local_to_global[n] = v; n++; }
        else loc[v] = -1;
    }
    orc_hg *s = hg_alloc(n, g->E, g->off[g->E]);
    for (int32_t v = 0; v < g->N; v++) if (loc[v] >= 0) s->nwt[loc[v]] = g->nwt[v];
    int32_t ne = 0, np = 0;
    s->off[0] = 0;
    for (int32_t e = 0; e < g->E; e++) {
        int32_t m = 0;
        for (int32_t i = g->off[e]; i < g->off[e + 1]; i++) {
            int32_t v = g->pin[i];
            if (loc[v] >= 0) s->pin[np + m++] = loc[v];
        }
        if (m < 2) continue;
        np += m;
        s->hwt[ne] = g->hwt[e];
        s->off[++ne] = np;
    }
    s->E = ne;
    free(loc);
    return s;
}

/* ------------------------------------------------------------------------------------------
 * Algorithm 6 (nested k-way), sequentially, for any k >= 1 (readings C16, G1-G3).  A subgraph
 * that owns the m parts [lo, lo + m) is bisected with side 0 meant for m0 = ceil(m / 2) of them
 * (targets and limits in proportion, G2); its side-0 nodes own [lo, lo + m0), its side-1 nodes
 * [lo + m0, lo + m); a range of one part is final.  Subgraphs are built as in C16 and bisected
 * with the same policy, levels and iters, and with e6 millionths of imbalance (or, with
 * ORC_FLAG_ADAPTIVE, the per-bisection e6 of reading G3; ORC_FLAG_MERGE: reading M1).  For k a power of two this is the paper's
 * scheme: every split is in halves and the parts of a tree level are 2j, 2j + 1.  Returns
 * ORC_WARN_IMBALANCED if any bisection ended above its limit.
 * ------------------------------------------------------------------------------------------ */
int orc_partition_ex(const orc_hg *g, int32_t k, int64_t e6, int flags, int policy,
                     int32_t levels, int32_t iters, int32_t *part) {
    if (k < 1) return ORC_ERR_INVALID_ARG;
    const int64_t eb = (flags & ORC_FLAG_ADAPTIVE) ? orc_adaptive_e6(e6, k) : e6;
    const int merge = (flags & ORC_FLAG_MERGE) != 0;
    for (int32_t v = 0; v < g->N; v++) part[v] = 0;  /* every node in the range starting at 0 */
    int status = ORC_OK;
    int32_t *l2g = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)(g->N > 0 ? g->N : 1));
    /* ranges of the current tree level: (lo, m); nodes carry the lo of their range */
    int32_t *rlo = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)k);
    int32_t *rm = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)k);
    int32_t *nlo = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)k);
    int32_t *nm = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)k);
    int32_t nr = 1;
    rlo[0] = 0;
    rm[0] = k;
    while (nr > 0) {
        int32_t nn = 0;
        for (int32_t r = 0; r < nr; r++) {
            const int32_t lo = rlo[r], m = rm[r];
            if (m < 2) continue;
            const int32_t m0 = (m + 1) / 2;
            orc_hg *s = orc_subgraph(g, part, lo, l2g);
            orc_run *run = orc_bisect_ex(s, eb, m0, m, merge, policy, levels, iters);
            if (run->status != ORC_OK) status = run->status;
            for (int32_t i = 0; i < s->N; i++) part[l2g[i]] = run->side[i] ? lo + m0 : lo;
            orc_run_free(run);
            orc_hg_free(s);
            nlo[nn] = lo; nm[nn] = m0; nn++;
            nlo[nn] = lo + m0; nm[nn] = m - m0; nn++;
        }
        memcpy(rlo, nlo, sizeof(int32_t) * (size_t)nn);
        memcpy(rm, nm, sizeof(int32_t) * (size_t)nn);
        nr = nn;
    }
    free(l2g); free(rlo); free(rm); free(nlo); free(nm);
    return status;
}

int orc_partition(const orc_hg *g, int32_t k, double eps, int policy, int32_t levels,
                  int32_t iters, int32_t *part) {
    return orc_partition_ex(g, k, llround(eps * 1e6), 0, policy, levels, iters, part);
}
