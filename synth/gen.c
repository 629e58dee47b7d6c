/*
 * Seeded synthetic hypergraph generators.
 *
 * This module only draws inputs: it holds none of the partitioner's arithmetic and is shared,
 * as plain data, by the CPU oracle and the CUDA path.  Every draw comes from xoshiro256**
 * (Blackman and Vigna, "Scrambled linear pseudorandom number generators", 2018) seeded through
 * SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number generators", 2014),
 * both written from their published definitions.  Each hyperedge (and each node-weight block)
 * owns an independent stream derived from (seed, stream id), so degrees and pins can be drawn in
 * two separate passes and in parallel without changing the result.
 *
 * Workload shapes (see synth/__init__.py for the parameter sets):
 *   uniform  - hyperedge degree U{dmin..dmax}, pins uniform over [0, N) without replacement.
 *   netlist  - circuit-like: a share of degree-2 nets, a geometric tail, rare high-fanout nets;
 *              pins drawn without replacement inside a window around a random centre.
 *   rownet   - row-net model of a power-law sparse matrix: rows are hyperedges with Zipf lengths,
 *              columns are nodes, a fraction of pins lands in a small set of hub columns.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64_step(uint64_t *state) {
    uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t rng_next(rng_t *r) {
    uint64_t *s = r->s;
    uint64_t out = rotl64(s[1] * 5u, 7) * 9u;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return out;
}

/* Independent stream for (seed, stream id). */
static void rng_init(rng_t *r, uint64_t seed, uint64_t stream) {
    uint64_t sm = seed * 0x9E3779B97F4A7C15ull ^ (stream + 0x632BE59BD9B4E019ull) * 0xD1B54A32D192ED03ull;
    for (int i = 0; i < 4; i++) r->s[i] = splitmix64_step(&sm);
}

/* Uniform integer in [0, n), n >= 1 (multiply-high mapping of a 64-bit draw). */
static inline uint64_t rng_below(rng_t *r, uint64_t n) {
    return (uint64_t)(((unsigned __int128)rng_next(r) * n) >> 64);
}

/* Uniform double in [0, 1). */
static inline double rng_unit(rng_t *r) { return (double)(rng_next(r) >> 11) * 0x1.0p-53; }

/* ---------------------------------------------------------------- bitmap for distinct draws */
typedef struct { uint64_t *w; int64_t nbits; } bitset_t;

static int bs_init(bitset_t *b, int64_t nbits) {
    b->nbits = nbits;
    b->w = (uint64_t *)calloc((size_t)((nbits + 63) / 64 + 1), sizeof(uint64_t));
    return b->w != NULL;
}
static inline int bs_test_set(bitset_t *b, int64_t i) {
    uint64_t m = 1ull << (i & 63);
    int was = (b->w[i >> 6] & m) != 0;
    b->w[i >> 6] |= m;
    return was;
}
static inline void bs_clear(bitset_t *b, int64_t i) { b->w[i >> 6] &= ~(1ull << (i & 63)); }

/* ---------------------------------------------------------------- uniform workload */
/* Stream layout: stream e draws the degree, then the pins of hyperedge e. */
static int32_t uniform_degree(rng_t *r, int32_t dmin, int32_t dmax) {
    return dmin + (int32_t)rng_below(r, (uint64_t)(dmax - dmin + 1));
}

int synth_uniform_degrees(uint64_t seed, int32_t N, int32_t E, int32_t dmin, int32_t dmax, int32_t *deg) {
    if (N < 1 || E < 0 || dmin < 1 || dmax < dmin || dmax > N) return -1;
    #pragma omp parallel for schedule(static)
    for (int32_t e = 0; e < E; e++) {
        rng_t r; rng_init(&r, seed, (uint64_t)e);
        deg[e] = uniform_degree(&r, dmin, dmax);
    }
    return 0;
}

int synth_uniform_pins(uint64_t seed, int32_t N, int32_t E, int32_t dmin, int32_t dmax,
                       const int64_t *off, int32_t *pins) {
    if (N < 1 || E < 0 || dmin < 1 || dmax < dmin || dmax > N) return -1;
    int bad = 0;
    #pragma omp parallel reduction(|:bad)
    {
        int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)dmax);
        if (!tmp) bad = 1;
        #pragma omp for schedule(dynamic, 4096)
        for (int32_t e = 0; e < E; e++) {
            if (!tmp) continue;
            rng_t r; rng_init(&r, seed, (uint64_t)e);
            int32_t d = uniform_degree(&r, dmin, dmax);
            int32_t k = 0;
            while (k < d) {                       /* rejection: redraw a repeated pin */
                int32_t v = (int32_t)rng_below(&r, (uint64_t)N);
                int dup = 0;
                for (int32_t j = 0; j < k; j++) if (tmp[j] == v) { dup = 1; break; }
                if (!dup) tmp[k++] = v;
            }
            memcpy(pins + off[e], tmp, sizeof(int32_t) * (size_t)d);
        }
        free(tmp);
    }
    return bad ? -2 : 0;
}

/* ---------------------------------------------------------------- netlist workload */
/* Net classes by one uniform draw u: u < p_hi -> high fanout U{hi_lo..hi_hi};
 * u < p_hi + p2 -> degree 2; otherwise 3 + Geom(1/2) clipped to tail_cap. */
static int32_t netlist_degree(rng_t *r, double p2, double p_hi, int32_t hi_lo, int32_t hi_hi,
                              int32_t tail_cap) {
    double u = rng_unit(r);
    if (u < p_hi) return hi_lo + (int32_t)rng_below(r, (uint64_t)(hi_hi - hi_lo + 1));
    if (u < p_hi + p2) return 2;
    int32_t d = 3;
    while (d < tail_cap && (rng_next(r) >> 63)) d++;   /* fair coin: continue with prob 1/2 */
    return d;
}

static int netlist_check(int32_t N, double p2, double p_hi, int32_t hi_lo, int32_t hi_hi,
                         int32_t tail_cap, int32_t win) {
    if (N < 2 || p2 < 0 || p_hi < 0 || p2 + p_hi > 1.0) return 0;
    if (hi_lo < 2 || hi_hi < hi_lo || tail_cap < 3 || win < 1) return 0;
    if (hi_hi > N || tail_cap > N) return 0;
    return 1;
}

int synth_netlist_degrees(uint64_t seed, int32_t N, int32_t E, double p2, double p_hi,
                          int32_t hi_lo, int32_t hi_hi, int32_t tail_cap, int32_t win, int32_t *deg) {
    if (!netlist_check(N, p2, p_hi, hi_lo, hi_hi, tail_cap, win) || E < 0) return -1;
    #pragma omp parallel for schedule(static)
    for (int32_t e = 0; e < E; e++) {
        rng_t r; rng_init(&r, seed, (uint64_t)e);
        deg[e] = netlist_degree(&r, p2, p_hi, hi_lo, hi_hi, tail_cap);
    }
    return 0;
}

/* Pins of net e: centre c ~ U[0, N), half-width h = max(win, d), window [c-h, c+h] clipped to
 * [0, N-1]; d distinct pins uniform in the window (the window always holds >= d+1 ids). */
int synth_netlist_pins(uint64_t seed, int32_t N, int32_t E, double p2, double p_hi,
                       int32_t hi_lo, int32_t hi_hi, int32_t tail_cap, int32_t win,
                       const int64_t *off, int32_t *pins) {
    if (!netlist_check(N, p2, p_hi, hi_lo, hi_hi, tail_cap, win) || E < 0) return -1;
    int bad = 0;
    #pragma omp parallel reduction(|:bad)
    {
        bitset_t bs;
        int64_t span = 2 * (int64_t)(win > hi_hi ? win : hi_hi) + 2;
        if (!bs_init(&bs, span)) bad = 1;
        #pragma omp for schedule(dynamic, 2048)
        for (int32_t e = 0; e < E; e++) {
            if (bad) continue;
            rng_t r; rng_init(&r, seed, (uint64_t)e);
            int32_t d = netlist_degree(&r, p2, p_hi, hi_lo, hi_hi, tail_cap);
            int64_t c = (int64_t)rng_below(&r, (uint64_t)N);
            int64_t h = d > win ? d : win;
            int64_t lo = c - h < 0 ? 0 : c - h;
            int64_t hi = c + h > N - 1 ? N - 1 : c + h;
            uint64_t width = (uint64_t)(hi - lo + 1);
            int32_t *out = pins + off[e];
            for (int32_t k = 0; k < d;) {
                int64_t v = lo + (int64_t)rng_below(&r, width);
                if (!bs_test_set(&bs, v - lo)) out[k++] = (int32_t)v;
            }
            for (int32_t k = 0; k < d; k++) bs_clear(&bs, out[k] - lo);
        }
        free(bs.w);
    }
    return bad ? -2 : 0;
}

/* Node weights U{wmin..wmax}; stream (1<<40) + block of 65536 nodes. */
int synth_node_weights(uint64_t seed, int32_t N, int32_t wmin, int32_t wmax, int32_t *w) {
    if (N < 0 || wmin < 1 || wmax < wmin) return -1;
    int32_t nblk = (N + 65535) / 65536;
    #pragma omp parallel for schedule(static)
    for (int32_t b = 0; b < nblk; b++) {
        rng_t r; rng_init(&r, seed, (1ull << 40) + (uint64_t)b);
        int32_t end = (b + 1) * 65536 < N ? (b + 1) * 65536 : N;
        for (int32_t v = b * 65536; v < end; v++)
            w[v] = wmin + (int32_t)rng_below(&r, (uint64_t)(wmax - wmin + 1));
    }
    return 0;
}

/* ---------------------------------------------------------------- row-net workload */
/* Zipf(alpha) on the support [lo, hi], sampled by inverse CDF over a table built per call. */
typedef struct { double *cdf; int32_t lo, hi; } zipf_t;

static int zipf_init(zipf_t *z, double alpha, int32_t lo, int32_t hi) {
    z->lo = lo; z->hi = hi;
    int32_t n = hi - lo + 1;
    z->cdf = (double *)malloc(sizeof(double) * (size_t)n);
    if (!z->cdf) return 0;
    double acc = 0;
    for (int32_t i = 0; i < n; i++) { acc += pow((double)(lo + i), -alpha); z->cdf[i] = acc; }
    for (int32_t i = 0; i < n; i++) z->cdf[i] /= acc;
    z->cdf[n - 1] = 1.0;
    return 1;
}
static int32_t zipf_draw(const zipf_t *z, rng_t *r) {
    double u = rng_unit(r);
    int32_t a = 0, b = z->hi - z->lo;             /* first index with cdf > u */
    while (a < b) { int32_t m = a + (b - a) / 2; if (z->cdf[m] > u) b = m; else a = m + 1; }
    return z->lo + a;
}

/* Row length cap: at most half the columns (keeps distinct draws cheap on small instances). */
static int32_t rownet_cap(int32_t C, int32_t lmax) {
    int32_t c = C / 2;
    return lmax < c ? lmax : c;
}

int synth_rownet_degrees(uint64_t seed, int32_t R, int32_t C, double alpha, int32_t lmin,
                         int32_t lmax, int32_t *deg) {
    if (R < 0 || C < 4 || lmin < 2) return -1;
    int32_t cap = rownet_cap(C, lmax);
    if (cap < lmin) return -1;
    zipf_t z;
    if (!zipf_init(&z, alpha, lmin, cap)) return -2;
    #pragma omp parallel for schedule(static)
    for (int32_t e = 0; e < R; e++) {
        rng_t r; rng_init(&r, seed, (uint64_t)e);
        deg[e] = zipf_draw(&z, &r);
    }
    free(z.cdf);
    return 0;
}

/* Hub columns: the first max(1, C*hub_share) entries of a seeded Fisher-Yates permutation of
 * [0, C).  Each pin is a hub column with probability p_hub (while the row still has unused hubs,
 * at most half of them), otherwise a uniform column; repeats are redrawn in the same category. */
int synth_rownet_pins(uint64_t seed, int32_t R, int32_t C, double alpha, int32_t lmin,
                      int32_t lmax, double p_hub, double hub_share, const int64_t *off,
                      int32_t *pins) {
    if (R < 0 || C < 4 || lmin < 2) return -1;
    int32_t cap = rownet_cap(C, lmax);
    if (cap < lmin) return -1;
    zipf_t z;
    if (!zipf_init(&z, alpha, lmin, cap)) return -2;
    int32_t H = (int32_t)((double)C * hub_share);
    if (H < 1) H = 1;
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)C);
    if (!perm) { free(z.cdf); return -2; }
    for (int32_t i = 0; i < C; i++) perm[i] = i;
    {
        rng_t r; rng_init(&r, seed, 1ull << 41);
        for (int32_t i = 0; i < H; i++) {             /* partial Fisher-Yates: first H slots */
            int32_t j = i + (int32_t)rng_below(&r, (uint64_t)(C - i));
            int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
        }
    }
    int bad = 0;
    #pragma omp parallel reduction(|:bad)
    {
        bitset_t bs;
        if (!bs_init(&bs, C)) bad = 1;
        #pragma omp for schedule(dynamic, 1024)
        for (int32_t e = 0; e < R; e++) {
            if (bad) continue;
            rng_t r; rng_init(&r, seed, (uint64_t)e);
            int32_t d = zipf_draw(&z, &r);
            int32_t *out = pins + off[e];
            int32_t hubs_used = 0;
            for (int32_t k = 0; k < d;) {
                int hub = rng_unit(&r) < p_hub && hubs_used < H / 2;
                int32_t v;
                for (;;) {
                    v = hub ? perm[rng_below(&r, (uint64_t)H)] : (int32_t)rng_below(&r, (uint64_t)C);
                    if (!bs_test_set(&bs, v)) break;
                }
                out[k++] = v;
                hubs_used += hub;
            }
            for (int32_t k = 0; k < d; k++) bs_clear(&bs, out[k]);
        }
        free(bs.w);
    }
    free(perm);
    free(z.cdf);
    return bad ? -2 : 0;
}

/* Poisson-process arrival gaps and per-request draws for the serving workload. */
int synth_uniform01(uint64_t seed, uint64_t stream, int32_t n, double *out) {
    rng_t r; rng_init(&r, seed, stream);
    for (int32_t i = 0; i < n; i++) out[i] = rng_unit(&r);
    return 0;
}
