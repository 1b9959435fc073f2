/*
 * Seeded synthetic graph generators (inputs only).
 *
 * This module produces the undirected input graphs that both the CPU oracle and
 * the CUDA path consume.  It holds none of the Log(Graph) arithmetic (no widths,
 * no packing, no offsets); it only draws edges and builds a plain symmetric CSR
 * (row_ptr u64[n+1], col u32[arcs], sorted strictly increasing rows, no self
 * loops), which is the adjacency-array input of the paper's Section 2.3.
 *
 * Randomness is counter-based: every draw is SplitMix64 (Steele, Lea, Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014) applied to a
 * tuple (seed, stream, i, j) (R-MAT: to a per-edge key plus the level), so any
 * subset of edges can be regenerated independently and the result does not
 * depend on the thread count.
 *
 * Generators:
 *   - R-MAT / Kronecker (Chakrabarti et al. 2004; the Kronecker graphs of the
 *     paper's evaluation, "sX_eY"): M = ef * 2^scale edges, quadrant per level
 *     with probabilities (a, b, c, 1-a-b-c), then a seeded Fisher-Yates
 *     relabeling so hubs are not clustered at low IDs (Graph500 practice).
 *   - Community graph: blocks of B vertices, out-degree c*z with z ~ Zipf(s)
 *     truncated to {1..K}, each out-edge inside the own block with probability
 *     p_intra (never a self loop) else uniform over V, then a global seeded
 *     permutation.
 * Both are symmetrized (each undirected edge stored as two arcs), with self
 * loops dropped and duplicates removed.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define LGGEN_OK 0
#define LGGEN_EINVAL 1
#define LGGEN_ENOMEM 2

enum { ST_RMAT = 1, ST_PERM = 2, ST_WEIGHT = 3, ST_COMM = 4, ST_SRC = 5, ST_CPERM = 6 };

typedef struct {
    uint64_t n, arcs;
    uint64_t *row_ptr; /* n+1 */
    uint32_t *col;     /* arcs */
    uint32_t *w;       /* arcs or NULL */
} lggen_csr;

static inline uint64_t sm64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
static inline uint64_t h4(uint64_t seed, uint64_t stream, uint64_t i, uint64_t j) {
    return sm64(sm64(sm64(sm64(seed) ^ stream) ^ i) ^ j);
}
static inline double u01(uint64_t h) { return (double)(h >> 11) * (1.0 / 9007199254740992.0); }

/* Public: the raw counter-based draw, so the Python side can reproduce it. */
uint64_t lggen_hash(uint64_t seed, uint64_t stream, uint64_t i, uint64_t j) { return h4(seed, stream, i, j); }

static void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/* Seeded Fisher-Yates permutation of 0..n-1 (sequential by construction). */
static uint32_t *fisher_yates(uint64_t n, uint64_t seed, uint64_t stream) {
    uint32_t *p = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    if (!p) return NULL;
    for (uint64_t i = 0; i < n; i++) p[i] = (uint32_t)i;
    for (uint64_t i = n; i > 1; i--) {
        uint64_t j = h4(seed, stream, i - 1, 0) % i;
        uint32_t t = p[i - 1]; p[i - 1] = p[j]; p[j] = t;
    }
    return p;
}

/* ------------------------------------------------------------------ */
/* edge sources                                                        */
/* ------------------------------------------------------------------ */
typedef struct {
    int kind; /* 0 rmat, 1 community, 2 explicit */
    uint64_t n, m;
    uint64_t seed;
    /* rmat */
    int scale; double a, ab, abc;
    /* community */
    uint64_t block; double p_intra; const uint64_t *dprefix; /* n+1 out-degree prefix */
    /* explicit */
    const uint32_t *src, *dst;
    const uint32_t *perm; /* label permutation or NULL */
} edge_src;

/* Edge e draws one key h4(seed, RMAT, e, 0) and then one SplitMix64 output per
   two levels (32 uniform bits per level). */
static inline void rmat_edge(const edge_src *g, uint64_t e, uint32_t *u, uint32_t *v) {
    uint64_t s = 0, d = 0;
    const uint64_t key = h4(g->seed, ST_RMAT, e, 0);
    uint64_t h = 0;
    for (int k = 0; k < g->scale; k++) {
        if ((k & 1) == 0) h = sm64(key + (uint64_t)k);
        const uint32_t r32 = (k & 1) ? (uint32_t)h : (uint32_t)(h >> 32);
        double x = (double)r32 * (1.0 / 4294967296.0);
        uint64_t sb, db;
        if (x < g->a) { sb = 0; db = 0; }
        else if (x < g->ab) { sb = 0; db = 1; }
        else if (x < g->abc) { sb = 1; db = 0; }
        else { sb = 1; db = 1; }
        s = (s << 1) | sb; d = (d << 1) | db;
    }
    *u = (uint32_t)s; *v = (uint32_t)d;
}

/* community: edge j of vertex v */
static inline uint32_t comm_target(const edge_src *g, uint64_t v, uint64_t j) {
    double x = u01(h4(g->seed, ST_COMM, v, 2 * j + 1));
    uint64_t r = h4(g->seed, ST_COMM, v, 2 * j + 2);
    if (x < g->p_intra && g->block > 1) {
        uint64_t base = (v / g->block) * g->block;
        uint64_t bsz = g->block;
        if (base + bsz > g->n) bsz = g->n - base;
        if (bsz <= 1) return (uint32_t)v; /* a lone vertex: self loop, dropped */
        uint64_t t = base + (r % (bsz - 1));
        if (t >= v) t++;
        return (uint32_t)t;
    }
    return (uint32_t)(r % g->n);
}

/* ------------------------------------------------------------------ */
/* symmetric CSR builder (count, scatter, per-row sort + dedup)        */
/* ------------------------------------------------------------------ */
static void sort_u32(uint32_t *a, int64_t n) {
    /* iterative quicksort with insertion-sort cutoff */
    int64_t stack_lo[64], stack_hi[64];
    int sp = 0;
    stack_lo[sp] = 0; stack_hi[sp] = n - 1; sp++;
    while (sp > 0) {
        sp--;
        int64_t lo = stack_lo[sp], hi = stack_hi[sp];
        while (hi - lo > 24) {
            int64_t mid = lo + (hi - lo) / 2;
            uint32_t x = a[lo], y = a[mid], z = a[hi], piv;
            if (x < y) { piv = (y < z) ? y : ((x < z) ? z : x); }
            else { piv = (x < z) ? x : ((y < z) ? z : y); }
            int64_t i = lo, j = hi;
            while (i <= j) {
                while (a[i] < piv) i++;
                while (a[j] > piv) j--;
                if (i <= j) { uint32_t t = a[i]; a[i] = a[j]; a[j] = t; i++; j--; }
            }
            /* recurse into the smaller part, loop on the larger */
            if (j - lo < hi - i) {
                if (i < hi) { stack_lo[sp] = i; stack_hi[sp] = hi; sp++; }
                hi = j;
            } else {
                if (lo < j) { stack_lo[sp] = lo; stack_hi[sp] = j; sp++; }
                lo = i;
            }
        }
        for (int64_t i = lo + 1; i <= hi; i++) {
            uint32_t t = a[i]; int64_t k = i - 1;
            while (k >= lo && a[k] > t) { a[k + 1] = a[k]; k--; }
            a[k + 1] = t;
        }
    }
}

static inline void get_edge(const edge_src *g, uint64_t e, uint64_t v_hint, uint32_t *u, uint32_t *v) {
    if (g->kind == 0) rmat_edge(g, e, u, v);
    else if (g->kind == 1) { *u = (uint32_t)v_hint; *v = comm_target(g, v_hint, e); }
    else { *u = g->src[e]; *v = g->dst[e]; }
    if (g->perm) { *u = g->perm[*u]; *v = g->perm[*v]; }
}

/* Iterate all edges; community edges are enumerated per vertex. */
#define FOR_EACH_EDGE(g, U, V, ...)                                                   \
    do {                                                                               \
        if ((g)->kind == 1) {                                                          \
            _Pragma("omp parallel for schedule(dynamic, 4096)")                        \
            for (int64_t vv = 0; vv < (int64_t)(g)->n; vv++) {                        \
                for (uint64_t jj = (g)->dprefix[vv]; jj < (g)->dprefix[vv + 1]; jj++) {  \
                    uint32_t U, V;                                                     \
                    get_edge((g), jj - (g)->dprefix[vv], (uint64_t)vv, &U, &V);        \
                    __VA_ARGS__                                                        \
                }                                                                      \
            }                                                                          \
        } else {                                                                       \
            _Pragma("omp parallel for schedule(static, 65536)")                        \
            for (int64_t ee = 0; ee < (int64_t)(g)->m; ee++) {                        \
                uint32_t U, V;                                                         \
                get_edge((g), (uint64_t)ee, 0, &U, &V);                                \
                __VA_ARGS__                                                            \
            }                                                                          \
        }                                                                              \
    } while (0)

static int build_csr(const edge_src *g, int weighted, lggen_csr *out) {
    uint64_t n = g->n;
    uint64_t *cnt = (uint64_t *)calloc(n + 1, sizeof(uint64_t));
    if (!cnt) return LGGEN_ENOMEM;
    FOR_EACH_EDGE(g, u, v, {
        if (u != v) {
            __atomic_fetch_add(&cnt[u], 1, __ATOMIC_RELAXED);
            __atomic_fetch_add(&cnt[v], 1, __ATOMIC_RELAXED);
        }
    });
    uint64_t *rp = (uint64_t *)malloc(sizeof(uint64_t) * (n + 1));
    if (!rp) { free(cnt); return LGGEN_ENOMEM; }
    uint64_t acc = 0;
    for (uint64_t i = 0; i < n; i++) { rp[i] = acc; acc += cnt[i]; }
    rp[n] = acc;
    uint64_t total = acc;
    uint32_t *col = (uint32_t *)malloc(sizeof(uint32_t) * (total ? total : 1));
    if (!col) { free(cnt); free(rp); return LGGEN_ENOMEM; }
    for (uint64_t i = 0; i < n; i++) cnt[i] = rp[i];
    FOR_EACH_EDGE(g, u, v, {
        if (u != v) {
            uint64_t pu = __atomic_fetch_add(&cnt[u], 1, __ATOMIC_RELAXED);
            uint64_t pv = __atomic_fetch_add(&cnt[v], 1, __ATOMIC_RELAXED);
            col[pu] = v; col[pv] = u;
        }
    });
    /* sort + dedup each row; cnt[i] := new degree */
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < (int64_t)n; i++) {
        uint32_t *r = col + rp[i];
        int64_t d = (int64_t)(rp[i + 1] - rp[i]);
        if (d > 1) sort_u32(r, d);
        int64_t k = 0;
        for (int64_t j = 0; j < d; j++)
            if (k == 0 || r[j] != r[k - 1]) r[k++] = r[j];
        cnt[i] = (uint64_t)k;
    }
    /* compact in place (moves only left) */
    uint64_t w = 0;
    for (uint64_t i = 0; i < n; i++) {
        uint64_t s0 = rp[i], d = cnt[i];
        rp[i] = w;
        if (w != s0) memmove(col + w, col + s0, d * sizeof(uint32_t));
        w += d;
    }
    rp[n] = w;
    free(cnt);
    uint32_t *c2 = (uint32_t *)realloc(col, sizeof(uint32_t) * (w ? w : 1));
    if (c2) col = c2;
    out->n = n; out->arcs = w; out->row_ptr = rp; out->col = col; out->w = NULL;
    if (weighted) {
        uint32_t *wt = (uint32_t *)malloc(sizeof(uint32_t) * (w ? w : 1));
        if (!wt) { free(rp); free(col); return LGGEN_ENOMEM; }
#pragma omp parallel for schedule(dynamic, 4096)
        for (int64_t i = 0; i < (int64_t)n; i++) {
            for (uint64_t j = rp[i]; j < rp[i + 1]; j++) {
                uint64_t a = (uint64_t)i, b = col[j];
                uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
                wt[j] = 1u + (uint32_t)(h4(g->seed, ST_WEIGHT, lo, hi) % 255u);
            }
        }
        out->w = wt;
    }
    return LGGEN_OK;
}

/* ------------------------------------------------------------------ */
/* public generators                                                   */
/* ------------------------------------------------------------------ */
int lggen_rmat(int scale, int edge_factor, double a, double b, double c, uint64_t seed,
               int weighted, int permute, int nthreads, lggen_csr *out) {
    if (scale < 1 || scale > 31 || edge_factor < 1 || !out) return LGGEN_EINVAL;
    if (a < 0 || b < 0 || c < 0 || a + b + c > 1.0) return LGGEN_EINVAL;
    set_threads(nthreads);
    memset(out, 0, sizeof(*out));
    edge_src g;
    memset(&g, 0, sizeof(g));
    g.kind = 0; g.n = 1ULL << scale; g.m = (uint64_t)edge_factor << scale; g.seed = seed;
    g.scale = scale; g.a = a; g.ab = a + b; g.abc = a + b + c;
    uint32_t *perm = NULL;
    if (permute) { perm = fisher_yates(g.n, seed, ST_PERM); if (!perm) return LGGEN_ENOMEM; }
    g.perm = perm;
    int rc = build_csr(&g, weighted, out);
    free(perm);
    return rc;
}

int lggen_community(int log2n, int log2block, uint32_t zipf_kmax, double zipf_s, double mean_out,
                    double p_intra, uint64_t seed, int permute, int nthreads, lggen_csr *out) {
    if (log2n < 1 || log2n > 31 || log2block < 0 || log2block > log2n || zipf_kmax < 1 || !out)
        return LGGEN_EINVAL;
    set_threads(nthreads);
    memset(out, 0, sizeof(*out));
    uint64_t n = 1ULL << log2n;
    /* truncated Zipf(s) on {1..K}: cdf and the scale c that makes E[c z] = mean_out */
    double *cdf = (double *)malloc(sizeof(double) * zipf_kmax);
    if (!cdf) return LGGEN_ENOMEM;
    double hs = 0.0, h1 = 0.0;
    for (uint32_t k = 1; k <= zipf_kmax; k++) { hs += pow((double)k, -zipf_s); h1 += (double)k * pow((double)k, -zipf_s); }
    double accp = 0.0;
    for (uint32_t k = 1; k <= zipf_kmax; k++) { accp += pow((double)k, -zipf_s) / hs; cdf[k - 1] = accp; }
    cdf[zipf_kmax - 1] = 1.0;
    double cscale = mean_out / (h1 / hs);
    uint64_t *dp = (uint64_t *)malloc(sizeof(uint64_t) * (n + 1));
    if (!dp) { free(cdf); return LGGEN_ENOMEM; }
#pragma omp parallel for schedule(static, 65536)
    for (int64_t v = 0; v < (int64_t)n; v++) {
        double x = u01(h4(seed, ST_COMM, (uint64_t)v, 0));
        uint32_t lo = 0, hi = zipf_kmax - 1;
        while (lo < hi) { uint32_t mid = (lo + hi) / 2; if (cdf[mid] < x) lo = mid + 1; else hi = mid; }
        double z = (double)(lo + 1);
        int64_t d = llround(cscale * z);
        if (d < 1) d = 1;
        dp[v] = (uint64_t)d;
    }
    uint64_t acc = 0;
    for (uint64_t v = 0; v < n; v++) { uint64_t d = dp[v]; dp[v] = acc; acc += d; }
    dp[n] = acc;
    free(cdf);
    edge_src g;
    memset(&g, 0, sizeof(g));
    g.kind = 1; g.n = n; g.m = acc; g.seed = seed; g.block = 1ULL << log2block;
    g.p_intra = p_intra; g.dprefix = dp;
    uint32_t *perm = NULL;
    if (permute) { perm = fisher_yates(n, seed, ST_CPERM); if (!perm) { free(dp); return LGGEN_ENOMEM; } }
    g.perm = perm;
    int rc = build_csr(&g, 0, out);
    free(perm);
    free(dp);
    return rc;
}

/* The label permutation lggen_rmat applies (for the GPU edge generator). */
int lggen_rmat_perm(int scale, uint64_t seed, uint32_t *out) {
    if (scale < 1 || scale > 31 || !out) return LGGEN_EINVAL;
    uint32_t *p = fisher_yates(1ULL << scale, seed, ST_PERM);
    if (!p) return LGGEN_ENOMEM;
    memcpy(out, p, sizeof(uint32_t) << scale);
    free(p);
    return LGGEN_OK;
}

/* Explicit edge list -> symmetric CSR (tests and small fixtures). */
int lggen_from_edges(uint64_t n, uint64_t m, const uint32_t *src, const uint32_t *dst, int weighted,
                     uint64_t seed, lggen_csr *out) {
    if (!out || (m && (!src || !dst))) return LGGEN_EINVAL;
    for (uint64_t e = 0; e < m; e++) if (src[e] >= n || dst[e] >= n) return LGGEN_EINVAL;
    memset(out, 0, sizeof(*out));
    edge_src g;
    memset(&g, 0, sizeof(g));
    g.kind = 2; g.n = n; g.m = m; g.src = src; g.dst = dst; g.seed = seed;
    return build_csr(&g, weighted, out);
}

/* S distinct sources, uniform over vertices with nonzero degree (Graph500 style). */
int lggen_sources(uint64_t n, const uint64_t *row_ptr, uint32_t S, uint64_t seed, uint32_t *out) {
    uint64_t nz = 0;
    for (uint64_t v = 0; v < n; v++) nz += (row_ptr[v + 1] > row_ptr[v]);
    if (S > nz) return LGGEN_EINVAL;
    for (uint32_t k = 0; k < S; k++) {
        for (uint64_t t = 0;; t++) {
            uint64_t v = h4(seed, ST_SRC, k, t) % n;
            if (row_ptr[v + 1] == row_ptr[v]) continue;
            int dup = 0;
            for (uint32_t q = 0; q < k; q++) if (out[q] == v) { dup = 1; break; }
            if (dup) continue;
            out[k] = (uint32_t)v;
            break;
        }
    }
    return LGGEN_OK;
}

void lggen_free(lggen_csr *g) {
    if (!g) return;
    free(g->row_ptr); free(g->col); free(g->w);
    g->row_ptr = NULL; g->col = NULL; g->w = NULL;
}
