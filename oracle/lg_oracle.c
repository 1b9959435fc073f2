/*
 * CPU oracle for the Log(Graph) hot path -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load this code.  The product path (the CUDA library) never calls it and shares
 * no code, header, table or helper with it.
 *
 * Everything here is the plain, slow, obviously correct definition, written from
 * the paper (Besta et al., "Log(Graph): A Near-Optimal High-Performance Graph
 * Representation", PACT'18, full version arXiv:2010.15879):
 *
 *   - Section 3.2.1 (global vertex IDs): every ID in ceil(log n) bits, so
 *     |A| = 2m ceil(log n).
 *   - Section 3.2.2 (local vertex IDs): neighborhood v uses ceil(log maxN_v)
 *     bits plus a fixed-size field holding that width.
 *   - Section 3.3 (edge weights): ceil(log maxW) bits stored right after each ID.
 *   - Section 3.4 (single offsets): each offset in ceil(log 2m) bits.
 *   - Section 3.6 (fixed-size gap encoding): the largest difference between
 *     consecutive neighbors sets the width of all differences of that
 *     neighborhood.
 *   - Section 3.7.2 (bitwise access, Listing 2): field i of v starts at bit
 *     s * (O[v] + i); a field is read from a little-endian word by shifting right
 *     and masking, i.e. bit k of the value is stream bit p + k.
 *   - Section 4.3 (bvSD): the offsets as the positions of ones of a sparse bit
 *     vector stored with Elias-Fano (Elias 1974, Fano 1971; Okanohara-Sadakane
 *     2007), select(j) = the j-th one = the start of A_j (Section 4.1).
 *   - Section 5.6 (DM permuter): a higher degree gives a smaller label.
 *   - Section 3.2.2, Listing 1 (greedy relabeling for local IDs): vertices by
 *     increasing degree hand out the smallest free labels to their neighbors.
 *   - Section 7.1.2: BFS (depth per vertex), PageRank without atomics, and
 *     SSSP (shortest-path distances; computed here by Dijkstra).
 *
 * Readings of silent or ambiguous points (the CUDA path follows the same ones):
 *   IDs are 0-based; bits(x) = 0 for x = 0, else floor(log2 x) + 1, so
 *   ceil(log2 n) = bits(n - 1) for n >= 2 and a stored value x needs bits(x)
 *   bits (this differs from ceil(log2 x) only when x is a power of two).
 *   s = max(1, bits(n-1)); omega = max(1, bits(maxW)) unless given;
 *   H = bits(s) is the fixed width of the per-neighborhood width field, stored
 *   at the start of each neighborhood; w_v = 0 iff d_v = 0, else
 *   max(1, bits(maxN_v)); in gap mode the first neighbor is stored at s bits and
 *   the differences N_i - N_{i-1} (>= 1) at g_v = max(1, bits(max difference))
 *   bits, g_v = 0 iff d_v <= 1; offsets count records in the global mode and
 *   bits in the local modes; Elias-Fano over x_0..x_n with N = n+1,
 *   U = x_n, l = floor(log2(floor(U/N))) (0 if U < N), high vector of
 *   N + (U >> l) + 1 bits with bit (x_i >> l) + i set, select samples
 *   S[k] = position of one number k*sample; DM orders by (degree desc, ID asc).
 *   Every stream is u64 words, zero padded to an even word count, followed by
 *   four zero guard words.
 *
 * Parity unpinned: none -- every function below is pinned by the test suite
 * (closed forms, hand-derived bitstreams, round trips, brute force, linear
 * algebra); see the tests for the list.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_EUNSUPPORTED 6

enum { ORC_ID_GLOBAL = 0, ORC_ID_LOCAL = 1, ORC_ID_LOCAL_GAP = 2 };
enum { ORC_OFF_PACKED = 0, ORC_OFF_EF = 1 };

typedef struct {
    uint64_t n, arcs;
    uint32_t id_mode, off_mode, relabel, sample, weighted;
    uint32_t s, H, omega, r, w_O, ef_l;
    uint64_t bits_A, bits_O, ef_N, ef_U, ef_low_bits, ef_high_bits, n_samples;
    uint64_t words_A, words_O, words_ef_low, words_ef_high, words_samples;
    /* host arrays owned by the handle (NULL when unused) */
    uint64_t *A, *O, *ef_low, *ef_high, *samples;
    uint32_t *perm, *inv_perm; /* perm[original] = new label; inv_perm[new] = original */
    uint64_t *x;               /* decoded offsets x_0..x_n, kept for reference */
} orc_graph;

/* ------------------------------------------------------------------ */
/* bit helpers, one bit at a time                                      */
/* ------------------------------------------------------------------ */
uint32_t orc_bits(uint64_t x) {
    uint32_t b = 0;
    while (x) { b++; x >>= 1; }
    return b;
}

static void put(uint64_t *stream, uint64_t p, uint32_t w, uint64_t value) {
    for (uint32_t k = 0; k < w; k++) {
        if ((value >> k) & 1ULL) {
            uint64_t q = p + k;
            stream[q / 64] |= (1ULL << (q % 64));
        }
    }
}

static uint64_t get(const uint64_t *stream, uint64_t p, uint32_t w) {
    uint64_t v = 0;
    for (uint32_t k = 0; k < w; k++) {
        uint64_t q = p + k;
        if ((stream[q / 64] >> (q % 64)) & 1ULL) v |= (1ULL << k);
    }
    return v;
}

/* data words for `bits` bits, padded to an even count, plus four zero guard words */
static uint64_t padded_words(uint64_t bits) {
    uint64_t w = (bits + 63) / 64;
    w += (w & 1);
    return w + 4;
}

static uint64_t *zalloc_words(uint64_t words) {
    return (uint64_t *)calloc(words ? words : 1, sizeof(uint64_t));
}

/* ------------------------------------------------------------------ */
/* DM permuter (Section 5.6): order by degree descending, ID ascending  */
/* ------------------------------------------------------------------ */
static const uint64_t *g_deg_for_cmp;
static int cmp_dm(const void *a, const void *b) {
    uint32_t u = *(const uint32_t *)a, v = *(const uint32_t *)b;
    uint64_t du = g_deg_for_cmp[u], dv = g_deg_for_cmp[v];
    if (du != dv) return du > dv ? -1 : 1;
    return (u > v) - (u < v);
}
static int cmp_u32(const void *a, const void *b) {
    uint32_t u = *(const uint32_t *)a, v = *(const uint32_t *)b;
    return (u > v) - (u < v);
}
typedef struct { uint32_t id, w; } idw;
static int cmp_idw(const void *a, const void *b) {
    uint32_t u = ((const idw *)a)->id, v = ((const idw *)b)->id;
    return (u > v) - (u < v);
}

/* Greedy relabeling heuristic for local IDs (Listing 1, Section 3.2.2):
   vertices taken by increasing degree (ties by ID), each giving the next new
   labels to those of its neighbors (in row order) that have none yet; the
   vertices never reached get the remaining labels in ID order.  Labels start
   at 0 and every vertex of the sorted order is visited (the listing's loops
   start at 1 and its last loop names the wrong variable; read as intended). */
static int cmp_deg_asc(const void *a, const void *b) {
    uint32_t u = *(const uint32_t *)a, v = *(const uint32_t *)b;
    uint64_t du = g_deg_for_cmp[u], dv = g_deg_for_cmp[v];
    if (du != dv) return du < dv ? -1 : 1;
    return (u > v) - (u < v);
}

static void greedy_perm(uint64_t n, const uint64_t *rp, const uint32_t *col, const uint64_t *deg,
                        uint32_t *perm, uint32_t *inv, unsigned char *visit) {
    uint32_t *id = inv; /* the sorted order, overwritten by the inverse at the end */
    for (uint64_t v = 0; v < n; v++) { id[v] = (uint32_t)v; visit[v] = 0; }
    g_deg_for_cmp = deg;
    qsort(id, n, sizeof(uint32_t), cmp_deg_asc);
    uint32_t nl = 0;
    for (uint64_t i = 0; i < n; i++) {
        uint32_t v = id[i];
        for (uint64_t j = rp[v]; j < rp[v + 1]; j++) {
            uint32_t u = col[j];
            if (!visit[u]) { perm[u] = nl++; visit[u] = 1; }
        }
    }
    for (uint64_t v = 0; v < n; v++)
        if (!visit[v]) { perm[v] = nl++; visit[v] = 1; }
    for (uint64_t v = 0; v < n; v++) inv[perm[v]] = (uint32_t)v;
}

/* Builds the relabeled CSR: row P(v) = sorted { P(u) : u in N_v }, with P
   the DM order (relabel = 1) or the greedy heuristic (relabel = 2). */
static int dm_relabel(uint64_t n, const uint64_t *rp, const uint32_t *col, const uint32_t *w, uint32_t relabel,
                      uint32_t *perm, uint32_t *inv, uint64_t *nrp, uint32_t *ncol, uint32_t *nw) {
    uint64_t *deg = (uint64_t *)malloc(sizeof(uint64_t) * (n ? n : 1));
    if (!deg) return ORC_ENOMEM;
    for (uint64_t v = 0; v < n; v++) { deg[v] = rp[v + 1] - rp[v]; inv[v] = (uint32_t)v; }
    if (relabel == 2) {
        unsigned char *visit = (unsigned char *)malloc(n ? n : 1);
        if (!visit) { free(deg); return ORC_ENOMEM; }
        greedy_perm(n, rp, col, deg, perm, inv, visit);
        free(visit);
    } else {
        g_deg_for_cmp = deg;
        qsort(inv, n, sizeof(uint32_t), cmp_dm);
        for (uint64_t i = 0; i < n; i++) perm[inv[i]] = (uint32_t)i;
    }
    nrp[0] = 0;
    for (uint64_t i = 0; i < n; i++) nrp[i + 1] = nrp[i] + deg[inv[i]];
    idw *tmp = NULL;
    if (w) {
        uint64_t mx = 1;
        for (uint64_t v = 0; v < n; v++) if (deg[v] > mx) mx = deg[v];
        tmp = (idw *)malloc(sizeof(idw) * mx);
        if (!tmp) { free(deg); return ORC_ENOMEM; }
    }
    for (uint64_t i = 0; i < n; i++) {
        uint32_t v = inv[i];
        uint64_t d = deg[v], o = nrp[i];
        if (w) {
            for (uint64_t k = 0; k < d; k++) { tmp[k].id = perm[col[rp[v] + k]]; tmp[k].w = w[rp[v] + k]; }
            qsort(tmp, d, sizeof(idw), cmp_idw);
            for (uint64_t k = 0; k < d; k++) { ncol[o + k] = tmp[k].id; nw[o + k] = tmp[k].w; }
        } else {
            for (uint64_t k = 0; k < d; k++) ncol[o + k] = perm[col[rp[v] + k]];
            qsort(ncol + o, d, sizeof(uint32_t), cmp_u32);
        }
    }
    free(tmp);
    free(deg);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* encoder                                                             */
/* ------------------------------------------------------------------ */
static int valid_csr(uint64_t n, uint64_t arcs, const uint64_t *rp, const uint32_t *col) {
    if (rp[0] != 0 || rp[n] != arcs) return 0;
    for (uint64_t v = 0; v < n; v++) {
        if (rp[v + 1] < rp[v]) return 0;
        for (uint64_t j = rp[v]; j < rp[v + 1]; j++) {
            if (col[j] >= n) return 0;
            if (j > rp[v] && col[j] <= col[j - 1]) return 0;
        }
    }
    return 1;
}

void orc_free(orc_graph *g) {
    if (!g) return;
    free(g->A); free(g->O); free(g->ef_low); free(g->ef_high); free(g->samples);
    free(g->perm); free(g->inv_perm); free(g->x);
    free(g);
}

int orc_encode(uint64_t n, uint64_t arcs, const uint64_t *row_ptr, const uint32_t *col,
               const uint32_t *weights, uint32_t id_mode, uint32_t off_mode, uint32_t relabel,
               uint32_t sample, uint32_t weight_bits, orc_graph **out) {
    if (!out || n == 0 || n > 0xFFFFFFFFULL || !row_ptr || (arcs && !col)) return ORC_EINVAL;
    if (id_mode > ORC_ID_LOCAL_GAP || off_mode > ORC_OFF_EF) return ORC_EINVAL;
    if (weights && id_mode != ORC_ID_GLOBAL) return ORC_EUNSUPPORTED;
    if (off_mode == ORC_OFF_EF && (sample == 0 || (sample & (sample - 1)))) return ORC_EINVAL;
    if (!valid_csr(n, arcs, row_ptr, col)) return ORC_EINVAL;
    *out = NULL;
    orc_graph *g = (orc_graph *)calloc(1, sizeof(orc_graph));
    if (!g) return ORC_ENOMEM;
    g->n = n; g->arcs = arcs; g->id_mode = id_mode; g->off_mode = off_mode;
    if (relabel > 2) { free(g); return ORC_EINVAL; }
    g->relabel = relabel; g->sample = sample; g->weighted = weights ? 1 : 0;

    /* optional DM relabel */
    const uint64_t *rp = row_ptr;
    const uint32_t *cl = col, *wt = weights;
    uint64_t *nrp = NULL; uint32_t *ncol = NULL, *nw = NULL;
    if (g->relabel) {
        g->perm = (uint32_t *)malloc(sizeof(uint32_t) * n);
        g->inv_perm = (uint32_t *)malloc(sizeof(uint32_t) * n);
        nrp = (uint64_t *)malloc(sizeof(uint64_t) * (n + 1));
        ncol = (uint32_t *)malloc(sizeof(uint32_t) * (arcs ? arcs : 1));
        if (weights) nw = (uint32_t *)malloc(sizeof(uint32_t) * (arcs ? arcs : 1));
        if (!g->perm || !g->inv_perm || !nrp || !ncol || (weights && !nw)) goto nomem;
        if (dm_relabel(n, row_ptr, col, weights, relabel, g->perm, g->inv_perm, nrp, ncol, nw) != ORC_OK) goto nomem;
        rp = nrp; cl = ncol; wt = nw;
    }

    /* widths (Sections 3.2-3.4) */
    g->s = orc_bits(n - 1); if (g->s < 1) g->s = 1;
    g->H = orc_bits(g->s);
    g->omega = 0;
    if (wt) {
        uint64_t maxw = 0;
        for (uint64_t j = 0; j < arcs; j++) if (wt[j] > maxw) maxw = wt[j];
        if (weight_bits) {
            if (weight_bits > 32 || (weight_bits < 32 && maxw >> weight_bits)) goto inval;
            g->omega = weight_bits;
        } else {
            g->omega = orc_bits(maxw); if (g->omega < 1) g->omega = 1;
        }
    }
    g->r = g->s + g->omega;

    /* per-vertex lengths and offsets x_v */
    g->x = (uint64_t *)malloc(sizeof(uint64_t) * (n + 1));
    if (!g->x) goto nomem;
    g->x[0] = 0;
    for (uint64_t v = 0; v < n; v++) {
        uint64_t d = rp[v + 1] - rp[v], len;
        if (id_mode == ORC_ID_GLOBAL) {
            len = d; /* offsets count records */
        } else if (id_mode == ORC_ID_LOCAL) {
            uint32_t wv = 0;
            if (d > 0) { wv = orc_bits(cl[rp[v + 1] - 1]); if (wv < 1) wv = 1; }
            len = g->H + d * wv;
        } else {
            uint32_t gv = 0;
            if (d >= 2) {
                uint64_t mg = 0;
                for (uint64_t j = rp[v] + 1; j < rp[v + 1]; j++)
                    if ((uint64_t)(cl[j] - cl[j - 1]) > mg) mg = cl[j] - cl[j - 1];
                gv = orc_bits(mg); if (gv < 1) gv = 1;
            }
            len = g->H + (d >= 1 ? g->s : 0) + (d >= 2 ? (d - 1) * gv : 0);
        }
        g->x[v + 1] = g->x[v] + len;
    }
    g->bits_A = (id_mode == ORC_ID_GLOBAL) ? arcs * g->r : g->x[n];

    /* A stream (Listing 2 bit order) */
    g->words_A = padded_words(g->bits_A);
    g->A = zalloc_words(g->words_A);
    if (!g->A) goto nomem;
    for (uint64_t v = 0; v < n; v++) {
        uint64_t d = rp[v + 1] - rp[v];
        if (id_mode == ORC_ID_GLOBAL) {
            for (uint64_t i = 0; i < d; i++) {
                uint64_t p = (g->x[v] + i) * g->r;
                put(g->A, p, g->s, cl[rp[v] + i]);
                if (wt) put(g->A, p + g->s, g->omega, wt[rp[v] + i]);
            }
        } else if (id_mode == ORC_ID_LOCAL) {
            uint32_t wv = 0;
            if (d > 0) { wv = orc_bits(cl[rp[v + 1] - 1]); if (wv < 1) wv = 1; }
            uint64_t p = g->x[v];
            put(g->A, p, g->H, wv); p += g->H;
            for (uint64_t i = 0; i < d; i++) { put(g->A, p, wv, cl[rp[v] + i]); p += wv; }
        } else {
            uint32_t gv = 0;
            if (d >= 2) {
                uint64_t mg = 0;
                for (uint64_t j = rp[v] + 1; j < rp[v + 1]; j++)
                    if ((uint64_t)(cl[j] - cl[j - 1]) > mg) mg = cl[j] - cl[j - 1];
                gv = orc_bits(mg); if (gv < 1) gv = 1;
            }
            uint64_t p = g->x[v];
            put(g->A, p, g->H, gv); p += g->H;
            if (d >= 1) { put(g->A, p, g->s, cl[rp[v]]); p += g->s; }
            for (uint64_t i = 1; i < d; i++) {
                put(g->A, p, gv, (uint64_t)(cl[rp[v] + i] - cl[rp[v] + i - 1]));
                p += gv;
            }
        }
    }

    /* offset structure */
    if (off_mode == ORC_OFF_PACKED) {
        g->w_O = orc_bits(g->x[n]); if (g->w_O < 1) g->w_O = 1;
        g->bits_O = (n + 1) * (uint64_t)g->w_O;
        g->words_O = padded_words(g->bits_O);
        g->O = zalloc_words(g->words_O);
        if (!g->O) goto nomem;
        for (uint64_t v = 0; v <= n; v++) put(g->O, v * g->w_O, g->w_O, g->x[v]);
    } else {
        uint64_t N = n + 1, U = g->x[n], q = U / N;
        g->ef_N = N; g->ef_U = U;
        g->ef_l = q ? orc_bits(q) - 1 : 0;
        g->ef_low_bits = N * (uint64_t)g->ef_l;
        g->ef_high_bits = N + (U >> g->ef_l) + 1;
        g->n_samples = (N + sample - 1) / sample;
        g->words_ef_low = padded_words(g->ef_low_bits);
        g->words_ef_high = padded_words(g->ef_high_bits);
        g->words_samples = padded_words(64 * g->n_samples);
        g->ef_low = zalloc_words(g->words_ef_low);
        g->ef_high = zalloc_words(g->words_ef_high);
        g->samples = zalloc_words(g->words_samples);
        if (!g->ef_low || !g->ef_high || !g->samples) goto nomem;
        uint64_t lowmask = g->ef_l ? ((g->ef_l == 64) ? ~0ULL : ((1ULL << g->ef_l) - 1)) : 0;
        for (uint64_t i = 0; i < N; i++) {
            if (g->ef_l) put(g->ef_low, i * g->ef_l, g->ef_l, g->x[i] & lowmask);
            put(g->ef_high, (g->x[i] >> g->ef_l) + i, 1, 1);
        }
        for (uint64_t k = 0; k < g->n_samples; k++)
            g->samples[k] = (g->x[k * sample] >> g->ef_l) + k * sample;
        g->bits_O = g->ef_low_bits + g->ef_high_bits + 64 * g->n_samples;
    }
    free(nrp); free(ncol); free(nw);
    *out = g;
    return ORC_OK;
nomem:
    free(nrp); free(ncol); free(nw);
    orc_free(g);
    return ORC_ENOMEM;
inval:
    free(nrp); free(ncol); free(nw);
    orc_free(g);
    return ORC_EINVAL;
}

/* ------------------------------------------------------------------ */
/* pieces of the encoder for graphs too large to encode whole          */
/* ------------------------------------------------------------------ */

/* The Elias-Fano arrays of x_0..x_{N-1} (Section 4.3), laid out exactly as
   orc_encode lays them out, into caller buffers of orc_ef_words() words. */
void orc_ef_words(uint64_t N, uint64_t U, uint32_t sample, uint64_t *low_words, uint64_t *high_words,
                  uint64_t *sample_words, uint32_t *l_out) {
    uint64_t q = N ? U / N : 0;
    uint32_t l = q ? orc_bits(q) - 1 : 0;
    *l_out = l;
    *low_words = padded_words(N * (uint64_t)l);
    *high_words = padded_words(N + (U >> l) + 1);
    *sample_words = padded_words(64 * ((N + sample - 1) / sample));
}

int orc_ef_build(uint64_t N, const uint64_t *x, uint32_t sample, uint64_t *low, uint64_t *high, uint64_t *samples) {
    if (N == 0 || sample == 0) return ORC_EINVAL;
    uint64_t U = x[N - 1], lw, hw, sw;
    uint32_t l;
    orc_ef_words(N, U, sample, &lw, &hw, &sw, &l);
    memset(low, 0, lw * 8); memset(high, 0, hw * 8); memset(samples, 0, sw * 8);
    uint64_t lowmask = l ? ((1ULL << l) - 1) : 0;
    for (uint64_t i = 0; i < N; i++) {
        if (l) put(low, i * l, l, x[i] & lowmask);
        put(high, (x[i] >> l) + i, 1, 1);
    }
    for (uint64_t k = 0; k * sample < N; k++) samples[k] = (x[k * sample] >> l) + k * sample;
    return ORC_OK;
}

/* Words [w0, w1) of the global-ID A stream (Sections 3.2.1 and 3.3): record j
   = [col_j : s][w_j : omega] at bit j (s + omega), one bit at a time. */
int orc_global_words(uint64_t arcs, const uint32_t *col, const uint32_t *w, uint32_t s, uint32_t omega,
                     uint64_t w0, uint64_t w1, uint64_t *out) {
    uint32_t r = s + omega;
    if (r == 0 || w1 < w0) return ORC_EINVAL;
    memset(out, 0, (w1 - w0) * 8);
    uint64_t b0 = w0 * 64, b1 = w1 * 64;
    uint64_t j0 = b0 / r, j1 = (b1 + r - 1) / r;
    if (j1 > arcs) j1 = arcs;
    for (uint64_t j = j0; j < j1; j++) {
        uint64_t rec = (uint64_t)col[j] | (w ? (uint64_t)w[j] << s : 0);
        for (uint32_t k = 0; k < r; k++) {
            uint64_t p = j * r + k;
            if (p >= b0 && p < b1 && ((rec >> k) & 1ULL)) out[(p - b0) / 64] |= 1ULL << ((p - b0) % 64);
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* decoder                                                             */
/* ------------------------------------------------------------------ */

/* select(j): position of the j-th one (0-based) of the high vector, by a plain
   linear scan of the bits from position 0 (the definition, Section 2.3.2). */
uint64_t orc_ef_select_linear(const orc_graph *g, uint64_t j) {
    uint64_t seen = 0;
    for (uint64_t p = 0; p < g->ef_high_bits; p++) {
        if (get(g->ef_high, p, 1)) {
            if (seen == j) return p;
            seen++;
        }
    }
    return UINT64_MAX;
}

/* select(j) starting from the stored sample S[j / sample] (the position of one
   number (j / sample) * sample), then the same bit-by-bit scan. */
uint64_t orc_ef_select(const orc_graph *g, uint64_t j) {
    uint64_t k = j / g->sample;
    uint64_t seen = k * g->sample;
    for (uint64_t p = g->samples[k]; p < g->ef_high_bits; p++) {
        if (get(g->ef_high, p, 1)) {
            if (seen == j) return p;
            seen++;
        }
    }
    return UINT64_MAX;
}

/* x_v read back from the offset structure (O[v] in Listing 2, select_O(v) in Section 4.1). */
uint64_t orc_offset(const orc_graph *g, uint64_t v) {
    if (g->off_mode == ORC_OFF_PACKED) return get(g->O, v * g->w_O, g->w_O);
    uint64_t hi = orc_ef_select(g, v) - v;
    uint64_t lo = g->ef_l ? get(g->ef_low, v * g->ef_l, g->ef_l) : 0;
    return (hi << g->ef_l) | lo;
}

/* d_v from consecutive offsets and the neighborhood header (Section 3.7.3). */
uint64_t orc_degree(const orc_graph *g, uint64_t v) {
    uint64_t a = orc_offset(g, v), b = orc_offset(g, v + 1);
    if (g->id_mode == ORC_ID_GLOBAL) return b - a;
    uint64_t len = b - a;
    uint64_t w = get(g->A, a, g->H);
    if (g->id_mode == ORC_ID_LOCAL) return w ? (len - g->H) / w : 0;
    if (len == g->H) return 0;
    if (w == 0) return 1;
    return 1 + (len - g->H - g->s) / w;
}

/* Decodes N_v of the stored (possibly relabeled) vertex v into ids/wts, in
   stored order and stored labels.  Returns the degree, or UINT64_MAX when cap
   is too small. */
uint64_t orc_decode_raw(const orc_graph *g, uint64_t v, uint32_t *ids, uint32_t *wts, uint64_t cap) {
    uint64_t d = orc_degree(g, v);
    if (d > cap) return UINT64_MAX;
    uint64_t a = orc_offset(g, v);
    if (g->id_mode == ORC_ID_GLOBAL) {
        for (uint64_t i = 0; i < d; i++) {
            uint64_t p = (a + i) * g->r;
            ids[i] = (uint32_t)get(g->A, p, g->s);
            if (wts) wts[i] = g->omega ? (uint32_t)get(g->A, p + g->s, g->omega) : 0;
        }
    } else if (g->id_mode == ORC_ID_LOCAL) {
        uint32_t w = (uint32_t)get(g->A, a, g->H);
        for (uint64_t i = 0; i < d; i++) ids[i] = (uint32_t)get(g->A, a + g->H + i * w, w);
    } else {
        uint32_t w = (uint32_t)get(g->A, a, g->H);
        if (d >= 1) ids[0] = (uint32_t)get(g->A, a + g->H, g->s);
        for (uint64_t i = 1; i < d; i++)
            ids[i] = ids[i - 1] + (uint32_t)get(g->A, a + g->H + g->s + (i - 1) * w, w);
    }
    return d;
}

/* N_v for an ORIGINAL vertex id, as original ids sorted ascending (weights follow). */
uint64_t orc_neighbors(const orc_graph *g, uint64_t v, uint32_t *ids, uint32_t *wts, uint64_t cap) {
    uint64_t sv = g->relabel ? g->perm[v] : v;
    uint64_t d = orc_decode_raw(g, sv, ids, wts, cap);
    if (d == UINT64_MAX || !g->relabel) return d;
    for (uint64_t i = 0; i < d; i++) ids[i] = g->inv_perm[ids[i]];
    if (wts) {
        idw *t = (idw *)malloc(sizeof(idw) * (d ? d : 1));
        if (!t) return UINT64_MAX;
        for (uint64_t i = 0; i < d; i++) { t[i].id = ids[i]; t[i].w = wts[i]; }
        qsort(t, d, sizeof(idw), cmp_idw);
        for (uint64_t i = 0; i < d; i++) { ids[i] = t[i].id; wts[i] = t[i].w; }
        free(t);
    } else {
        qsort(ids, d, sizeof(uint32_t), cmp_u32);
    }
    return d;
}

/* ------------------------------------------------------------------ */
/* accessors for the test harness                                      */
/* ------------------------------------------------------------------ */
typedef struct {
    uint64_t n, arcs;
    uint32_t id_mode, off_mode, relabel, sample, weighted;
    uint32_t s, H, omega, r, w_O, ef_l;
    uint64_t bits_A, bits_O, ef_N, ef_U, ef_low_bits, ef_high_bits, n_samples;
    uint64_t words_A, words_O, words_ef_low, words_ef_high, words_samples;
    const uint64_t *A, *O, *ef_low, *ef_high, *samples, *x;
    const uint32_t *perm, *inv_perm;
} orc_info;

void orc_get_info(const orc_graph *g, orc_info *o) {
    o->n = g->n; o->arcs = g->arcs; o->id_mode = g->id_mode; o->off_mode = g->off_mode;
    o->relabel = g->relabel; o->sample = g->sample; o->weighted = g->weighted;
    o->s = g->s; o->H = g->H; o->omega = g->omega; o->r = g->r; o->w_O = g->w_O; o->ef_l = g->ef_l;
    o->bits_A = g->bits_A; o->bits_O = g->bits_O; o->ef_N = g->ef_N; o->ef_U = g->ef_U;
    o->ef_low_bits = g->ef_low_bits; o->ef_high_bits = g->ef_high_bits; o->n_samples = g->n_samples;
    o->words_A = g->words_A; o->words_O = g->words_O; o->words_ef_low = g->words_ef_low;
    o->words_ef_high = g->words_ef_high; o->words_samples = g->words_samples;
    o->A = g->A; o->O = g->O; o->ef_low = g->ef_low; o->ef_high = g->ef_high; o->samples = g->samples;
    o->x = g->x; o->perm = g->perm; o->inv_perm = g->inv_perm;
}

/* ------------------------------------------------------------------ */
/* graph kernels on the INPUT csr (not on the decoder)                 */
/* ------------------------------------------------------------------ */

/* Textbook FIFO breadth-first search (Section 7.1.2 "BFS"): depth[v] = number
   of edges on a shortest path from src, UINT32_MAX if unreachable. */
int orc_bfs(uint64_t n, const uint64_t *rp, const uint32_t *col, uint32_t src, uint32_t *depth) {
    if (src >= n) return ORC_EINVAL;
    uint32_t *queue = (uint32_t *)malloc(sizeof(uint32_t) * n);
    if (!queue) return ORC_ENOMEM;
    for (uint64_t v = 0; v < n; v++) depth[v] = UINT32_MAX;
    uint64_t head = 0, tail = 0;
    depth[src] = 0;
    queue[tail++] = src;
    while (head < tail) {
        uint32_t v = queue[head++];
        for (uint64_t j = rp[v]; j < rp[v + 1]; j++) {
            uint32_t u = col[j];
            if (depth[u] == UINT32_MAX) { depth[u] = depth[v] + 1; queue[tail++] = u; }
        }
    }
    free(queue);
    return ORC_OK;
}

/* Single-source shortest paths on the weighted INPUT csr (Section 7.1.2
   "SSSP"; the paper runs GAPBS's delta-stepping, whose result is the plain
   shortest-path distance): dist[v] = minimum over paths src -> v of the sum of
   the arc weights, UINT64_MAX if unreachable.  Dijkstra's algorithm with a
   binary heap of (distance, vertex) entries and lazy deletion; weights >= 0. */
typedef struct { uint64_t d; uint32_t v; } orc_heap_entry;

static void heap_push(orc_heap_entry *h, uint64_t *len, uint64_t d, uint32_t v) {
    uint64_t i = (*len)++;
    while (i > 0) {
        uint64_t p = (i - 1) / 2;
        if (h[p].d <= d) break;
        h[i] = h[p];
        i = p;
    }
    h[i].d = d;
    h[i].v = v;
}

static orc_heap_entry heap_pop(orc_heap_entry *h, uint64_t *len) {
    orc_heap_entry top = h[0], last = h[--(*len)];
    uint64_t i = 0;
    for (;;) {
        uint64_t c = 2 * i + 1;
        if (c >= *len) break;
        if (c + 1 < *len && h[c + 1].d < h[c].d) c++;
        if (h[c].d >= last.d) break;
        h[i] = h[c];
        i = c;
    }
    if (*len) h[i] = last;
    return top;
}

int orc_sssp(uint64_t n, const uint64_t *rp, const uint32_t *col, const uint32_t *w, uint32_t src, uint64_t *dist) {
    if (src >= n || !w) return ORC_EINVAL;
    const uint64_t arcs = rp[n];
    orc_heap_entry *h = (orc_heap_entry *)malloc(sizeof(orc_heap_entry) * (arcs + 1));
    if (!h) return ORC_ENOMEM;
    for (uint64_t v = 0; v < n; v++) dist[v] = UINT64_MAX;
    uint64_t len = 0;
    dist[src] = 0;
    heap_push(h, &len, 0, src);
    while (len) {
        orc_heap_entry e = heap_pop(h, &len);
        if (e.d != dist[e.v]) continue; /* stale entry */
        for (uint64_t j = rp[e.v]; j < rp[e.v + 1]; j++) {
            uint64_t nd = e.d + w[j];
            if (nd < dist[col[j]]) {
                dist[col[j]] = nd;
                heap_push(h, &len, nd, col[j]);
            }
        }
    }
    free(h);
    return ORC_OK;
}

/* PageRank, pull form without atomics (Section 7.1.2 "PR"), FP64, exactly
   `iters` iterations:
     global:        r_0 = 1/n,    r_t[v] = (1-d)/n     + d * sum_{u in N_v} r_{t-1}[u] / d_u
     personalized:  r_0 = e_src,  r_t[v] = (1-d)[v=src] + d * sum_{u in N_v} r_{t-1}[u] / d_u
   Vertices of degree 0 contribute nothing (no dangling redistribution). */
int orc_pagerank_threads(uint64_t n, const uint64_t *rp, const uint32_t *col, double damping, uint32_t iters,
                         int64_t personalize, double *rank, int threads);
int orc_pagerank(uint64_t n, const uint64_t *rp, const uint32_t *col, double damping, uint32_t iters,
                 int64_t personalize, double *rank) {
    return orc_pagerank_threads(n, rp, col, damping, iters, personalize, rank, 1);
}

/* Same arithmetic; vertices split over `threads` OpenMP threads when built with
   OpenMP (each vertex's sum keeps its order, so results do not change). */
int orc_pagerank_threads(uint64_t n, const uint64_t *rp, const uint32_t *col, double damping, uint32_t iters,
                         int64_t personalize, double *rank, int threads) {
    if (n == 0 || (personalize >= 0 && (uint64_t)personalize >= n)) return ORC_EINVAL;
    double *prev = (double *)malloc(sizeof(double) * n);
    if (!prev) return ORC_ENOMEM;
    for (uint64_t v = 0; v < n; v++)
        rank[v] = personalize < 0 ? 1.0 / (double)n : (v == (uint64_t)personalize ? 1.0 : 0.0);
    for (uint32_t t = 0; t < iters; t++) {
        memcpy(prev, rank, sizeof(double) * n);
        (void)threads;
#pragma omp parallel for schedule(dynamic, 4096) num_threads(threads > 0 ? threads : 1)
        for (uint64_t v = 0; v < n; v++) {
            double sum = 0.0;
            for (uint64_t j = rp[v]; j < rp[v + 1]; j++) {
                uint32_t u = col[j];
                uint64_t du = rp[u + 1] - rp[u];
                if (du) sum += prev[u] / (double)du;
            }
            double base = personalize < 0 ? (1.0 - damping) / (double)n
                                           : (v == (uint64_t)personalize ? 1.0 - damping : 0.0);
            rank[v] = base + damping * sum;
        }
    }
    free(prev);
    return ORC_OK;
}
