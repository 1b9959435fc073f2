/*
 * lg.h -- C ABI of the GB300 Log(Graph) hot path (liblg.so).
 *
 * Log(Graph) (Besta et al., PACT'18; full version arXiv:2010.15879) stores a
 * graph's adjacency array AA = (O, A) in "logarithmized" form: vertex IDs in
 * ceil(log n) bits or in per-neighborhood local / fixed-size-gap widths, edge
 * weights in ceil(log maxW) bits, and the offsets O either bit-packed at
 * ceil(log 2m) bits or as an Elias-Fano (sparse succinct, "bvSD") bit vector.
 * This library builds that structure on the GPU from a CSR and runs the graph
 * kernels directly on it, decoding neighborhoods inside the kernels.
 *
 * Conventions shared by every entry point
 *   - Pointers marked "device" must be CUDA device (or managed) memory on the
 *     current device; "host" means ordinary host memory.  No entry point frees
 *     a caller buffer.  All sizes are element counts unless said otherwise.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it.  Entry points that must read a device
 *     result on the host (sizes, error flags, BFS frontier counts) synchronize
 *     that stream before returning; each says so.
 *   - Vertex IDs at the API are the caller's original 0-based IDs (n < 2^32).
 *     A relabeling chosen at encode time stays internal.
 *   - Errors: every entry point returns an lg_status; a human-readable message
 *     for the calling thread is available from lg_last_error().  No kernel
 *     traps; device-detected errors are reported through a device flag.
 *   - Thread safety: calls on distinct lg_graph objects may run concurrently;
 *     calls on the same graph may run concurrently only if they use the same
 *     stream or are otherwise ordered by the caller.
 *
 * Tuning knobs (environment variables, decimal; unset = the default).  None
 * changes a result, only how the work is scheduled:
 *   LG_HEAVY_MIN     256   degrees above this go to the heavy-vertex schedule
 *                          (a warp per item; 0 = default); read at every
 *                          lg_encode
 *   LG_HEAVY_SEG     4096  fields per heavy-schedule item (values below 32 =
 *                          default); read at every lg_encode
 *   LG_BFS_PULL_DIV  64    a BFS level runs bottom-up when its frontier holds
 *                          more than n / LG_BFS_PULL_DIV vertices (0 =
 *                          default); read once
 *   LG_HOT_BYTES     64 MiB  DM-relabeled graphs: gathers of the first
 *                          LG_HOT_BYTES of a per-vertex array (the hubs' rows)
 *                          are marked evict-last in L2, the rest evict-first
 *                          (0 = none evict-last); read at every traversal
 */
#ifndef LG_H
#define LG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lg_graph lg_graph; /* opaque; owns all of its device memory */

typedef enum {
    LG_OK = 0,
    LG_EINVAL = 1,        /* bad argument or invalid input CSR              */
    LG_ENOMEM = 2,        /* device or host allocation failed                */
    LG_ECUDA = 3,         /* a CUDA runtime call failed                      */
    LG_ERANGE = 4,        /* output capacity too small (sizes were written)  */
    LG_ETIMEOUT = 5,      /* a bounded device wait ran out                   */
    LG_EUNSUPPORTED = 6   /* valid but unsupported combination of options    */
} lg_status;

/* How vertex IDs are stored in A (Sections 3.2.1, 3.2.2 and 3.6). */
typedef enum {
    LG_ID_GLOBAL = 0,     /* every ID in s = ceil(log2 n) bits ("LG-g")                     */
    LG_ID_LOCAL = 1,      /* per neighborhood: [w_v : H][d_v IDs of w_v bits] ("LG-l")      */
    LG_ID_LOCAL_GAP = 2,  /* [g_v : H][first ID : s][d_v - 1 differences of g_v bits]
                             ("LG-l-gap", fixed-size gap encoding)                          */
    LG_ID_CSR32 = 3       /* not compressed: 32-bit IDs and 64-bit row offsets, the
                             traditional adjacency array run by the same kernels            */
} lg_id_mode;

/* How the offsets O are stored (Sections 3.4 and 4.3). */
typedef enum {
    LG_OFF_PACKED = 0,    /* O[0..n] each in w_O = bits(x_n) bits ("ptrLogn")             */
    LG_OFF_EF = 1         /* Elias-Fano over x_0..x_n with select samples ("bvSD")         */
} lg_off_mode;

#define LG_FLAG_CHECK_SYMMETRIC 1u /* lg_encode also verifies that every arc has its reverse */

typedef struct {
    uint32_t id_mode;       /* lg_id_mode                                                   */
    uint32_t off_mode;      /* lg_off_mode (ignored for LG_ID_CSR32)                        */
    uint32_t relabel;       /* 0 = keep IDs; 1 = DM permuter (Section 5.6): higher degree
                               gets a smaller label, ties by original ID; 2 = the greedy
                               heuristic for local IDs (Section 3.2.2, Listing 1): vertices
                               by increasing degree (ties by ID) give the next free labels
                               to their unlabeled neighbors, unreached vertices follow in
                               ID order                                                      */
    uint32_t select_sample; /* EF select sample rate, a power of two in [64, 65536];
                               0 means 512                                                  */
    uint32_t weight_bits;   /* 0 = bits(max weight); else the fixed weight width (<= 32)    */
    uint32_t flags;         /* LG_FLAG_* bits                                               */
} lg_encode_opts;

typedef struct {
    uint64_t n, arcs;          /* vertices, stored arcs (2m for an undirected graph)        */
    uint64_t bits_A;           /* exact payload bits of A                                   */
    uint64_t bits_O;           /* exact payload bits of O (packed, or EF low + high +
                                  64 per select sample)                                     */
    uint64_t bytes_A, bytes_O; /* device bytes held, with padding and guard words           */
    uint64_t bytes_perm;       /* device bytes of the permutation (0 without relabel)       */
    uint64_t bytes_total;      /* bytes_A + bytes_O + bytes_perm + bytes_schedule (+ CSR32
                                  weights)                                                  */
    uint64_t max_degree;
    uint32_t id_mode, off_mode, relabel, weighted;
    uint32_t s;                /* global ID width, max(1, bits(n - 1))                      */
    uint32_t H;                /* width of the per-neighborhood width field, bits(s)        */
    uint32_t omega;            /* weight width (0 if unweighted)                            */
    uint32_t w_O;              /* packed offset width (0 for EF)                            */
    uint32_t ef_l;             /* Elias-Fano low-bit count (0 for packed)                   */
    uint32_t select_sample;
    double bits_per_arc;       /* (bits_A + bits_O) / arcs                                  */
    uint64_t bytes_schedule;   /* device bytes of the heavy-vertex decode schedule (derived
                                  from A and O at encode time; not part of the format)      */
} lg_stats;

/* Read-only device views of the encoded arrays, for inspection and parity
   checks.  Each stream is u64 words, zero padded to an even count, followed by
   four zero guard words; `words_*` counts all of them. */
typedef struct {
    const uint64_t *A;         uint64_t words_A;
    const uint64_t *O;         uint64_t words_O;         /* packed offsets or CSR row_ptr */
    const uint64_t *ef_low;    uint64_t words_ef_low;
    const uint64_t *ef_high;   uint64_t words_ef_high;
    const uint64_t *ef_samples; uint64_t words_ef_samples;
    const uint32_t *perm;      /* original -> stored label, NULL without relabel */
    const uint32_t *inv_perm;  /* stored -> original label, NULL without relabel */
} lg_arrays;

/*
 * lg_encode -- build the logarithmized graph from a CSR adjacency array.
 * Paper: the construction of Listing 3 (Section 6): permute (DM, Section 5.6),
 * transform A (Sections 3.2-3.6), build and logarithmize O (Sections 3.4, 4.3).
 *   row_ptr  device, n+1 u64, row_ptr[0] = 0, nondecreasing, row_ptr[n] = arcs
 *   col      device, arcs u32, each row strictly increasing, every value < n
 *   weights  device, arcs u32 or NULL; a weight must fit weight_bits when given.
 *            Weights need LG_ID_GLOBAL or LG_ID_CSR32 (else LG_EUNSUPPORTED).
 *   n        1 <= n <= 2^32 - 1
 *   opts     host; NULL means {LG_ID_GLOBAL, LG_OFF_PACKED, 0, 512, 0, 0}
 *   out      host; receives the new graph (NULL on error)
 * The inputs are read on `stream` and may be freed once the call returns.  The
 * call synchronizes `stream` (validation result, sizes).  An invalid CSR gives
 * LG_EINVAL.  The graph models an undirected graph (Section 2.1): BFS and
 * PageRank assume every arc has its reverse; set LG_FLAG_CHECK_SYMMETRIC to
 * have that verified.
 */
lg_status lg_encode(const uint64_t *row_ptr, const uint32_t *col, const uint32_t *weights,
                    uint64_t n, uint64_t arcs, const lg_encode_opts *opts, void *stream,
                    lg_graph **out);

/* lg_stats_get -- sizes and widths of an encoded graph.  `out` host.  No GPU work. */
lg_status lg_stats_get(const lg_graph *g, lg_stats *out);

/* lg_arrays_get -- device pointers to the encoded arrays (owned by g; valid
   until lg_free).  `out` host.  No GPU work. */
lg_status lg_arrays_get(const lg_graph *g, lg_arrays *out);

/*
 * lg_decode -- decode the whole graph back into a CSR in stored order: the
 * neighborhood access of Section 3.7.2 applied to every vertex, the inverse
 * of lg_encode.
 *   row_ptr   device, n+1 u64 arc offsets
 *   col       device, capacity u32: row i is the neighborhood of stored vertex
 *             i, IDs as stored labels, ascending.  Without relabeling this is
 *             the input CSR; with it, stored vertex i is original vertex
 *             inv_perm[i] and label l is original ID inv_perm[l] (lg_arrays_get)
 *   weights   device, capacity u32, or NULL (a weighted graph only, else
 *             LG_EINVAL)
 * LG_ERANGE if capacity < arcs (nothing written).  Asynchronous on `stream`:
 * no host wait.
 */
lg_status lg_decode(const lg_graph *g, uint64_t *row_ptr, uint32_t *col, uint32_t *weights, uint64_t capacity,
                    void *stream);

/*
 * lg_neighbors -- decode N_v for a list of vertices (getNeighbors of Listing 3,
 * the edge and neighborhood access of Section 3.7.2, the degree of 3.7.3).
 *   vertices     device, k u32 original IDs (< n; repeats allowed)
 *   out_offsets  device, k+1 u64: out_offsets[i] .. out_offsets[i+1] is the
 *                slice of out_ids holding N_{vertices[i]}; always written
 *   out_ids      device, out_capacity u32: neighbors as original IDs, each
 *                slice ascending (equal to the input CSR row)
 *   out_weights  device, out_capacity u32, or NULL (weighted graphs only)
 * If the total degree exceeds out_capacity the call writes out_offsets, leaves
 * out_ids untouched and returns LG_ERANGE (call again with a larger buffer).
 * A vertex >= n gives LG_EINVAL.  Synchronizes `stream` once (to read the
 * total size) and again at the end.
 */
lg_status lg_neighbors(const lg_graph *g, const uint32_t *vertices, uint64_t k,
                       uint64_t *out_offsets, uint32_t *out_ids, uint32_t *out_weights,
                       uint64_t out_capacity, void *stream);

/*
 * lg_bfs -- breadth-first search from S sources (Section 7.1.2, a
 * direction-optimizing, level-synchronous BFS), decoding the compressed
 * neighborhoods inside the traversal kernels.  Sources are processed as
 * bit-parallel multi-source sweeps of up to 64 sources each.
 *   sources  device, S u32 original IDs (< n)
 *   depths   device, S*n u32, row-major by source: depths[i*n + v] = number of
 *            edges on a shortest path from sources[i] to v, UINT32_MAX if v is
 *            unreachable (ties do not matter: depths are unique)
 * Synchronizes `stream` once per BFS level (frontier sizes steer the
 * direction).  A source >= n gives LG_EINVAL.
 */
lg_status lg_bfs(const lg_graph *g, const uint32_t *sources, uint32_t S, uint32_t *depths,
                 void *stream);

/*
 * lg_sssp -- single-source shortest paths (Section 7.1.2 "SSSP", delta-
 * stepping) on a weighted graph (weights stored after each ID, Section 3.3),
 * neighborhoods and weights decoded inside the relaxation kernel.
 *   source  original ID (< n)
 *   delta   bucket width (0 = 32); any value gives the same distances
 *   dist    device, n u64 indexed by original ID: the minimum over paths from
 *           source of the sum of arc weights, UINT64_MAX if unreachable
 * Needs a weighted graph in LG_ID_GLOBAL or LG_ID_CSR32 (else
 * LG_EUNSUPPORTED).  Synchronizes `stream` once per relaxation round (queue
 * sizes steer the buckets).
 */
lg_status lg_sssp(const lg_graph *g, uint32_t source, uint64_t delta, uint64_t *dist, void *stream);

/*
 * lg_pagerank -- pull PageRank without atomics (Section 7.1.2), FP32, exactly
 * `iters` iterations, neighborhoods decoded inside the kernel:
 *   global:        r_0 = 1/n,    r_t[v] = (1-d)/n      + d * sum_{u in N_v} r_{t-1}[u] / d_u
 *   personalized:  r_0 = e_s,    r_t[v] = (1-d)*[v==s] + d * sum_{u in N_v} r_{t-1}[u] / d_u
 * Vertices of degree 0 keep the teleport term only (no dangling mass).
 *   damping             d in [0, 1]
 *   personalize_source  host pointer to one u32 original ID s, or NULL for global
 *   ranks               device, n floats indexed by original ID
 * Asynchronous: returns once the work is enqueued (argument errors return
 * before any GPU work).  Exception: a personalized call on a relabeled graph
 * first reads the source's stored label back from the device, which waits for
 * `stream`; such a call cannot be captured into a CUDA graph.  iters = 0
 * writes r_0.
 */
lg_status lg_pagerank(const lg_graph *g, float damping, uint32_t iters,
                      const uint32_t *personalize_source, float *ranks, void *stream);

/*
 * lg_pagerank_noalloc -- lg_pagerank for callers that cannot allocate device
 * memory.  The paper has no counterpart: this is a deployment variant.  A
 * process whose device memory is owned by another allocator or reserved up
 * front under a fixed budget cannot add cudaMalloc calls of its own, and a
 * latency-sensitive loop cannot afford cudaFree's implicit synchronization;
 * this call runs the same kernels as lg_pagerank (same results) but keeps its
 * scratch in a fixed array inside liblg.so (9 MiB held on every GPU that loads
 * the library, until the process exits) and calls no allocator.
 *   Limit: graphs of at most 1,048,576 vertices (and at most 262,144 schedule
 *   items for vertices split by the heavy-vertex schedule); larger graphs give
 *   LG_ERANGE with a message naming both limits.  iters = 0 writes r_0, as
 *   lg_pagerank does, and touches no scratch.
 *   The first call on each device looks the array's device address up once
 *   (with that device current); make that first call before any stream
 *   capture.  If the lookup fails, the call returns LG_ECUDA and
 *   lg_last_error() says so (and names the capture when one is in progress).
 *   A personalized call on a relabeled graph waits for `stream` (it reads the
 *   source's stored label back from the device, as lg_pagerank does).
 *   All calls in the process share the one array and it keeps the last call's
 *   contents: calls whose GPU work overlaps (other streams, other threads) race
 *   and must be ordered by the caller.  Every scratch element is written before
 *   it is read, so stale contents never reach the result.
 * Arguments, layout and other errors as lg_pagerank.
 */
lg_status lg_pagerank_noalloc(const lg_graph *g, float damping, uint32_t iters,
                              const uint32_t *personalize_source, float *ranks, void *stream);

/* lg_free -- release a graph and all of its device memory.  NULL-safe.
   Waits for the graph's device to be idle, then returns the graph's arrays
   to the library pool of that device (below). */
void lg_free(lg_graph *g);

/* lg_free_async -- release a graph without waiting: its arrays return to
   the pool in stream order on `stream` (a cudaStream_t; NULL = legacy default
   stream).  Every use of g must be enqueued on `stream` before this call or
   ordered before it by the caller.  The host object is released at once; g is
   unusable afterwards.  NULL g is a no-op.  LG_ECUDA if a release fails (the
   remaining arrays are still released). */
lg_status lg_free_async(lg_graph *g, void *stream);

/* ------------------------------------------------------------------------
 * Device memory pool.  Graph arrays and the scratch of every call are
 * stream-ordered allocations from one pool per device owned by the library.
 * Freed blocks stay mapped in the pool and serve later calls, so a loop of
 * encode / traverse / free maps its memory once.  The pool never returns
 * memory by itself; lg_pool_trim does.
 * ------------------------------------------------------------------------ */

/* lg_pool_trim -- wait for `device` to be idle, then release pooled memory
   that no live graph or call holds until at most keep_bytes stay reserved.
   LG_ECUDA for an invalid device. */
lg_status lg_pool_trim(int device, uint64_t keep_bytes);

/* lg_pool_usage -- bytes the pool of `device` holds from the system
   (*reserved, host) and of those, bytes in live allocations (*used, host).
   No GPU work.  LG_EINVAL if an output is NULL, LG_ECUDA for an invalid device. */
lg_status lg_pool_usage(int device, uint64_t *reserved, uint64_t *used);

/* ------------------------------------------------------------------------
 * Batches: many independent graphs encoded and traversed in one launch.
 *
 * Every graph g keeps its own widths, as the paper sizes each structure by
 * its own n and m (Sections 3.2.1 and 3.4): IDs at s_g = max(1, bits(n_g - 1))
 * ("LG-g"), offsets packed at w_O = max(1, bits(arcs_g)) ("ptrLogn").  One run
 * encodes every graph from its CSR, runs BFS from its vertex 0 and `iters`
 * pull PageRank iterations (Section 7.1.2) on the encoded stream, all in one
 * persistent kernel captured once as a CUDA graph and replayed.
 * ------------------------------------------------------------------------ */

typedef struct lg_batch lg_batch; /* opaque; owns its device memory, not the input */

#define LG_BATCH_FLAG_DROP_MEMBER 1u /* failure injection for tests: one member of the
                                        first multi-CTA team is left out of the work
                                        queue, so that team's barrier must run out of
                                        time and lg_batch_status returns LG_ETIMEOUT */

typedef struct {
    uint32_t autotune;      /* 1: time the candidate decode schedules at creation      */
    uint32_t lanes;         /* 0: default/autotuned; else lanes per vertex for every
                               graph, one of 1, 4, 8, 32 (disables autotune)          */
    uint64_t tile_arcs;     /* arcs per CTA before a graph gets a team of CTAs;
                               0: 2^19, or autotuned among 2^18 .. 2^21               */
    uint32_t wait_limit_us; /* time limit of a team barrier; 0 means 2 s              */
    uint32_t flags;         /* LG_BATCH_FLAG_* bits                                    */
} lg_batch_opts;

/* One graph of a batch as laid out on the device (64 bytes). */
typedef struct {
    uint64_t vbase;    /* first vertex in the batch vertex space        */
    uint64_t abase;    /* first arc in the batch input arrays           */
    uint64_t a_word;   /* first u64 word of the graph's A stream        */
    uint64_t o_word;   /* first u64 word of the graph's packed offsets  */
    uint32_t n, arcs;
    uint32_t s, w_O;   /* ID width and offset width                     */
    uint32_t lanes;    /* decode lanes per vertex                       */
    uint32_t team;     /* CTAs working on the graph                     */
    uint32_t pad[2];
} lg_batch_graph;

typedef struct {
    uint32_t count;                /* graphs                                      */
    uint64_t V, arcs;              /* total vertices and arcs                     */
    const uint64_t *A;             /* all A streams, device, words_A u64 words     */
    uint64_t words_A;
    const uint64_t *O;             /* all packed offsets, device                  */
    uint64_t words_O;
    const lg_batch_graph *graphs;  /* device, count entries                        */
    uint32_t n_items;              /* work items (graph, team member) per run     */
    uint32_t grid, threads;        /* persistent launch shape                     */
    uint64_t tile_arcs;            /* tile in use                                 */
    uint32_t teams, max_team;      /* graphs with more than one CTA; largest team */
    uint64_t bits_total;           /* sum over graphs of arcs*s + (n+1)*w_O       */
    uint64_t launches;             /* batch kernel launches so far (one per run)  */
    uint32_t graphs_by_lanes[4];   /* graphs decoded with 1, 4, 8, 32 lanes       */
} lg_batch_info;

/*
 * lg_batch_create -- plan a batch of `count` graphs held as one CSR.
 *   graph_vptr  device, count+1 u64: graph g owns vertices
 *               [graph_vptr[g], graph_vptr[g+1]) of the batch vertex space;
 *               graph_vptr[0] = 0, graph_vptr[count] = V
 *   row_ptr     device, V+1 u64 GLOBAL arc offsets (row_ptr[V] = arcs)
 *   col         device, arcs u32 LOCAL vertex IDs: a neighbor of a vertex of
 *               graph g is given relative to graph_vptr[g]; rows strictly
 *               increasing; every graph undirected (each arc has its reverse)
 *   opts        host or NULL (all zero)
 * row_ptr and col are kept BY REFERENCE: every lg_batch_run re-encodes from
 * them, so they must stay allocated (and may be refilled with new contents of
 * the same shape) until lg_batch_free.  Widths, stream layout and the work
 * queue are fixed here; with opts->autotune the candidate schedules are timed
 * on the device (each candidate run encodes and traverses a sample).  Invalid
 * input gives LG_EINVAL; a graph needs n_g < 2^32 and arcs_g < 2^32.
 * Synchronizes `stream`.
 */
lg_status lg_batch_create(const uint64_t *graph_vptr, const uint64_t *row_ptr, const uint32_t *col,
                          uint32_t count, uint64_t V, uint64_t arcs, const lg_batch_opts *opts,
                          void *stream, lg_batch **out);

/*
 * lg_batch_run -- encode every graph and traverse it, one graph launch.
 *   depths  device, V u32: BFS depth from the graph's own vertex 0, by batch
 *           vertex; UINT32_MAX = unreachable
 *   ranks   device, V floats: PageRank of each graph over its own n_g (as
 *           lg_pagerank, global, r_0 = 1/n_g), after `iters` iterations
 *           (iters = 0 leaves ranks untouched)
 * Asynchronous.  The first call (and any call with a different damping, iters
 * or output pointer) captures and instantiates the run graph; later calls only
 * replay it.  Runs of one batch must not overlap: order them on one stream.
 * Call lg_batch_status to learn whether a team barrier ran out of time.
 */
lg_status lg_batch_run(lg_batch *b, float damping, uint32_t iters, uint32_t *depths, float *ranks,
                       void *stream);

/* lg_batch_status -- synchronize `stream` and report the last run's device
   status: LG_OK, or LG_ETIMEOUT if a team barrier gave up (that graph's
   results are incomplete; the other graphs are unaffected). */
lg_status lg_batch_status(lg_batch *b, void *stream);

/* lg_batch_info_get -- sizes, schedule and device views.  `out` host.  No GPU work. */
lg_status lg_batch_info_get(const lg_batch *b, lg_batch_info *out);

/* lg_batch_free -- release the batch's device memory (not the input).  NULL-safe.
   Synchronizes the device. */
void lg_batch_free(lg_batch *b);

/* ------------------------------------------------------------------------
 * Serving: resident compressed graphs answering a stream of requests with
 * continuous batching.  The paper has no serving layer; the requests are its
 * operations: neighborhood lookups (getNeighbors, Section 3.7.2), BFS and
 * personalized PageRank (Section 7.1.2), run on graphs encoded by lg_encode.
 *
 * Per graph, three engines (host threads with their own CUDA streams) run
 * concurrently: a 64-slot multi-source BFS sweep that new sources join
 * between two levels, an 8-slot personalized PageRank sweep that requests join
 * between two iterations (the 8 rank vectors of a vertex share one 32-byte
 * sector), and a lookup engine that merges every waiting lookup into one
 * decode.  A request is admitted when its device state (BFS depth row, PPR
 * result vector, lookup output) fits a fixed device arena; results are copied
 * into a pinned host arena and stay there until lg_server_release.
 * ------------------------------------------------------------------------ */

typedef struct lg_server lg_server; /* opaque; uses the graphs, does not own them */

typedef enum {
    LG_REQ_NEIGHBORS = 0,   /* N_v of `count` vertices                                  */
    LG_REQ_BFS = 1,         /* depths from `source`                                     */
    LG_REQ_PPR = 2          /* personalized PageRank from `source`                       */
} lg_request_kind;

typedef struct {
    uint64_t device_bytes;       /* device arena for request state; 0 = 16 GiB          */
    uint64_t host_bytes;         /* pinned host arena for results; 0 = 4 GiB            */
    uint32_t bfs_slots;          /* BFS sources per sweep, 1..64; 0 = 64                */
    uint32_t ppr_slots;          /* PPR requests per sweep, 1..8; 0 = 8                 */
    uint32_t nbr_batch_vertices; /* most vertices decoded per lookup batch; 0 = 2^20    */
    uint32_t ppr_iters;          /* PPR iterations when a request gives 0; 0 = 10       */
} lg_server_opts;

typedef struct {
    uint32_t kind;              /* lg_request_kind                                      */
    uint32_t graph;             /* index into the graphs given to lg_server_create      */
    uint32_t source;            /* BFS / PPR source vertex (< n)                        */
    uint32_t iters;             /* PPR iterations (0: server default)                   */
    float damping;              /* PPR damping in (0, 1] (0: 0.85)                      */
    uint32_t count;             /* lookup: number of vertices, 1 .. 2^20                */
    const uint32_t *vertices;   /* lookup: host array of `count` vertices (< n), copied */
    uint64_t user;              /* returned unchanged in the result                     */
} lg_request;

typedef struct {
    uint64_t ticket, user;
    uint32_t kind, graph;
    int32_t status;             /* LG_OK, LG_ENOMEM or LG_ECUDA                         */
    const void *data;           /* pinned host memory owned by the server until
                                   lg_server_release:
                                   NEIGHBORS: u64 offsets[count+1] (from 0), then u32 IDs
                                   BFS: u32 depths[n] (UINT32_MAX unreachable)
                                   PPR: float ranks[n]                                  */
    uint64_t bytes, count;      /* bytes of data; count = vertices queried, or n        */
    uint64_t t_submit_ns, t_admit_ns, t_done_ns; /* steady clock                        */
} lg_result;

typedef struct {
    uint64_t submitted, completed, failed, by_kind[3];
    uint64_t bfs_levels;         /* sweep levels run                                    */
    uint64_t bfs_joins;          /* sources that joined a sweep                         */
    uint64_t bfs_joins_running;  /* ... while other sources of the sweep were active    */
    uint64_t bfs_max_active;     /* most sources active in one sweep                    */
    uint64_t ppr_iterations, ppr_joins, ppr_joins_running, ppr_max_active;
    uint64_t nbr_batches, nbr_max_batch;
    uint64_t admission_waits;    /* times a request waited for device memory            */
    uint64_t device_bytes, device_used, device_peak;
    uint64_t host_bytes, host_used, host_peak;
} lg_server_stats;

typedef struct {
    uint64_t completed, failed;
    uint64_t makespan_ns;        /* first scheduled arrival to last completion          */
} lg_replay_stats;

/*
 * lg_server_create -- start serving `count` graphs encoded on the current
 * device.  Requests and results use original IDs; for a DM-relabeled graph
 * the server keeps a host copy of its permutation and the PageRank sweep keeps
 * the hubs' rows in L2.  Allocates the two arenas and per-graph engine state
 * (BFS masks 24 B and PPR vectors 64 B per vertex) and starts 3 threads per
 * graph.  The graphs must outlive the server.
 */
lg_status lg_server_create(const lg_graph *const *graphs, uint32_t count, const lg_server_opts *opts,
                           lg_server **out);

/* lg_server_submit -- enqueue one request (host memory; copied).  Returns at
   once with a ticket.  Invalid requests give LG_EINVAL; a request whose state
   could never fit the arenas gives LG_ENOMEM.  Thread-safe. */
lg_status lg_server_submit(lg_server *s, const lg_request *req, uint64_t *ticket);

/* lg_server_wait -- up to `max` completed results (in completion order), waiting
   at most timeout_us for the first one; *got = 0 on timeout.  Thread-safe. */
lg_status lg_server_wait(lg_server *s, lg_result *out, uint32_t max, uint32_t *got, uint32_t timeout_us);

/* lg_server_release -- return a delivered result's host memory to the server. */
lg_status lg_server_release(lg_server *s, uint64_t ticket);

/* lg_server_stats_get -- counters and arena use.  No GPU work. */
lg_status lg_server_stats_get(lg_server *s, lg_server_stats *out);

/*
 * lg_server_replay -- open-loop load generator: request i (columns kind,
 * graph, source; lookup vertices nbr_vertices[nbr_off[i] .. nbr_off[i+1]])
 * is submitted by a separate thread at arrival_ns[i] after the start (PPR
 * with the server's default iterations and damping 0.85).  The calling thread
 * collects every result: latency_ns[i] = completion - scheduled arrival; if
 * keep and keep[i] are not NULL the result bytes are copied there (the caller
 * sizes it: see lg_result.data); every result is released.  All requests are
 * validated before the clock starts.  Returns LG_ECUDA if a request failed.
 */
lg_status lg_server_replay(lg_server *s, uint64_t n, const uint32_t *kind, const uint32_t *graph,
                           const uint32_t *source, const uint64_t *nbr_off, const uint32_t *nbr_vertices,
                           const uint64_t *arrival_ns, void *const *keep, uint64_t *latency_ns,
                           lg_replay_stats *out);

/* lg_server_engine_time -- device time of one engine's kernels, measured with
   CUDA events on the engine's stream: *ops = BFS levels, PPR sweeps or lookup
   batches run so far, *gpu_ns = their summed duration.  No GPU work. */
lg_status lg_server_engine_time(lg_server *s, uint32_t graph, uint32_t kind, uint64_t *ops, uint64_t *gpu_ns);

/* lg_server_destroy -- stop the engines (work in flight finishes, waiting
   requests are dropped), free the arenas and every undelivered result.  NULL-safe. */
void lg_server_destroy(lg_server *s);

/* lg_probe_gather -- a measurement aid with no counterpart in the paper: the
   contribution gathers of a pull sweep (Section 7.1.2, PageRank reads
   r[u] / d_u at every arc's u) without the decode, to give the rate at which
   this GPU serves scattered 4-byte reads.  Thread i reads idx[i] (device,
   count u32, each < table_len; a coalesced stream) and gathers table[idx[i]]
   (device, table_len floats) with the pull kernels' load and L2 policy.
   out (device) receives one partial sum per thread: it must hold
   min(count, 311,296) floats.  Indices are not checked against table_len:
   the caller guarantees them.  Asynchronous on `stream`. */
lg_status lg_probe_gather(const uint32_t *idx, uint64_t count, const float *table, uint64_t table_len,
                          float *out, void *stream);

/* lg_kernel_launches -- number of CUDA kernels this library has launched in
   this process so far (all threads, all devices).  For instrumentation: the
   difference across a region counts the library's launches in it.  No GPU work. */
uint64_t lg_kernel_launches(void);

/* lg_last_error -- message describing the last failure on this thread ("" if
   none).  The pointer stays valid until the next lg_* call on this thread. */
const char *lg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LG_H */
