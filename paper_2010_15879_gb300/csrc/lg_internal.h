// Host-side internals of liblg.so: the graph object, the kernel launchers and
// the argument blocks of the traversal kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "lg.h"
#include "lg_device.cuh"

struct lg_graph {
  int device;
  uint64_t n, arcs;
  uint32_t id_mode, off_mode, relabel, weighted;
  uint32_t s, H, omega, r, w_O, ef_l, sample, sample_log2;
  uint64_t bits_A, bits_O;
  uint64_t ef_N, ef_U, ef_low_bits, ef_high_bits, n_samples;
  uint64_t max_degree;
  uint64_t *A;          uint64_t words_A;
  uint64_t *O;          uint64_t words_O;  // packed offsets, or row_ptr for CSR32
  uint64_t *ef_low;     uint64_t words_ef_low;
  uint64_t *ef_high;    uint64_t words_ef_high;
  uint64_t *ef_samples; uint64_t words_ef_samples;
  uint32_t *perm, *inv_perm;
  uint32_t *W;          // CSR32 weights (nullptr otherwise)
  // heavy-vertex schedule, derived from the encoded arrays at encode time
  lg::HeavyItem *items; uint64_t n_items;
  uint32_t *multi;      uint64_t n_multi;
  uint32_t heavy_min, heavy_seg;
};

namespace lg {

// u64 words for `bits` payload bits: padded to an even count plus four zero
// guard words (32 bytes).
inline uint64_t padded_words(uint64_t bits) {
  uint64_t w = (bits + 63) / 64;
  w += (w & 1);
  return w + 4;
}
inline uint32_t host_bits(uint64_t x) {
  uint32_t b = 0;
  while (x) { b++; x >>= 1; }
  return b;
}
inline unsigned grid_for(uint64_t items, unsigned per_block, unsigned cap = 1u << 30) {
  uint64_t g = (items + per_block - 1) / per_block;
  if (g == 0) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

GView make_view(const lg_graph* g);

// every kernel launch site calls this right after its <<<...>>> (instrumentation)
void count_launch();

// Stream-ordered allocation from the library's pool on the current device.
// Graph arrays and every call's scratch come from it; blocks released with
// cudaFreeAsync stay mapped for reuse (lg_pool_trim returns them).
cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t st);

// sets the calling thread's lg_last_error() message
void set_error_message(const char* msg);

// ------------------------------------------------------------------ scan
// out[0] = 0, out[i+1] = out[i] + in[i] for i < n (n+1 outputs).  `tmp` needs
// scan_tmp_words(n) u64 words.
uint64_t scan_tmp_words(uint64_t n);
cudaError_t scan_excl_u64(const uint64_t* in, uint64_t n, uint64_t* out, uint64_t* tmp, cudaStream_t st);
cudaError_t scan_excl_u32(const uint32_t* in, uint64_t n, uint64_t* out, uint64_t* tmp, cudaStream_t st);

// ------------------------------------------------------------------ sort
// Stable LSD radix sort of (key, value) pairs on the low `key_bits` bits.
// Buffers *_alt have the same size; the result ends in keys/vals.
size_t radix_tmp_bytes(uint64_t n);
cudaError_t radix_sort_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                           uint64_t n, uint32_t key_bits, void* tmp, cudaStream_t st);
cudaError_t radix_sort_u64(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt,
                           uint64_t n, uint32_t key_bits, void* tmp, cudaStream_t st);
// Sort each row [off[i], off[i+1]) of keys ascending, moving vals (nullable) along.
// Rows of <= 32 keys are skipped when `small_done` (their producer sorted them).
// Every key is below 2^key_bits.  `big_prefix`: the rows above 4,096 keys are
// the first rows (degrees descending), so they are sorted where they lie.
cudaError_t segmented_sort(uint32_t* keys, uint32_t* vals, const uint64_t* off, uint64_t rows,
                           uint64_t total, uint64_t max_row, cudaStream_t st, bool small_done = false,
                           uint32_t key_bits = 32, bool big_prefix = false);

// ------------------------------------------------------------------ encoder
cudaError_t enc_validate(const uint64_t* rp, const uint32_t* col, const uint32_t* w, uint64_t n,
                         uint64_t arcs, uint32_t wbits, int* err, unsigned long long* max_deg,
                         uint32_t* max_w, cudaStream_t st);
cudaError_t enc_check_symmetric(const uint64_t* rp, const uint32_t* col, uint64_t n, int* err,
                                cudaStream_t st);
// relabeled CSR for permuter `mode`: 1 = DM (Section 5.6), 2 = greedy (Listing 1)
cudaError_t enc_dm_relabel(const uint64_t* rp, const uint32_t* col, const uint32_t* w, uint64_t n,
                           uint64_t arcs, uint64_t max_deg, uint32_t mode, uint32_t* perm, uint32_t* inv_perm,
                           uint64_t* nrp, uint32_t* ncol, uint32_t* nw, cudaStream_t st);
cudaError_t enc_local_lengths(const uint64_t* rp, const uint32_t* col, uint64_t n, int gap, uint32_t s,
                              uint32_t H, uint8_t* wid, uint64_t* len, cudaStream_t st);
cudaError_t enc_pack_global(const uint32_t* col, const uint32_t* w, uint64_t arcs, uint32_t s,
                            uint32_t omega, uint64_t* out, uint64_t data_words, cudaStream_t st);
cudaError_t enc_pack_local(const uint64_t* rp, const uint32_t* col, const uint64_t* x, const uint8_t* wid,
                           uint64_t n, int gap, uint32_t s, uint32_t H, uint64_t* out, uint64_t data_words,
                           cudaStream_t st);
cudaError_t enc_pack_u64(const uint64_t* vals, uint64_t count, uint32_t w, uint64_t* out,
                         uint64_t data_words, cudaStream_t st);
cudaError_t enc_ef_high(const uint64_t* x, uint64_t N, uint32_t l, uint64_t* out, cudaStream_t st);
cudaError_t enc_ef_samples(const uint64_t* x, uint64_t N, uint32_t l, uint32_t sample, uint64_t* out,
                           uint64_t ns, cudaStream_t st);

// ------------------------------------------------------------------ traversal
struct PlanArgs {
  uint32_t* tile_count;      // items per tile (count pass) / multi vertices per tile
  const uint64_t* tile_off;  // exclusive prefix of tile_count (fill pass)
  const uint64_t* multi_off; // exclusive prefix of multi vertices per tile
  uint32_t* multi_count;
  HeavyItem* items;
  uint32_t* multi;
  uint32_t* segsum;          // per item: sum of its (gap) values
};

struct PrArgs {
  const float* contrib_in;   // r_{t-1}[u] / d_u, stored labels
  float* contrib_out;        // r_t[v] / d_v
  float* ranks_out;          // written on the last iteration (original labels)
  int last;                  // 1 on the last iteration
  float base_all;            // (1-d)/n for global PageRank
  float damp;
  int64_t personal;          // stored label of the personalization source, -1 = global
  float r0_all;              // 1/n (initial rank, global)
  float* part;               // per heavy item partial sums (split vertices)
  uint32_t hot;              // gathers of contributions u < hot keep their L2 lines (evict-last), the
                             // others are evict-first (DM order puts the most gathered vertices first)
};

struct BfsArgs {
  void* vis;                 // visited masks [n]
  const void* front_in;      // frontier masks of this level [n]
  void* front_out;           // frontier masks of the next level [n] (zero before a push level)
  uint32_t* depth;           // depths in stored labels: S x n, or n x S when vmajor
  uint32_t* const* rows;     // or, if not null, one depth row per source (device array of S pointers)
  const uint32_t* row_base;  // with rows: level at which each source joined (depth = level - base)
  const uint32_t* row_perm;  // with rows: row index of stored vertex v (inv_perm), or null = v
  uint64_t all_mask;         // bits of the active sources
  uint32_t S;
  uint32_t vmajor;           // depth[v * S + s] (one record per vertex) instead of depth[s * n + v]
  uint32_t level;            // depth of the current frontier
  const uint32_t* queue_in;  // frontier vertices (push levels)
  uint32_t queue_in_len;
  uint32_t* queue_out;       // vertices of the next frontier
  uint32_t* counters;        // [0] next queue length, [1] new (vertex, source) pairs
  void* hacc;                // per split vertex: OR of its items' frontier masks
  int* err;
  uint32_t hot;              // pull gathers of masks u < hot are evict-last in L2, the others evict-first
};

// Personalized PageRank for up to PPR_K requests at once (the serving
// engine): contributions are PPR_K floats per vertex, slot k of vertex v at
// [v * PPR_K + k], so one 32-byte sector gather serves every slot.
constexpr int PPR_K = 8;
struct PprArgs {
  const float* cin;          // [n][PPR_K] r_{t-1}[u] / d_u per slot
  float* cout;               // [n][PPR_K]; slots not in `active` are written 0
  float* part;               // [n_items][PPR_K] partial sums of split vertices
  uint32_t active;           // slots iterating in this launch
  uint32_t last;             // slots whose final ranks are written to result[k]
  uint32_t src[PPR_K];       // personalization vertex of each slot (stored label)
  float damp[PPR_K];
  float* result[PPR_K];      // n floats each (slots in `last`)
  const uint32_t* result_perm;  // result index of stored vertex v (inv_perm), or null = v
  uint32_t hot;              // gathers of rows u < hot are kept in L2 (evict-last), the others evict-first
};

struct NbrArgs {
  const uint32_t* vertices;  // original IDs
  uint64_t k;
  uint64_t* out_offsets;     // k+1 (the degree pass writes degrees into [0..k))
  uint32_t* out_ids;
  uint32_t* out_weights;
  int* err;
};

// whole-graph decode into a CSR in stored order (lg_decode)
// Global-ID and CSR-32 graphs hold their records in arc order, so their
// offsets are the row offsets: the row pass writes row_out[0..n] directly and
// the decode pass maps record j to col[j].  Local-ID graphs: one launch
// writes both (row offsets by a look-back over the tiles).
struct DecArgs {
  uint64_t* row_out;         // n+1 row offsets, written by the decode
  const uint64_t* row_ptr;   // the same array, read back by the heavy items (local modes)
  uint32_t* ids;             // arcs
  uint32_t* weights;         // arcs, or null
  // local modes: single-pass row offsets (zeroed before the launch)
  unsigned long long* tile_status;  // per tile: 0, aggregate (flag 1) or inclusive prefix (flag 2) in bits 62-63
  uint32_t* tile_ready;      // per tile: 1 once its row offsets are written
  uint32_t* ticket;          // next block to start (blocks take tiles in start order)
  int* err;                  // DERR_INTERNAL if a wait for another block ran out
  uint64_t wait_ns;          // limit of each such wait
};

struct TravOps {
  cudaError_t (*pr_init)(const GView&, const PrArgs&, cudaStream_t);
  cudaError_t (*pr_pull)(const GView&, const PrArgs&, cudaStream_t);
  cudaError_t (*bfs_pull)(const GView&, const BfsArgs&, int mask_bytes, cudaStream_t);
  cudaError_t (*bfs_push)(const GView&, const BfsArgs&, int mask_bytes, cudaStream_t);
  cudaError_t (*nbr_degrees)(const GView&, const NbrArgs&, cudaStream_t);
  cudaError_t (*nbr_decode)(const GView&, const NbrArgs&, cudaStream_t);
  cudaError_t (*plan_count)(const GView&, const PlanArgs&, cudaStream_t);
  cudaError_t (*plan_fill)(const GView&, const PlanArgs&, cudaStream_t);
  cudaError_t (*plan_carry)(const GView&, const PlanArgs&, cudaStream_t);
  cudaError_t (*ppr_pull)(const GView&, const PprArgs&, cudaStream_t);
  cudaError_t (*ppr_join)(const GView&, float* cin, uint32_t slot, uint32_t src, cudaStream_t);
  cudaError_t (*dec_all)(const GView&, const DecArgs&, cudaStream_t);
};

// finishing kernels for vertices split into several heavy items (lg_api.cu)
cudaError_t pr_finish_multi(const GView& g, const PrArgs& a, cudaStream_t st);
cudaError_t bfs_finish_multi(const GView& g, const BfsArgs& a, int mask_bytes, cudaStream_t st);
cudaError_t ppr_finish_multi(const GView& g, const PprArgs& a, cudaStream_t st);
cudaError_t plan_carry_scan(HeavyItem* items, const uint32_t* multi, uint64_t n_multi, const uint32_t* segsum,
                            cudaStream_t st);

const TravOps* trav_ops(int id_mode, int off_mode);
const TravOps* trav_ops_global_packed();
const TravOps* trav_ops_global_ef();
const TravOps* trav_ops_local_packed();
const TravOps* trav_ops_local_ef();
const TravOps* trav_ops_gap_packed();
const TravOps* trav_ops_gap_ef();
const TravOps* trav_ops_csr32();

// Stored labels below which pull gathers of an array of `elem_bytes` per
// vertex keep their L2 lines: on a DM-relabeled graph (hubs first) the first
// LG_HOT_BYTES (default 64 MiB) of the array, else every vertex.
uint32_t hot_rows(const lg_graph* g, uint32_t elem_bytes);

// ranks = r_0 (1/n, or the indicator of personal_orig >= 0): PageRank after zero
// iterations (lg_api.cu)
cudaError_t pr_fill0(float* ranks, uint64_t n, int64_t personal_orig, cudaStream_t st);

// BFS helpers (lg_api.cu); vmajor: depth[v * S + s] instead of depth[s * n + v]
cudaError_t bfs_seed(void* vis, void* front, uint32_t* depth, uint64_t n, const uint32_t* sources_stored,
                     uint32_t S, uint32_t vmajor, int mask_bytes, uint32_t* queue, uint32_t* counters,
                     cudaStream_t st);
cudaError_t bfs_permute_depths(const uint32_t* tmp, uint32_t* out, const uint32_t* perm, uint64_t n,
                               uint32_t S, cudaStream_t st);
cudaError_t map_ids(const uint32_t* in, uint32_t* out, const uint32_t* perm, uint64_t k, uint64_t n,
                    int* err, cudaStream_t st);

}  // namespace lg
