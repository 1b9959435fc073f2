// liblg.so: the C ABI declared in include/lg.h.
//
// The construction follows Listing 3 (Section 6) of the Log(Graph) paper:
// permute (DM, Section 5.6), transform A (Sections 3.2-3.6), build the offsets
// and logarithmize them (Sections 3.4 and 4.3).  getNeighbors, BFS and
// PageRank decode the structure inside their kernels.
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "lg_internal.h"
#include "lg_traverse.cuh"

namespace {

thread_local char g_err[768] = "";

void set_errf(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}

lg_status from_cuda(cudaError_t e, const char* what) {
  set_errf("%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? LG_ENOMEM : LG_ECUDA;
}

#define LG_TRY(call)                                    \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return from_cuda(e_, #call); \
  } while (0)

// stream-ordered temporary buffer, released (stream-ordered) on scope exit
struct Tmp {
  void* p = nullptr;
  cudaStream_t st;
  explicit Tmp(cudaStream_t s) : st(s) {}
  ~Tmp() {
    if (p) cudaFreeAsync(p, st);
  }
  Tmp(const Tmp&) = delete;
  Tmp& operator=(const Tmp&) = delete;
  cudaError_t alloc(size_t bytes) { return lg::pool_alloc(&p, bytes ? bytes : 16, st); }
  template <typename T> T* as() const { return reinterpret_cast<T*>(p); }
};

struct DeviceGuard {
  int prev = -1;
  bool changed = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
      cudaSetDevice(dev);
      changed = true;
    }
  }
  ~DeviceGuard() {
    if (changed) cudaSetDevice(prev);
  }
};

lg_status describe_dev_err(int flags) {
  set_errf("invalid input:%s%s%s%s%s%s%s", (flags & lg::DERR_ROWPTR) ? " row_ptr not monotone or out of range;" : "",
           (flags & lg::DERR_COL_RANGE) ? " neighbor id >= n;" : "",
           (flags & lg::DERR_UNSORTED) ? " a row is not strictly increasing;" : "",
           (flags & lg::DERR_WEIGHT) ? " a weight does not fit weight_bits;" : "",
           (flags & lg::DERR_ASYM) ? " an arc has no reverse arc;" : "",
           (flags & lg::DERR_QUERY) ? " a vertex id is >= n;" : "",
           (flags & lg::DERR_INTERNAL) ? " internal invariant failed;" : "");
  return LG_EINVAL;
}

// graph arrays: the bit readers fetch whole 32-byte sectors of them, so a
// block that is not 32-byte aligned is refused (pool blocks are)
cudaError_t alloc_words(uint64_t** p, uint64_t words, cudaStream_t st) {
  cudaError_t e = lg::pool_alloc((void**)p, words * sizeof(uint64_t), st);
  if (e != cudaSuccess) return e;
  if (reinterpret_cast<uintptr_t>(*p) & 31u) {
    cudaFreeAsync(*p, st);
    *p = nullptr;
    return cudaErrorMisalignedAddress;
  }
  return cudaMemsetAsync(*p, 0, words * sizeof(uint64_t), st);
}

// tunables (environment overrides; include/lg.h lists them)
uint32_t env_u32(const char* name, uint32_t dflt) {
  const char* s = getenv(name);
  if (!s || !*s) return dflt;
  return (uint32_t)strtoul(s, nullptr, 10);
}
// Light/heavy degree limit and the split size of the heavy-vertex schedule,
// read at every encode (LG_HEAVY_MIN, LG_HEAVY_SEG).
uint32_t heavy_min_env() {
  const uint32_t v = env_u32("LG_HEAVY_MIN", 256);
  return v ? v : 256;
}
uint32_t heavy_seg_env() {
  const uint32_t v = env_u32("LG_HEAVY_SEG", 4096);
  return v >= 32 ? v : 4096;
}
uint32_t pull_divisor() {
  static const uint32_t v = env_u32("LG_BFS_PULL_DIV", 64);
  return v ? v : 64;
}

}  // namespace

#include <atomic>
#include <mutex>

namespace lg {

static std::atomic<unsigned long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// One pool per device, created on first use, release threshold unlimited:
// repeated encodes, traversals and frees reuse mapped memory instead of
// mapping and unmapping gigabytes per call.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pools[64] = {};

static cudaError_t device_pool(int dev, cudaMemPool_t* out) {
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pools[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool;
    cudaError_t e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = UINT64_MAX;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(pool);
      return e;
    }
    g_pools[dev] = pool;
  }
  *out = g_pools[dev];
  return cudaSuccess;
}

cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  cudaMemPool_t pool = nullptr;
  if (e == cudaSuccess) e = device_pool(dev, &pool);
  if (e != cudaSuccess) return e;
  return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

void set_error_message(const char* msg) { snprintf(g_err, sizeof g_err, "%s", msg); }

GView make_view(const lg_graph* g) {
  GView v;
  memset(&v, 0, sizeof(v));
  v.A32 = reinterpret_cast<const uint32_t*>(g->A);
  v.A64 = g->A;
  v.O = g->O;
  v.ef_low = g->ef_low;
  v.ef_high32 = reinterpret_cast<const uint32_t*>(g->ef_high);
  v.ef_samples = g->ef_samples;
  v.perm = g->perm;
  v.inv_perm = g->inv_perm;
  v.W32 = g->W;
  v.n = g->n;
  v.arcs = g->arcs;
  v.ef_high_words32 = (g->ef_high_bits + 31) / 32;
  v.s = g->s; v.H = g->H; v.omega = g->omega; v.r = g->r; v.w_O = g->w_O; v.ef_l = g->ef_l;
  v.sample_log2 = g->sample_log2;
  v.items = g->items;
  v.multi = g->multi;
  v.n_items = g->n_items;
  v.n_multi = g->n_multi;
  v.heavy_min = g->heavy_min;
  v.heavy_seg = g->heavy_seg;
  return v;
}

// ---------------------------------------------------------------- split vertices
// A vertex split into several heavy items: its items' partial sums are added
// in item order (deterministic), then the vertex is finished.
__global__ void k_pr_finish_multi(GView g, PrArgs a) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.n_multi; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t first = g.multi[i];
    const HeavyItem h = g.items[first];
    float s = 0.f;
    for (uint32_t k = 0; k < h.nitems; k++) s += a.part[first + k];
    pr_finish(g, a, h.v, h.deg, s);
  }
}

cudaError_t pr_finish_multi(const GView& g, const PrArgs& a, cudaStream_t st) {
  if (g.n_multi == 0) return cudaSuccess;
  k_pr_finish_multi<<<grid_for(g.n_multi, 256, 4096), 256, 0, st>>>(g, a);
  count_launch();
  return cudaGetLastError();
}

__global__ void k_ppr_finish_multi(GView g, PprArgs a) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.n_multi; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t first = g.multi[i];
    const HeavyItem h = g.items[first];
    float s[PPR_K];
    for (int k = 0; k < PPR_K; k++) s[k] = 0.f;
    for (uint32_t j = 0; j < h.nitems; j++)
      for (int k = 0; k < PPR_K; k++) s[k] += a.part[(uint64_t)(first + j) * PPR_K + k];
    ppr_finish(a, h.v, h.deg, s);
  }
}

cudaError_t ppr_finish_multi(const GView& g, const PprArgs& a, cudaStream_t st) {
  if (g.n_multi == 0) return cudaSuccess;
  k_ppr_finish_multi<<<grid_for(g.n_multi, 256, 4096), 256, 0, st>>>(g, a);
  count_launch();
  return cudaGetLastError();
}

template <typename M>
__global__ void k_bfs_finish_multi(GView g, BfsArgs a) {
  M* hacc = reinterpret_cast<M*>(a.hacc);
  const M* vis = reinterpret_cast<const M*>(a.vis);
  M* fout = reinterpret_cast<M*>(a.front_out);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.n_multi; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t v = g.items[g.multi[i]].v;
    const M need = (M)((M)a.all_mask & (M)~vis[v]);
    const M acc = hacc[i];
    hacc[i] = 0;
    if (need == 0) fout[v] = 0;
    else bfs_finish<M>(g, a, v, need, acc, nullptr, nullptr, nullptr);
  }
}

cudaError_t bfs_finish_multi(const GView& g, const BfsArgs& a, int mb, cudaStream_t st) {
  if (g.n_multi == 0) return cudaSuccess;
  const unsigned grid = grid_for(g.n_multi, 256, 4096);
  if (mb == 2) { k_bfs_finish_multi<uint16_t><<<grid, 256, 0, st>>>(g, a); count_launch(); }
  else if (mb == 4) { k_bfs_finish_multi<uint32_t><<<grid, 256, 0, st>>>(g, a); count_launch(); }
  else { k_bfs_finish_multi<uint64_t><<<grid, 256, 0, st>>>(g, a); count_launch(); }
  return cudaGetLastError();
}

// carries of split gap-coded vertices: exclusive sums of the item sums, in order
__global__ void k_plan_carry_scan(HeavyItem* items, const uint32_t* multi, uint64_t n_multi, const uint32_t* segsum) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_multi; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t first = multi[i];
    const uint32_t k = items[first].nitems;
    uint32_t run = 0;
    for (uint32_t j = 0; j < k; j++) {
      items[first + j].carry = run;
      run += segsum[first + j];
    }
  }
}

cudaError_t plan_carry_scan(HeavyItem* items, const uint32_t* multi, uint64_t n_multi, const uint32_t* segsum,
                            cudaStream_t st) {
  if (n_multi == 0) return cudaSuccess;
  k_plan_carry_scan<<<grid_for(n_multi, 256, 4096), 256, 0, st>>>(items, multi, n_multi, segsum);
  count_launch();
  return cudaGetLastError();
}

const TravOps* trav_ops(int id_mode, int off_mode) {
  if (id_mode == ID_CSR32) return trav_ops_csr32();
  if (id_mode == ID_GLOBAL) return off_mode == OFF_EF ? trav_ops_global_ef() : trav_ops_global_packed();
  if (id_mode == ID_LOCAL) return off_mode == OFF_EF ? trav_ops_local_ef() : trav_ops_local_packed();
  return off_mode == OFF_EF ? trav_ops_gap_ef() : trav_ops_gap_packed();
}

// ---------------------------------------------------------------- small kernels
// Sources are few (<= 64 per sweep): one thread seeds them in order, so
// duplicates merge into one frontier entry.
template <typename M>
__global__ void k_bfs_seed(M* vis, M* front, uint32_t* depth, uint64_t n, const uint32_t* src, uint32_t S,
                           uint32_t vmajor, uint32_t* queue, uint32_t* counters) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  uint32_t q = 0;
  for (uint32_t i = 0; i < S; i++) {
    const uint32_t v = src[i];
    const M bit = (M)((M)1 << i);
    if (front[v] == 0) queue[q++] = v;
    front[v] = (M)(front[v] | bit);
    vis[v] = (M)(vis[v] | bit);
    depth[vmajor ? (uint64_t)v * S + i : (uint64_t)i * n + v] = 0;
  }
  counters[0] = q;
}

cudaError_t bfs_seed(void* vis, void* front, uint32_t* depth, uint64_t n, const uint32_t* src, uint32_t S,
                     uint32_t vmajor, int mb, uint32_t* queue, uint32_t* counters, cudaStream_t st) {
  if (mb == 2) { k_bfs_seed<uint16_t><<<1, 32, 0, st>>>((uint16_t*)vis, (uint16_t*)front, depth, n, src, S, vmajor, queue, counters); count_launch(); }
  else if (mb == 4) { k_bfs_seed<uint32_t><<<1, 32, 0, st>>>((uint32_t*)vis, (uint32_t*)front, depth, n, src, S, vmajor, queue, counters); count_launch(); }
  else { k_bfs_seed<uint64_t><<<1, 32, 0, st>>>((uint64_t*)vis, (uint64_t*)front, depth, n, src, S, vmajor, queue, counters); count_launch(); }
  return cudaGetLastError();
}

// zero the mask entries listed in a queue (the nonzeros of a frontier)
__global__ void k_clear_queue(uint8_t* masks, int mb, const uint32_t* queue, uint32_t len) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x) {
    uint8_t* p = masks + (uint64_t)queue[i] * mb;
    if (mb == 2) *reinterpret_cast<uint16_t*>(p) = 0;
    else if (mb == 4) *reinterpret_cast<uint32_t*>(p) = 0;
    else *reinterpret_cast<uint64_t*>(p) = 0;
  }
}

// out[s][o] = tmp[perm[o]][s]: the relabeled depths are one record of S
// values per vertex, so a thread gathers the record of perm[o] (16-byte loads
// when S is a multiple of 4) and writes its S values, each store coalesced
// over the warp's consecutive o
template <bool VEC>
__global__ void __launch_bounds__(256) k_permute_depths(const uint32_t* __restrict__ tmp, uint32_t* __restrict__ out,
                                                        const uint32_t* __restrict__ perm, uint64_t n, uint32_t S) {
  for (uint64_t o = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t p = perm[o];
    if (VEC) {
      const uint4* rec = reinterpret_cast<const uint4*>(tmp + p * S);
      for (uint32_t q = 0; q < S / 4; q++) {
        const uint4 x = __ldg(rec + q);
        __stcs(out + (uint64_t)(4 * q) * n + o, x.x);
        __stcs(out + (uint64_t)(4 * q + 1) * n + o, x.y);
        __stcs(out + (uint64_t)(4 * q + 2) * n + o, x.z);
        __stcs(out + (uint64_t)(4 * q + 3) * n + o, x.w);
      }
    } else {
      for (uint32_t s = 0; s < S; s++) __stcs(out + (uint64_t)s * n + o, __ldg(tmp + p * S + s));
    }
  }
}

cudaError_t bfs_permute_depths(const uint32_t* tmp, uint32_t* out, const uint32_t* perm, uint64_t n, uint32_t S,
                               cudaStream_t st) {
  if (S % 4 == 0) k_permute_depths<true><<<grid_for(n, 256, 152 * 16), 256, 0, st>>>(tmp, out, perm, n, S);
  else k_permute_depths<false><<<grid_for(n, 256, 152 * 16), 256, 0, st>>>(tmp, out, perm, n, S);
  count_launch();
  return cudaGetLastError();
}

// stored labels of caller ids (perm may be null), with a range check
__global__ void k_map_ids(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                          const uint32_t* __restrict__ perm, uint64_t k, uint64_t n, int* err) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t v = in[i];
    if (v >= n) { set_err(err, DERR_QUERY); out[i] = 0; continue; }
    out[i] = perm ? perm[v] : v;
  }
}

cudaError_t map_ids(const uint32_t* in, uint32_t* out, const uint32_t* perm, uint64_t k, uint64_t n, int* err,
                    cudaStream_t st) {
  if (k == 0) return cudaSuccess;
  k_map_ids<<<grid_for(k, 256, 4096), 256, 0, st>>>(in, out, perm, k, n, err);
  count_launch();
  return cudaGetLastError();
}

// r_0 written straight to the output (zero iterations)
__global__ void k_pr_fill0(float* ranks, uint64_t n, float r0, int64_t personal_orig) {
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x)
    ranks[v] = personal_orig < 0 ? r0 : ((int64_t)v == personal_orig ? 1.0f : 0.0f);
}

uint32_t hot_rows(const lg_graph* g, uint32_t elem_bytes) {
  const uint64_t all = g->n < 0xffffffffull ? g->n : 0xffffffffull;
  if (g->relabel != 1 || elem_bytes == 0) return (uint32_t)all;
  const char* e = getenv("LG_HOT_BYTES");  // read per traversal: a few ns
  const uint64_t bytes = (e && *e) ? (uint64_t)strtoull(e, nullptr, 10) : (64ull << 20);
  const uint64_t rows = bytes / elem_bytes;
  return (uint32_t)(rows < all ? rows : all);
}

cudaError_t pr_fill0(float* ranks, uint64_t n, int64_t personal_orig, cudaStream_t st) {
  k_pr_fill0<<<grid_for(n, 256, 152 * 32), 256, 0, st>>>(ranks, n, 1.0f / (float)n, personal_orig);
  count_launch();
  return cudaGetLastError();
}

}  // namespace lg

using namespace lg;

// =========================================================================
// C ABI
// =========================================================================
extern "C" const char* lg_last_error(void) { return g_err; }

extern "C" uint64_t lg_kernel_launches(void) { return (uint64_t)g_launches.load(std::memory_order_relaxed); }

extern "C" void lg_free(lg_graph* g) {
  if (!g) return;
  DeviceGuard dg(g->device);
  // nothing still uses g once the device is idle; the blocks go back to the
  // pool (they stay mapped for the next graph)
  cudaDeviceSynchronize();
  void* bufs[] = {g->A, g->O, g->ef_low, g->ef_high, g->ef_samples, g->perm, g->inv_perm, g->W, g->items, g->multi};
  for (void* p : bufs)
    if (p) cudaFreeAsync(p, cudaStreamLegacy);
  delete g;
}

extern "C" lg_status lg_decode(const lg_graph* g, uint64_t* row_ptr, uint32_t* col, uint32_t* weights,
                               uint64_t capacity, void* stream) {
  g_err[0] = 0;
  if (!g || !row_ptr || (g->arcs && !col)) { set_errf("lg_decode: null argument"); return LG_EINVAL; }
  if (weights && !g->weighted) { set_errf("lg_decode: weights requested from an unweighted graph"); return LG_EINVAL; }
  if (capacity < g->arcs) {
    set_errf("lg_decode: capacity %llu < %llu arcs", (unsigned long long)capacity, (unsigned long long)g->arcs);
    return LG_ERANGE;
  }
  DeviceGuard dg(g->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const uint64_t n = g->n;
  if (n == 0) {
    LG_TRY(cudaMemsetAsync(row_ptr, 0, sizeof(uint64_t), st));
    return LG_OK;
  }
  const GView v = make_view(g);
  const TravOps* ops = trav_ops((int)g->id_mode, (int)g->off_mode);
  DecArgs a;
  memset(&a, 0, sizeof(a));
  a.row_ptr = row_ptr;
  a.ids = col;
  a.weights = weights;
  if (g->id_mode == ID_GLOBAL || g->id_mode == ID_CSR32) {
    // records are in arc order: the offsets are the row offsets (one launch
    // writes both)
    a.row_out = row_ptr;
    LG_TRY(ops->dec_all(v, a, st));
    return LG_OK;
  }
  // local IDs: one launch (row offsets by a single-pass look-back over the
  // tiles, then the rows); its small state is zeroed first
  const uint64_t ntiles = (n + LG_TILE_V - 1) / LG_TILE_V;
  Tmp t_state(st);
  const size_t bytes = ntiles * (sizeof(unsigned long long) + sizeof(uint32_t)) + 16;
  LG_TRY(t_state.alloc(bytes));
  LG_TRY(cudaMemsetAsync(t_state.p, 0, bytes, st));
  a.tile_status = t_state.as<unsigned long long>();
  a.tile_ready = reinterpret_cast<uint32_t*>(a.tile_status + ntiles);
  a.ticket = a.tile_ready + ntiles;
  a.err = reinterpret_cast<int*>(a.ticket + 1);
  a.row_out = row_ptr;
  a.wait_ns = 200ull * 1000 * 1000;
  LG_TRY(ops->dec_all(v, a, st));
  int err = 0;
  LG_TRY(cudaMemcpyAsync(&err, a.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  LG_TRY(cudaStreamSynchronize(st));
  if (err) {
    set_errf("lg_decode: a wait between the decode's blocks ran out (row offsets incomplete)");
    return LG_ETIMEOUT;
  }
  return LG_OK;
}

extern "C" lg_status lg_free_async(lg_graph* g, void* stream) {
  g_err[0] = 0;
  if (!g) return LG_OK;
  DeviceGuard dg(g->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t first = cudaSuccess;
  void* bufs[] = {g->A, g->O, g->ef_low, g->ef_high, g->ef_samples, g->perm, g->inv_perm, g->W, g->items, g->multi};
  for (void* p : bufs) {
    if (!p) continue;
    const cudaError_t e = cudaFreeAsync(p, st);
    if (first == cudaSuccess) first = e;
  }
  delete g;
  if (first != cudaSuccess) return from_cuda(first, "lg_free_async");
  return LG_OK;
}

extern "C" lg_status lg_pool_trim(int device, uint64_t keep_bytes) {
  g_err[0] = 0;
  cudaMemPool_t pool = nullptr;
  LG_TRY(device_pool(device, &pool));
  DeviceGuard dg(device);
  LG_TRY(cudaDeviceSynchronize());
  LG_TRY(cudaMemPoolTrimTo(pool, (size_t)keep_bytes));
  return LG_OK;
}

extern "C" lg_status lg_pool_usage(int device, uint64_t* reserved, uint64_t* used) {
  g_err[0] = 0;
  if (!reserved || !used) { set_errf("lg_pool_usage: null argument"); return LG_EINVAL; }
  cudaMemPool_t pool = nullptr;
  LG_TRY(device_pool(device, &pool));
  unsigned long long r = 0, u = 0;
  LG_TRY(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &r));
  LG_TRY(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &u));
  *reserved = (uint64_t)r;
  *used = (uint64_t)u;
  return LG_OK;
}

extern "C" lg_status lg_stats_get(const lg_graph* g, lg_stats* out) {
  g_err[0] = 0;
  if (!g || !out) { set_errf("lg_stats_get: null argument"); return LG_EINVAL; }
  memset(out, 0, sizeof(*out));
  out->n = g->n; out->arcs = g->arcs;
  out->bits_A = g->bits_A; out->bits_O = g->bits_O;
  out->bytes_A = g->words_A * 8;
  out->bytes_O = (g->words_O + g->words_ef_low + g->words_ef_high + g->words_ef_samples) * 8;
  out->bytes_perm = g->perm ? 2 * g->n * sizeof(uint32_t) : 0;
  out->bytes_schedule = g->n_items * sizeof(HeavyItem) + g->n_multi * sizeof(uint32_t);
  out->bytes_total = out->bytes_A + out->bytes_O + out->bytes_perm + out->bytes_schedule + (g->W ? g->arcs * 4 : 0);
  out->max_degree = g->max_degree;
  out->id_mode = g->id_mode; out->off_mode = g->off_mode; out->relabel = g->relabel; out->weighted = g->weighted;
  out->s = g->s; out->H = g->H; out->omega = g->omega; out->w_O = g->w_O; out->ef_l = g->ef_l;
  out->select_sample = g->sample;
  out->bits_per_arc = g->arcs ? (double)(g->bits_A + g->bits_O) / (double)g->arcs : 0.0;
  return LG_OK;
}

extern "C" lg_status lg_arrays_get(const lg_graph* g, lg_arrays* out) {
  g_err[0] = 0;
  if (!g || !out) { set_errf("lg_arrays_get: null argument"); return LG_EINVAL; }
  out->A = g->A; out->words_A = g->words_A;
  out->O = g->O; out->words_O = g->words_O;
  out->ef_low = g->ef_low; out->words_ef_low = g->words_ef_low;
  out->ef_high = g->ef_high; out->words_ef_high = g->words_ef_high;
  out->ef_samples = g->ef_samples; out->words_ef_samples = g->words_ef_samples;
  out->perm = g->perm; out->inv_perm = g->inv_perm;
  return LG_OK;
}

// Heavy-vertex schedule, derived from the encoded arrays: every vertex of
// degree > heavy_min becomes ceil(d / HEAVY_SEG) items, listed in vertex order.
static lg_status build_schedule(lg_graph* g, cudaStream_t st) {
  g->heavy_min = heavy_min_env();
  g->heavy_seg = heavy_seg_env();
  const uint64_t ntiles = (g->n + LG_TILE_V - 1) / LG_TILE_V;
  Tmp t_cnt(st), t_mcnt(st), t_off(st), t_moff(st), t_stmp(st), t_seg(st);
  LG_TRY(t_cnt.alloc(ntiles * sizeof(uint32_t)));
  LG_TRY(t_mcnt.alloc(ntiles * sizeof(uint32_t)));
  LG_TRY(t_off.alloc((ntiles + 1) * sizeof(uint64_t)));
  LG_TRY(t_moff.alloc((ntiles + 1) * sizeof(uint64_t)));
  LG_TRY(t_stmp.alloc(scan_tmp_words(ntiles) * sizeof(uint64_t)));
  PlanArgs p;
  memset(&p, 0, sizeof(p));
  p.tile_count = t_cnt.as<uint32_t>();
  p.multi_count = t_mcnt.as<uint32_t>();
  p.tile_off = t_off.as<uint64_t>();
  p.multi_off = t_moff.as<uint64_t>();
  GView v = make_view(g);
  const TravOps* ops = trav_ops((int)g->id_mode, (int)g->off_mode);
  LG_TRY(ops->plan_count(v, p, st));
  LG_TRY(scan_excl_u32(p.tile_count, ntiles, t_off.as<uint64_t>(), t_stmp.as<uint64_t>(), st));
  LG_TRY(scan_excl_u32(p.multi_count, ntiles, t_moff.as<uint64_t>(), t_stmp.as<uint64_t>(), st));
  uint64_t tot[2] = {0, 0};
  LG_TRY(cudaMemcpyAsync(&tot[0], t_off.as<uint64_t>() + ntiles, 8, cudaMemcpyDeviceToHost, st));
  LG_TRY(cudaMemcpyAsync(&tot[1], t_moff.as<uint64_t>() + ntiles, 8, cudaMemcpyDeviceToHost, st));
  LG_TRY(cudaStreamSynchronize(st));
  g->n_items = tot[0];
  g->n_multi = tot[1];
  if (g->n_items == 0) return LG_OK;
  LG_TRY(pool_alloc((void**)&g->items, g->n_items * sizeof(HeavyItem), st));
  if (g->n_multi) LG_TRY(pool_alloc((void**)&g->multi, g->n_multi * sizeof(uint32_t), st));
  p.items = g->items;
  p.multi = g->multi;
  LG_TRY(ops->plan_fill(v, p, st));
  if (g->n_multi && g->id_mode == ID_LOCAL_GAP) {
    LG_TRY(t_seg.alloc(g->n_items * sizeof(uint32_t)));
    p.segsum = t_seg.as<uint32_t>();
    v = make_view(g);
    LG_TRY(ops->plan_carry(v, p, st));
    LG_TRY(plan_carry_scan(g->items, g->multi, g->n_multi, p.segsum, st));
  }
  LG_TRY(cudaStreamSynchronize(st));
  return LG_OK;
}

static lg_status encode_impl(lg_graph* g, const uint64_t* row_ptr, const uint32_t* col, const uint32_t* weights,
                             const lg_encode_opts& o, cudaStream_t st) {
  const uint64_t n = g->n, arcs = g->arcs;
  // ---- validation (one pass; device flag, never traps)
  Tmp small(st);
  LG_TRY(small.alloc(64));
  int* d_err = small.as<int>();
  unsigned long long* d_maxdeg = reinterpret_cast<unsigned long long*>(small.as<char>() + 8);
  uint32_t* d_maxw = reinterpret_cast<uint32_t*>(small.as<char>() + 16);
  LG_TRY(cudaMemsetAsync(small.p, 0, 64, st));
  LG_TRY(enc_validate(row_ptr, col, weights, n, arcs, o.weight_bits, d_err, d_maxdeg, d_maxw, st));
  struct { int err; int pad; unsigned long long maxdeg; uint32_t maxw; } h{};
  LG_TRY(cudaMemcpyAsync(&h, small.p, 20, cudaMemcpyDeviceToHost, st));
  LG_TRY(cudaStreamSynchronize(st));
  if (h.err) return describe_dev_err(h.err);
  if (o.flags & LG_FLAG_CHECK_SYMMETRIC) {
    LG_TRY(enc_check_symmetric(row_ptr, col, n, d_err, st));
    LG_TRY(cudaMemcpyAsync(&h.err, d_err, 4, cudaMemcpyDeviceToHost, st));
    LG_TRY(cudaStreamSynchronize(st));
    if (h.err) return describe_dev_err(h.err);
  }
  g->max_degree = h.maxdeg;

  // ---- widths (Sections 3.2.1, 3.3)
  g->s = host_bits(n - 1);
  if (g->s < 1) g->s = 1;
  g->H = host_bits(g->s);
  g->omega = 0;
  if (weights) {
    g->omega = o.weight_bits ? o.weight_bits : host_bits(h.maxw);
    if (g->omega < 1) g->omega = 1;
  }
  g->r = g->s + g->omega;

  // ---- optional relabel: DM (Section 5.6) or the greedy heuristic (Listing 1)
  const uint64_t* rp = row_ptr;
  const uint32_t* cl = col;
  const uint32_t* wt = weights;
  Tmp t_nrp(st), t_ncol(st), t_nw(st);
  if (g->relabel) {
    LG_TRY(pool_alloc((void**)&g->perm, n * sizeof(uint32_t), st));
    LG_TRY(pool_alloc((void**)&g->inv_perm, n * sizeof(uint32_t), st));
    LG_TRY(t_nrp.alloc((n + 1) * sizeof(uint64_t)));
    LG_TRY(t_ncol.alloc(arcs * sizeof(uint32_t)));
    if (weights) LG_TRY(t_nw.alloc(arcs * sizeof(uint32_t)));
    LG_TRY(enc_dm_relabel(row_ptr, col, weights, n, arcs, g->max_degree, g->relabel, g->perm, g->inv_perm,
                          t_nrp.as<uint64_t>(),
                          t_ncol.as<uint32_t>(), weights ? t_nw.as<uint32_t>() : nullptr, st));
    rp = t_nrp.as<uint64_t>();
    cl = t_ncol.as<uint32_t>();
    wt = weights ? t_nw.as<uint32_t>() : nullptr;
  }

  // ---- uncompressed baseline: copy the (possibly relabeled) CSR
  if (g->id_mode == ID_CSR32) {
    g->bits_A = 32 * arcs;
    g->words_A = padded_words(g->bits_A);
    LG_TRY(alloc_words(&g->A, g->words_A, st));
    if (arcs) LG_TRY(cudaMemcpyAsync(g->A, cl, arcs * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
    g->bits_O = 64 * (n + 1);
    g->words_O = padded_words(g->bits_O);
    LG_TRY(alloc_words(&g->O, g->words_O, st));
    LG_TRY(cudaMemcpyAsync(g->O, rp, (n + 1) * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
    if (wt) {
      LG_TRY(pool_alloc((void**)&g->W, (arcs ? arcs : 1) * sizeof(uint32_t), st));
      if (arcs) LG_TRY(cudaMemcpyAsync(g->W, wt, arcs * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
    }
    g->off_mode = OFF_ROWPTR;
    LG_TRY(cudaStreamSynchronize(st));
    return build_schedule(g, st);
  }

  // ---- A stream
  const uint64_t* xsrc = rp;  // offsets x_0..x_n: record index (global) or bit (local)
  uint64_t U = arcs;
  Tmp t_wid(st), t_len(st), t_x(st), t_stmp(st);
  if (g->id_mode == ID_GLOBAL) {
    g->bits_A = arcs * g->r;
    g->words_A = padded_words(g->bits_A);
    LG_TRY(alloc_words(&g->A, g->words_A, st));
    LG_TRY(enc_pack_global(cl, wt, arcs, g->s, g->omega, g->A, (g->bits_A + 63) / 64, st));
  } else {
    const int gap = g->id_mode == ID_LOCAL_GAP;
    LG_TRY(t_wid.alloc(n));
    LG_TRY(t_len.alloc(n * sizeof(uint64_t)));
    LG_TRY(t_x.alloc((n + 1) * sizeof(uint64_t)));
    LG_TRY(t_stmp.alloc(scan_tmp_words(n) * sizeof(uint64_t)));
    LG_TRY(enc_local_lengths(rp, cl, n, gap, g->s, g->H, t_wid.as<uint8_t>(), t_len.as<uint64_t>(), st));
    LG_TRY(scan_excl_u64(t_len.as<uint64_t>(), n, t_x.as<uint64_t>(), t_stmp.as<uint64_t>(), st));
    LG_TRY(cudaMemcpyAsync(&U, t_x.as<uint64_t>() + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    LG_TRY(cudaStreamSynchronize(st));
    g->bits_A = U;
    g->words_A = padded_words(g->bits_A);
    LG_TRY(alloc_words(&g->A, g->words_A, st));
    LG_TRY(enc_pack_local(rp, cl, t_x.as<uint64_t>(), t_wid.as<uint8_t>(), n, gap, g->s, g->H, g->A,
                          (g->bits_A + 63) / 64, st));
    xsrc = t_x.as<uint64_t>();
  }

  // ---- offsets (Section 3.4 packed, Section 4.3 Elias-Fano)
  if (g->off_mode == OFF_PACKED) {
    g->w_O = host_bits(U);
    if (g->w_O < 1) g->w_O = 1;
    g->bits_O = (n + 1) * (uint64_t)g->w_O;
    g->words_O = padded_words(g->bits_O);
    LG_TRY(alloc_words(&g->O, g->words_O, st));
    LG_TRY(enc_pack_u64(xsrc, n + 1, g->w_O, g->O, (g->bits_O + 63) / 64, st));
  } else {
    const uint64_t N = n + 1, q = U / N;
    g->ef_N = N; g->ef_U = U;
    g->ef_l = q ? host_bits(q) - 1 : 0;
    g->ef_low_bits = N * (uint64_t)g->ef_l;
    g->ef_high_bits = N + (U >> g->ef_l) + 1;
    g->n_samples = (N + g->sample - 1) / g->sample;
    g->words_ef_low = padded_words(g->ef_low_bits);
    g->words_ef_high = padded_words(g->ef_high_bits);
    g->words_ef_samples = padded_words(64 * g->n_samples);
    LG_TRY(alloc_words(&g->ef_low, g->words_ef_low, st));
    LG_TRY(alloc_words(&g->ef_high, g->words_ef_high, st));
    LG_TRY(alloc_words(&g->ef_samples, g->words_ef_samples, st));
    if (g->ef_l) LG_TRY(enc_pack_u64(xsrc, N, g->ef_l, g->ef_low, (g->ef_low_bits + 63) / 64, st));
    LG_TRY(enc_ef_high(xsrc, N, g->ef_l, g->ef_high, st));
    LG_TRY(enc_ef_samples(xsrc, N, g->ef_l, g->sample, g->ef_samples, g->n_samples, st));
    g->bits_O = g->ef_low_bits + g->ef_high_bits + 64 * g->n_samples;
  }
  LG_TRY(cudaStreamSynchronize(st));
  return build_schedule(g, st);
}

extern "C" lg_status lg_encode(const uint64_t* row_ptr, const uint32_t* col, const uint32_t* weights, uint64_t n,
                               uint64_t arcs, const lg_encode_opts* opts, void* stream, lg_graph** out) {
  g_err[0] = 0;
  if (!out) { set_errf("lg_encode: out is NULL"); return LG_EINVAL; }
  *out = nullptr;
  if (!row_ptr || (arcs && !col)) { set_errf("lg_encode: row_ptr/col is NULL"); return LG_EINVAL; }
  if (n == 0 || n > 0xffffffffull) { set_errf("lg_encode: n must be in [1, 2^32-1], got %llu", (unsigned long long)n); return LG_EINVAL; }
  if (arcs > 0xffffffffull * 0xffffull) { set_errf("lg_encode: arcs too large"); return LG_EINVAL; }
  lg_encode_opts o = {LG_ID_GLOBAL, LG_OFF_PACKED, 0, 512, 0, 0};
  if (opts) o = *opts;
  if (o.select_sample == 0) o.select_sample = 512;
  if (o.id_mode > LG_ID_CSR32 || o.off_mode > LG_OFF_EF) { set_errf("lg_encode: unknown id_mode/off_mode"); return LG_EINVAL; }
  if (o.select_sample < 64 || o.select_sample > 65536 || (o.select_sample & (o.select_sample - 1))) {
    set_errf("lg_encode: select_sample must be a power of two in [64, 65536]");
    return LG_EINVAL;
  }
  if (o.weight_bits > 32) { set_errf("lg_encode: weight_bits must be <= 32"); return LG_EINVAL; }
  if (o.relabel > 2) { set_errf("lg_encode: relabel must be 0, 1 (DM) or 2 (greedy)"); return LG_EINVAL; }
  if (weights && (o.id_mode == LG_ID_LOCAL || o.id_mode == LG_ID_LOCAL_GAP)) {
    set_errf("lg_encode: weights are supported with LG_ID_GLOBAL and LG_ID_CSR32 only");
    return LG_EUNSUPPORTED;
  }
  lg_graph* g = new (std::nothrow) lg_graph;
  if (!g) { set_errf("lg_encode: host allocation failed"); return LG_ENOMEM; }
  memset(g, 0, sizeof(*g));
  if (cudaGetDevice(&g->device) != cudaSuccess) { delete g; set_errf("lg_encode: no CUDA device"); return LG_ECUDA; }
  g->n = n; g->arcs = arcs;
  g->id_mode = o.id_mode; g->off_mode = o.off_mode; g->relabel = o.relabel; g->weighted = weights ? 1 : 0;
  g->sample = o.select_sample;
  g->sample_log2 = host_bits(o.select_sample) - 1;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  lg_status s = encode_impl(g, row_ptr, col, weights, o, st);
  if (s != LG_OK) {
    cudaStreamSynchronize(st);
    lg_free(g);
    return s;
  }
  *out = g;
  return LG_OK;
}

extern "C" lg_status lg_neighbors(const lg_graph* g, const uint32_t* vertices, uint64_t k, uint64_t* out_offsets,
                                  uint32_t* out_ids, uint32_t* out_weights, uint64_t out_capacity, void* stream) {
  g_err[0] = 0;
  if (!g || !out_offsets || (k && !vertices)) { set_errf("lg_neighbors: null argument"); return LG_EINVAL; }
  if (out_weights && !g->weighted) { set_errf("lg_neighbors: graph has no weights"); return LG_EINVAL; }
  DeviceGuard dg(g->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Tmp small(st), stmp(st);
  LG_TRY(small.alloc(16));
  LG_TRY(stmp.alloc(scan_tmp_words(k) * sizeof(uint64_t)));
  LG_TRY(cudaMemsetAsync(small.p, 0, 16, st));
  const GView v = make_view(g);
  const TravOps* ops = trav_ops((int)g->id_mode, (int)g->off_mode);
  NbrArgs a;
  a.vertices = vertices; a.k = k; a.out_offsets = out_offsets; a.out_ids = out_ids; a.out_weights = out_weights;
  a.err = small.as<int>();
  LG_TRY(ops->nbr_degrees(v, a, st));
  LG_TRY(scan_excl_u64(out_offsets, k, out_offsets, stmp.as<uint64_t>(), st));
  struct { int err; int pad; } he{};
  uint64_t total = 0;
  LG_TRY(cudaMemcpyAsync(&he, small.p, sizeof(he), cudaMemcpyDeviceToHost, st));
  LG_TRY(cudaMemcpyAsync(&total, out_offsets + k, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
  LG_TRY(cudaStreamSynchronize(st));
  if (he.err) return describe_dev_err(he.err);
  if (total > out_capacity) {
    set_errf("lg_neighbors: %llu neighbors do not fit out_capacity %llu", (unsigned long long)total,
             (unsigned long long)out_capacity);
    return LG_ERANGE;
  }
  if (total && !out_ids) { set_errf("lg_neighbors: out_ids is NULL"); return LG_EINVAL; }
  LG_TRY(ops->nbr_decode(v, a, st));
  if (g->relabel) LG_TRY(segmented_sort(out_ids, out_weights, out_offsets, k, total, g->max_degree, st));
  LG_TRY(cudaStreamSynchronize(st));
  return LG_OK;
}

extern "C" lg_status lg_bfs(const lg_graph* g, const uint32_t* sources, uint32_t S, uint32_t* depths, void* stream) {
  g_err[0] = 0;
  if (!g || (S && (!sources || !depths))) { set_errf("lg_bfs: null argument"); return LG_EINVAL; }
  if (S == 0) return LG_OK;
  DeviceGuard dg(g->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const uint64_t n = g->n;
  const uint32_t maxb = S >= 64 ? 64 : S;
  const int mb = maxb <= 16 ? 2 : (maxb <= 32 ? 4 : 8);
  Tmp t_src(st), t_vis(st), t_fa(st), t_fb(st), t_qa(st), t_qb(st), t_small(st), t_depth(st), t_hacc(st);
  LG_TRY(t_src.alloc(S * sizeof(uint32_t)));
  LG_TRY(t_vis.alloc(n * mb + 16));
  LG_TRY(t_fa.alloc(n * mb + 16));
  LG_TRY(t_fb.alloc(n * mb + 16));
  LG_TRY(t_qa.alloc(n * sizeof(uint32_t)));
  LG_TRY(t_qb.alloc(n * sizeof(uint32_t)));
  LG_TRY(t_small.alloc(64));
  if (g->relabel) LG_TRY(t_depth.alloc((uint64_t)maxb * n * sizeof(uint32_t)));
  LG_TRY(t_hacc.alloc(g->n_multi * mb + 16));
  LG_TRY(cudaMemsetAsync(t_hacc.p, 0, g->n_multi * mb + 16, st));
  int* d_err = t_small.as<int>();
  uint32_t* counters = reinterpret_cast<uint32_t*>(t_small.as<char>() + 16);
  LG_TRY(cudaMemsetAsync(t_small.p, 0, 64, st));
  LG_TRY(map_ids(sources, t_src.as<uint32_t>(), g->perm, S, n, d_err, st));
  int herr = 0;
  LG_TRY(cudaMemcpyAsync(&herr, d_err, 4, cudaMemcpyDeviceToHost, st));
  LG_TRY(cudaStreamSynchronize(st));
  if (herr) return describe_dev_err(herr);

  const GView v = make_view(g);
  const TravOps* ops = trav_ops((int)g->id_mode, (int)g->off_mode);
  const uint64_t pull_threshold = n / pull_divisor();
  for (uint32_t b0 = 0; b0 < S; b0 += 64) {
    const uint32_t Sb = (S - b0) < 64 ? (S - b0) : 64;
    uint32_t* depth_b = g->relabel ? t_depth.as<uint32_t>() : depths + (uint64_t)b0 * n;
    LG_TRY(cudaMemsetAsync(depth_b, 0xff, (uint64_t)Sb * n * sizeof(uint32_t), st));
    LG_TRY(cudaMemsetAsync(t_vis.p, 0, n * mb, st));
    LG_TRY(cudaMemsetAsync(t_fa.p, 0, n * mb, st));
    LG_TRY(cudaMemsetAsync(t_fb.p, 0, n * mb, st));
    LG_TRY(cudaMemsetAsync(counters, 0, 16, st));
    LG_TRY(bfs_seed(t_vis.p, t_fa.p, depth_b, n, t_src.as<uint32_t>() + b0, Sb, g->relabel ? 1u : 0u, mb,
                    t_qa.as<uint32_t>(), counters, st));
    uint32_t hc[2] = {0, 0};
    LG_TRY(cudaMemcpyAsync(hc, counters, 8, cudaMemcpyDeviceToHost, st));
    LG_TRY(cudaStreamSynchronize(st));
    uint32_t nq = hc[0];
    void* cur = t_fa.p;
    void* nxt = t_fb.p;
    uint32_t* qcur = t_qa.as<uint32_t>();
    uint32_t* qnxt = t_qb.as<uint32_t>();
    BfsArgs a;
    memset(&a, 0, sizeof(a));
    a.vis = t_vis.p;
    a.depth = depth_b;
    a.all_mask = Sb == 64 ? ~0ull : ((1ull << Sb) - 1ull);
    a.S = Sb;
    a.vmajor = g->relabel ? 1u : 0u;  // relabeled depths are permuted afterwards
    a.counters = counters;
    a.hacc = t_hacc.p;
    a.err = d_err;
    a.hot = hot_rows(g, mb);
    for (uint32_t level = 0; nq > 0; level++) {
      LG_TRY(cudaMemsetAsync(counters, 0, 8, st));
      a.front_in = cur; a.front_out = nxt; a.level = level;
      a.queue_in = qcur; a.queue_in_len = nq; a.queue_out = qnxt;
      if ((uint64_t)nq > pull_threshold) {
        LG_TRY(ops->bfs_pull(v, a, mb, st));
        LG_TRY(bfs_finish_multi(v, a, mb, st));
      } else {
        LG_TRY(ops->bfs_push(v, a, mb, st));
      }
      LG_TRY(cudaMemcpyAsync(hc, counters, 8, cudaMemcpyDeviceToHost, st));
      // the frontier just consumed becomes the next output buffer: clear it
      if ((uint64_t)nq * 16 < n) {
        k_clear_queue<<<grid_for(nq, 256, 4096), 256, 0, st>>>(reinterpret_cast<uint8_t*>(cur), mb, qcur, nq);
        count_launch();
        LG_TRY(cudaGetLastError());
      } else {
        LG_TRY(cudaMemsetAsync(cur, 0, n * mb, st));
      }
      LG_TRY(cudaStreamSynchronize(st));
      void* t = cur; cur = nxt; nxt = t;
      uint32_t* tq = qcur; qcur = qnxt; qnxt = tq;
      nq = hc[0];
    }
    if (g->relabel) LG_TRY(bfs_permute_depths(depth_b, depths + (uint64_t)b0 * n, g->perm, n, Sb, st));
  }
  LG_TRY(cudaStreamSynchronize(st));
  return LG_OK;
}

extern "C" lg_status lg_pagerank(const lg_graph* g, float damping, uint32_t iters, const uint32_t* personalize_source,
                                 float* ranks, void* stream) {
  g_err[0] = 0;
  if (!g || !ranks) { set_errf("lg_pagerank: null argument"); return LG_EINVAL; }
  if (!(damping >= 0.0f && damping <= 1.0f)) { set_errf("lg_pagerank: damping must be in [0, 1]"); return LG_EINVAL; }
  int64_t personal_orig = -1, personal = -1;
  if (personalize_source) {
    if (*personalize_source >= g->n) { set_errf("lg_pagerank: personalize_source >= n"); return LG_EINVAL; }
    personal_orig = *personalize_source;
  }
  DeviceGuard dg(g->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const uint64_t n = g->n;
  if (iters == 0) {
    LG_TRY(pr_fill0(ranks, n, personal_orig, st));
    return LG_OK;
  }
  if (personal_orig >= 0) {
    if (g->perm) {
      uint32_t ps = 0;
      LG_TRY(cudaMemcpyAsync(&ps, g->perm + personal_orig, 4, cudaMemcpyDeviceToHost, st));
      LG_TRY(cudaStreamSynchronize(st));
      personal = ps;
    } else {
      personal = personal_orig;
    }
  }
  Tmp ca(st), cb(st), tpart(st);
  LG_TRY(ca.alloc(n * sizeof(float)));
  LG_TRY(cb.alloc(n * sizeof(float)));
  if (g->n_multi) LG_TRY(tpart.alloc(g->n_items * sizeof(float)));
  const GView v = make_view(g);
  const TravOps* ops = trav_ops((int)g->id_mode, (int)g->off_mode);
  PrArgs a;
  memset(&a, 0, sizeof(a));
  a.damp = damping;
  a.personal = personal;
  a.base_all = personal < 0 ? (1.0f - damping) / (float)n : (1.0f - damping);
  a.r0_all = 1.0f / (float)n;
  a.part = tpart.as<float>();
  a.ranks_out = ranks;
  a.contrib_out = ca.as<float>();
  a.hot = hot_rows(g, sizeof(float));
  LG_TRY(ops->pr_init(v, a, st));
  float* cur = ca.as<float>();
  float* nxt = cb.as<float>();
  for (uint32_t t = 0; t < iters; t++) {
    a.contrib_in = cur;
    a.contrib_out = nxt;
    a.last = (t + 1 == iters);
    LG_TRY(ops->pr_pull(v, a, st));
    LG_TRY(pr_finish_multi(v, a, st));
    float* tt = cur; cur = nxt; nxt = tt;
  }
  return LG_OK;
}
