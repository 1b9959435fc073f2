// Single-source shortest paths on the weighted compressed graph (Section
// 7.1.2: SSSP by delta-stepping; weights stored at omega bits right after each
// ID, Section 3.3).
//
// A GPU form of delta-stepping ("near / far" piles):
//   * bucket [lo, lo + delta) is processed in rounds: the arcs of the near
//     queue are spread evenly over warps, each lane decoding its arc's neighbor
//     and weight from the compressed stream and lowering dist[u] with
//     atomicMin; a vertex improved to a distance below
//     lo + delta joins the next round's near queue (a per-round stamp keeps
//     one entry per vertex), any other improved vertex joins the far list (a
//     per-bucket stamp keeps one entry per vertex, so the list never exceeds n);
//   * when a round leaves the near queue empty, the far list is reduced to its
//     smallest live distance, the next non-empty bucket starts there, and the
//     far list is split into that bucket's near queue and the rest.
// Distances are integers (sums of stored weights), so the result is the exact
// shortest-path distance whatever the order of relaxations.
#include <cstdio>
#include <cstring>
#include <utility>

#include "lg_traverse.cuh"

namespace lg {

constexpr uint64_t DINF = ~0ull;

struct SsspArgs {
  unsigned long long* dist;  // n, stored labels
  const uint32_t* near_in;
  uint32_t near_len;
  uint32_t* near_out;
  uint32_t* far;              // far list (append)
  uint32_t* stamp_near;       // per vertex: last round it was queued for
  uint32_t* stamp_far;        // per vertex: last bucket it was put in the far list
  uint32_t round, bucket;
  uint64_t hi;                // upper end of the current bucket
  uint32_t* counters;         // [0] near_out length, [1] far length
  int* err;
};

__device__ __forceinline__ uint32_t arc_weight(const GView& g, int idm, uint64_t start, uint64_t i) {
  if (idm == ID_CSR32) return g.W32 ? __ldg(g.W32 + (start >> 5) + i) : 1u;
  return g.omega ? ext32(g.A32, start + i * g.r + g.s, g.omega) : 1u;
}

// Edge-balanced relaxation.  Per round: the degree and first-field bit of
// every near vertex, an exclusive scan of the degrees (eoff[near_len] = the
// round's arcs E), then warps take 256 consecutive arc slots at a time; lane l
// relaxes slots c + l, c + l + 32, ...: its near vertex q is the last with
// eoff[q] <= slot (found once per chunk, then advanced), its field index is
// slot - eoff[q].  Hubs are spread over as many warps as their arcs need.
template <int IDM, int OFF>
__global__ void __launch_bounds__(256) k_sssp_degrees(GView g, const uint32_t* near, uint32_t len, uint64_t* eoff,
                                                      uint64_t* start) {
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t q = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < len; q += warps) {
    uint64_t x0, x1, st;
    uint32_t d, w;
    offset_pair<OFF>(g, near[q], x0, x1);
    vgeo<IDM>(g, x0, x1, st, d, w);
    if ((threadIdx.x & 31) == 0) {
      eoff[q] = d;
      start[q] = st;
    }
  }
}

template <int IDM>
__global__ void __launch_bounds__(256) k_sssp_relax_lb(GView g, SsspArgs a, const uint64_t* eoff,
                                                       const uint64_t* start) {
  constexpr uint32_t CH = 256;  // arc slots per warp chunk
  const int lane = threadIdx.x & 31;
  const uint64_t E = eoff[a.near_len];
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t c = ((uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * CH; c < E; c += warps * CH) {
    // near vertex holding slot c + lane: last q with eoff[q] <= slot
    const uint64_t first = c + lane;
    uint32_t lo = 0, hi = a.near_len - 1;
    while (lo < hi) {
      const uint32_t m = (lo + hi + 1) >> 1;
      if (eoff[m] <= first) lo = m; else hi = m - 1;
    }
    uint32_t q = lo;
    // Distances are read with ordinary (L1-cached) loads: they only decrease,
    // so a stale value is never below the true one; a stale dist[u] only costs
    // an atomicMin that changes nothing, and a stale dist[v] only weakens one
    // relaxation -- a vertex improved during a round is queued again, and the
    // next round is a new launch that sees the new value.
    // The chunk runs in phases so that each lane has its 8 slots' loads in
    // flight together: decode all, load all distances, then the atomics.
    constexpr int S = CH / 32;
    uint32_t uu[S];
    uint64_t nd[S];
    uint32_t qv = 0xffffffffu;
    uint64_t dv = 0, st = 0;
#pragma unroll
    for (int t = 0; t < S; t++) {
      const uint64_t slot = c + lane + 32u * t;
      uu[t] = 0xffffffffu;
      nd[t] = DINF;
      if (slot < E) {
        while (eoff[q + 1] <= slot) q++;
        if (q != qv) {  // a new near vertex for this lane
          qv = q;
          dv = a.dist[a.near_in[q]];
          st = start[q];
        }
        const uint64_t k = slot - eoff[q];
        uu[t] = IDM == ID_CSR32 ? __ldg(g.A32 + (st >> 5) + k) : ext32(g.A32, st + k * g.r, g.s);
        nd[t] = dv + arc_weight(g, IDM, st, k);
      }
    }
    uint64_t du[S];
#pragma unroll
    for (int t = 0; t < S; t++) du[t] = uu[t] != 0xffffffffu ? a.dist[uu[t]] : 0;
    // all atomics of the chunk are issued before any result is used
#pragma unroll
    for (int t = 0; t < S; t++)
      du[t] = (uu[t] != 0xffffffffu && nd[t] < du[t]) ? atomicMin(a.dist + uu[t], (unsigned long long)nd[t]) : 0;
    uint32_t stamp_old[S];
#pragma unroll
    for (int t = 0; t < S; t++) {
      stamp_old[t] = 0;
      if (nd[t] < du[t]) {  // improved (du now holds the value before the atomicMin)
        stamp_old[t] = nd[t] < a.hi ? atomicExch(a.stamp_near + uu[t], a.round)
                                    : atomicExch(a.stamp_far + uu[t], a.bucket);
      }
    }
    uint32_t near_bits = 0, far_bits = 0;
#pragma unroll
    for (int t = 0; t < S; t++) {
      if (nd[t] < du[t]) {
        if (nd[t] < a.hi) {
          if (stamp_old[t] != a.round) near_bits |= 1u << t;
        } else if (stamp_old[t] != a.bucket) {
          far_bits |= 1u << t;
        }
      }
    }
    // one warp-aggregated append per list
    const uint32_t cn = __popc(near_bits), cf = __popc(far_bits);
    const uint32_t in = warp_incl_scan<uint32_t>(cn), inf = warp_incl_scan<uint32_t>(cf);
    uint32_t bn = 0, bf = 0;
    if (lane == 31) {
      if (in) bn = atomicAdd(&a.counters[0], in);
      if (inf) bf = atomicAdd(&a.counters[1], inf);
    }
    bn = __shfl_sync(LG_FULL_MASK, bn, 31) + in - cn;
    bf = __shfl_sync(LG_FULL_MASK, bf, 31) + inf - cf;
#pragma unroll
    for (int t = 0; t < S; t++) {
      if ((near_bits >> t) & 1u) a.near_out[bn++] = uu[t];
      if ((far_bits >> t) & 1u) a.far[bf++] = uu[t];
    }
  }
}

// smallest distance among far entries that are still at or above `lo`
__global__ void k_far_min(const uint32_t* far, uint32_t len, const unsigned long long* dist, uint64_t lo,
                          unsigned long long* out) {
  uint64_t m = DINF;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x) {
    const uint64_t d = dist[far[i]];
    if (d >= lo && d < m) m = d;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t y = __shfl_xor_sync(LG_FULL_MASK, m, o);
    m = y < m ? y : m;
  }
  if ((threadIdx.x & 31) == 0 && m != DINF) atomicMin(out, (unsigned long long)m);
}

// split the far list at the new bucket [lo, hi): entries inside go to the near
// queue (once per vertex), entries above stay far (once per vertex), entries
// below lo were settled in an earlier bucket and are dropped
__global__ void k_far_split(const uint32_t* far, uint32_t len, const unsigned long long* dist, uint64_t lo,
                            uint64_t hi, uint32_t* near_out, uint32_t* far_out, uint32_t* stamp_near,
                            uint32_t* stamp_far, uint32_t round, uint32_t bucket, uint32_t* counters) {
  const int lane = threadIdx.x & 31;
  for (uint32_t base = blockIdx.x * blockDim.x; base < len; base += gridDim.x * blockDim.x) {
    const uint32_t i = base + threadIdx.x;
    bool tn = false, tf = false;
    uint32_t v = 0;
    if (i < len) {
      v = far[i];
      const uint64_t d = dist[v];
      if (d >= lo && d < hi) tn = atomicExch(stamp_near + v, round) != round;
      else if (d >= hi) tf = atomicExch(stamp_far + v, bucket) != bucket;
    }
    const uint32_t bn = __ballot_sync(LG_FULL_MASK, tn), bf = __ballot_sync(LG_FULL_MASK, tf);
    uint32_t pn = 0, pf = 0;
    if (lane == 0) {
      if (bn) pn = atomicAdd(&counters[0], (uint32_t)__popc(bn));
      if (bf) pf = atomicAdd(&counters[1], (uint32_t)__popc(bf));
    }
    pn = __shfl_sync(LG_FULL_MASK, pn, 0);
    pf = __shfl_sync(LG_FULL_MASK, pf, 0);
    const uint32_t below = lane_lt_mask();
    if (tn) near_out[pn + __popc(bn & below)] = v;
    if (tf) far_out[pf + __popc(bf & below)] = v;
  }
}

__global__ void k_sssp_init(unsigned long long* dist, uint32_t* s_near, uint32_t* s_far, uint64_t n,
                            const uint32_t* perm, uint32_t src, uint32_t* near, uint32_t* src_stored) {
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
    dist[v] = DINF;
    s_near[v] = 0xffffffffu;
    s_far[v] = 0xffffffffu;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const uint32_t s = perm ? perm[src] : src;
    *src_stored = s;
    near[0] = s;
  }
}

__global__ void k_sssp_seed(unsigned long long* dist, const uint32_t* src_stored) { dist[*src_stored] = 0; }

// distances back to original IDs: out[v] = dist[perm[v]]
__global__ void k_sssp_unpermute(const unsigned long long* dist, const uint32_t* perm, uint64_t n, uint64_t* out) {
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x)
    out[v] = dist[perm[v]];
}

// degrees, scan, edge-balanced relaxation (even a single near vertex can be a
// hub with 10^5 arcs, so every round is balanced by arcs)
template <int IDM, int OFF>
cudaError_t launch_sssp_relax(const GView& g, const SsspArgs& a, uint64_t* eoff, uint64_t* start, uint64_t* tmp,
                              cudaStream_t st) {
  if (a.near_len == 0) return cudaSuccess;
  k_sssp_degrees<IDM, OFF><<<grid_for(a.near_len, 8, 152 * 16), 256, 0, st>>>(g, a.near_in, a.near_len, eoff, start);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = scan_excl_u64(eoff, a.near_len, eoff, tmp, st);
  if (e != cudaSuccess) return e;
  k_sssp_relax_lb<IDM><<<152 * 8, 256, 0, st>>>(g, a, eoff, start);
  count_launch();
  return cudaGetLastError();
}

}  // namespace lg

using namespace lg;

namespace {

struct DevBuf {
  void* p = nullptr;
  cudaStream_t st;
  explicit DevBuf(cudaStream_t s) : st(s) {}
  ~DevBuf() {
    if (p) cudaFreeAsync(p, st);
  }
  cudaError_t alloc(size_t b) { return lg::pool_alloc(&p, b, st); }
  template <typename T>
  T* as() const {
    return reinterpret_cast<T*>(p);
  }
};

lg_status fail(const char* what, cudaError_t e) {
  char msg[256];
  snprintf(msg, sizeof msg, "%s: %s", what, cudaGetErrorString(e));
  set_error_message(msg);
  return e == cudaErrorMemoryAllocation ? LG_ENOMEM : LG_ECUDA;
}
#define STRY(call)                                 \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return fail(#call, e_); \
  } while (0)

}  // namespace

extern "C" lg_status lg_sssp(const lg_graph* g, uint32_t source, uint64_t delta, uint64_t* dist, void* stream) {
  set_error_message("");
  if (!g || !dist) {
    set_error_message("lg_sssp: null argument");
    return LG_EINVAL;
  }
  if (source >= g->n) {
    set_error_message("lg_sssp: source >= n");
    return LG_EINVAL;
  }
  if (!g->weighted) {
    set_error_message("lg_sssp: the graph has no weights (encode with weights, global IDs or CSR-32)");
    return LG_EUNSUPPORTED;
  }
  if (g->id_mode != ID_GLOBAL && g->id_mode != ID_CSR32) {
    set_error_message("lg_sssp: weights exist only in global-ID and CSR-32 graphs");
    return LG_EUNSUPPORTED;
  }
  if (delta == 0) delta = 32;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != g->device) cudaSetDevice(g->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const uint64_t n = g->n;
  const GView v = make_view(g);
  lg_status status = LG_OK;
  do {
    DevBuf tdist(st), sn(st), sf(st), na(st), nb(st), fa(st), fb(st), small(st), eo(st), sb(st), tmp(st);
    unsigned long long* d = reinterpret_cast<unsigned long long*>(dist);
    if (g->perm) {
      if ((status = tdist.alloc(n * 8) == cudaSuccess ? LG_OK : LG_ENOMEM) != LG_OK) break;
      d = tdist.as<unsigned long long>();
    }
    cudaError_t e = sn.alloc(n * 4 + 16);
    if (e == cudaSuccess) e = sf.alloc(n * 4 + 16);
    if (e == cudaSuccess) e = na.alloc(n * 4 + 16);
    if (e == cudaSuccess) e = nb.alloc(n * 4 + 16);
    if (e == cudaSuccess) e = fa.alloc(n * 4 + 16);
    if (e == cudaSuccess) e = fb.alloc(n * 4 + 16);
    if (e == cudaSuccess) e = small.alloc(64);
    if (e == cudaSuccess) e = eo.alloc((n + 1) * 8 + 16);
    if (e == cudaSuccess) e = sb.alloc(n * 8 + 16);
    if (e == cudaSuccess) e = tmp.alloc(scan_tmp_words(n) * 8 + 16);
    if (e != cudaSuccess) {
      status = fail("lg_sssp: scratch", e);
      break;
    }
    uint32_t* counters = small.as<uint32_t>();
    unsigned long long* dmin = reinterpret_cast<unsigned long long*>(small.as<char>() + 16);
    uint32_t* src_stored = small.as<uint32_t>() + 8;
    k_sssp_init<<<grid_for(n, 256, 152 * 32), 256, 0, st>>>(d, sn.as<uint32_t>(), sf.as<uint32_t>(), n, g->perm,
                                                            source, na.as<uint32_t>(), src_stored);
    count_launch();
    k_sssp_seed<<<1, 1, 0, st>>>(d, src_stored);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) {
      status = fail("lg_sssp: init", e);
      break;
    }
    uint32_t* near_in = na.as<uint32_t>();
    uint32_t* near_out = nb.as<uint32_t>();
    uint32_t* far = fa.as<uint32_t>();
    uint32_t* far_alt = fb.as<uint32_t>();
    uint32_t near_len = 1, far_len = 0, round = 0, bucket = 0;
    uint64_t lo = 0, hi = delta;
    uint32_t hc[2] = {0, 0};
    uint64_t hmin = 0;
    SsspArgs a;
    memset(&a, 0, sizeof(a));
    a.dist = d;
    a.stamp_near = sn.as<uint32_t>();
    a.stamp_far = sf.as<uint32_t>();
    a.counters = counters;
    const uint64_t max_steps = 4 * n + 64;  // every step settles or moves work; this only bounds a bug
    uint64_t steps = 0;
    for (;;) {
      if (++steps > max_steps) {
        set_error_message("lg_sssp: no progress (internal error)");
        status = LG_ECUDA;
        break;
      }
      if (near_len) {
        // one round of the current bucket: next near queue into near_out, far appended after far_len
        round++;
        hc[0] = 0;
        hc[1] = far_len;
        if ((e = cudaMemcpyAsync(counters, hc, 8, cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
        a.near_in = near_in;
        a.near_len = near_len;
        a.near_out = near_out;
        a.far = far;
        a.round = round;
        a.bucket = bucket;
        a.hi = hi;
        uint64_t* eoff = eo.as<uint64_t>();
        uint64_t* sbit = sb.as<uint64_t>();
        uint64_t* stmp = tmp.as<uint64_t>();
        if (g->id_mode == ID_CSR32) e = launch_sssp_relax<ID_CSR32, OFF_ROWPTR>(v, a, eoff, sbit, stmp, st);
        else if (g->off_mode == OFF_EF) e = launch_sssp_relax<ID_GLOBAL, OFF_EF>(v, a, eoff, sbit, stmp, st);
        else e = launch_sssp_relax<ID_GLOBAL, OFF_PACKED>(v, a, eoff, sbit, stmp, st);
        if (e != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(hc, counters, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
        near_len = hc[0];
        far_len = hc[1];
        std::swap(near_in, near_out);
        continue;
      }
      if (far_len == 0) break;  // done
      // next non-empty bucket: the smallest far distance at or above hi
      hmin = DINF;
      if ((e = cudaMemcpyAsync(dmin, &hmin, 8, cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
      k_far_min<<<grid_for(far_len, 256, 152 * 8), 256, 0, st>>>(far, far_len, d, hi, dmin);
      count_launch();
      if ((e = cudaGetLastError()) != cudaSuccess) break;
      if ((e = cudaMemcpyAsync(&hmin, dmin, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
      if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
      if (hmin == DINF) break;  // every far entry was settled: done
      lo = hmin / delta * delta;
      hi = lo + delta;
      round++;
      bucket++;
      hc[0] = 0;
      hc[1] = 0;
      if ((e = cudaMemcpyAsync(counters, hc, 8, cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
      k_far_split<<<grid_for(far_len, 256, 152 * 8), 256, 0, st>>>(far, far_len, d, lo, hi, near_in, far_alt,
                                                                   a.stamp_near, a.stamp_far, round, bucket,
                                                                   counters);
      count_launch();
      if ((e = cudaGetLastError()) != cudaSuccess) break;
      if ((e = cudaMemcpyAsync(hc, counters, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
      if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
      near_len = hc[0];
      far_len = hc[1];
      std::swap(far, far_alt);
    }
    if (status == LG_OK && e != cudaSuccess) status = fail("lg_sssp", e);
    if (status == LG_OK && g->perm) {
      k_sssp_unpermute<<<grid_for(n, 256, 152 * 32), 256, 0, st>>>(d, g->perm, n, dist);
      count_launch();
      if ((e = cudaGetLastError()) != cudaSuccess) status = fail("lg_sssp: unpermute", e);
    }
    if (status == LG_OK && (e = cudaStreamSynchronize(st)) != cudaSuccess) status = fail("lg_sssp", e);
  } while (0);
  if (prev != g->device) cudaSetDevice(prev);
  return status;
}
