// GPU side of the seeded input generator (inputs only; no Log(Graph) arithmetic).
//
// Draws the same R-MAT edges as lggen.c (per-edge SplitMix64 key, one draw per
// two levels, the host's Fisher-Yates label table) and builds the symmetric CSR
// on the device for graphs too large to build quickly on the host: degree
// count, scatter of both arcs of every non-loop edge, and the per-arc weight
// hash.  Row sorting, deduplication and prefix sums are done by the caller.
#include <cstdint>
#include <cuda_runtime.h>

namespace {

__device__ __forceinline__ uint64_t sm64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t h4(uint64_t seed, uint64_t stream, uint64_t i, uint64_t j) {
  return sm64(sm64(sm64(sm64(seed) ^ stream) ^ i) ^ j);
}
constexpr uint64_t ST_RMAT = 1, ST_WEIGHT = 3;

struct RmatParams {
  uint64_t seed, m;
  int scale;
  double a, ab, abc;
  const uint32_t* perm;  // n labels (nullptr: identity)
};

__device__ __forceinline__ void rmat_edge(const RmatParams& p, uint64_t e, uint32_t& u, uint32_t& v) {
  uint64_t s = 0, d = 0, h = 0;
  const uint64_t key = h4(p.seed, ST_RMAT, e, 0);
  for (int k = 0; k < p.scale; k++) {
    if ((k & 1) == 0) h = sm64(key + (uint64_t)k);
    const uint32_t r32 = (k & 1) ? (uint32_t)h : (uint32_t)(h >> 32);
    const double x = (double)r32 * (1.0 / 4294967296.0);
    uint64_t sb, db;
    if (x < p.a) { sb = 0; db = 0; }
    else if (x < p.ab) { sb = 0; db = 1; }
    else if (x < p.abc) { sb = 1; db = 0; }
    else { sb = 1; db = 1; }
    s = (s << 1) | sb;
    d = (d << 1) | db;
  }
  u = p.perm ? p.perm[s] : (uint32_t)s;
  v = p.perm ? p.perm[d] : (uint32_t)d;
}

__global__ void k_count(RmatParams p, unsigned long long* deg) {
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < p.m; e += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t u, v;
    rmat_edge(p, e, u, v);
    if (u != v) {
      atomicAdd(&deg[u], 1ull);
      atomicAdd(&deg[v], 1ull);
    }
  }
}

__global__ void k_scatter(RmatParams p, unsigned long long* cursor, uint32_t* col) {
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < p.m; e += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t u, v;
    rmat_edge(p, e, u, v);
    if (u != v) {
      col[atomicAdd(&cursor[u], 1ull)] = v;
      col[atomicAdd(&cursor[v], 1ull)] = u;
    }
  }
}

// weight of arc (row, col[j]) = 1 + hash(seed, min, max) mod 255; one warp per row
__global__ void k_weights(const uint64_t* rp, const uint32_t* col, uint64_t n, uint64_t seed, uint32_t* w) {
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t v = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); v < n; v += warps) {
    for (uint64_t j = rp[v] + (threadIdx.x & 31); j < rp[v + 1]; j += 32) {
      const uint64_t a = v, b = col[j];
      const uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
      w[j] = 1u + (uint32_t)(h4(seed, ST_WEIGHT, lo, hi) % 255u);
    }
  }
}

// Batches: edge e of the whole batch belongs to graph g with
// ebase[g] <= e < ebase[g+1]; graph g draws its local edge e - ebase[g] with its
// own seed, scale and label table, and its vertices sit at vbase[g] onward.
struct BatchGen {
  const uint64_t* ebase;  // count+1
  const uint64_t* vbase;  // count
  const uint64_t* seeds;  // count
  const int32_t* scales;  // count
  const uint64_t* pbase;  // count: first entry of the graph's label table
  const uint32_t* perms;
  uint32_t count;
  double a, ab, abc;
};

__device__ __forceinline__ uint32_t batch_graph_of(const BatchGen& b, uint64_t e) {
  uint32_t lo = 0, hi = b.count;  // largest g with ebase[g] <= e
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (b.ebase[mid] <= e) lo = mid; else hi = mid;
  }
  return lo;
}

template <bool SCATTER>
__global__ void k_batch_edges(BatchGen b, unsigned long long* deg_or_cursor, uint32_t* col) {
  const uint64_t M = b.ebase[b.count];
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < M; e += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t g = batch_graph_of(b, e);
    RmatParams p{b.seeds[g], b.ebase[g + 1] - b.ebase[g], b.scales[g], b.a, b.ab, b.abc, b.perms + b.pbase[g]};
    uint32_t u, v;
    rmat_edge(p, e - b.ebase[g], u, v);
    if (u == v) continue;
    const uint64_t vb = b.vbase[g];
    if (SCATTER) {
      col[atomicAdd(&deg_or_cursor[vb + u], 1ull)] = v;
      col[atomicAdd(&deg_or_cursor[vb + v], 1ull)] = u;
    } else {
      atomicAdd(&deg_or_cursor[vb + u], 1ull);
      atomicAdd(&deg_or_cursor[vb + v], 1ull);
    }
  }
}

}  // namespace

extern "C" int lggen_gpu_batch_edges(int scatter, const uint64_t* ebase, const uint64_t* vbase,
                                     const uint64_t* seeds, const int32_t* scales, const uint64_t* pbase,
                                     const uint32_t* perms, uint32_t count, double a, double ab, double abc,
                                     unsigned long long* deg_or_cursor, uint32_t* col, void* stream) {
  BatchGen b{ebase, vbase, seeds, scales, pbase, perms, count, a, ab, abc};
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (scatter) k_batch_edges<true><<<152 * 32, 256, 0, st>>>(b, deg_or_cursor, col);
  else k_batch_edges<false><<<152 * 32, 256, 0, st>>>(b, deg_or_cursor, col);
  return (int)cudaGetLastError();
}

extern "C" int lggen_gpu_rmat_count(int scale, uint64_t m, double a, double ab, double abc, uint64_t seed,
                                    const uint32_t* perm, unsigned long long* deg, void* stream) {
  RmatParams p{seed, m, scale, a, ab, abc, perm};
  k_count<<<152 * 32, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(p, deg);
  return (int)cudaGetLastError();
}

extern "C" int lggen_gpu_rmat_scatter(int scale, uint64_t m, double a, double ab, double abc, uint64_t seed,
                                      const uint32_t* perm, unsigned long long* cursor, uint32_t* col, void* stream) {
  RmatParams p{seed, m, scale, a, ab, abc, perm};
  k_scatter<<<152 * 32, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(p, cursor, col);
  return (int)cudaGetLastError();
}

extern "C" int lggen_gpu_weights(const uint64_t* rp, const uint32_t* col, uint64_t n, uint64_t seed, uint32_t* w,
                                 void* stream) {
  k_weights<<<152 * 32, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(rp, col, n, seed, w);
  return (int)cudaGetLastError();
}
