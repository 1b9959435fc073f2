// Sorting used by the encoder: a stable LSD radix sort (8-bit digits) of
// (key, value) pairs, the DM permuter of Section 5.6 (vertices ordered by
// degree descending, ties by original ID) built on it, and a segmented sort of
// CSR rows (the relabeled neighborhoods must be sorted again, Section 2.3).
#include "lg_internal.h"

namespace lg {

// =========================================================================
// stable LSD radix sort
// =========================================================================
constexpr int RS_NT = 256;
constexpr int RS_ROUNDS = 16;
constexpr int RS_TILE = RS_NT * RS_ROUNDS;  // keys per CTA
constexpr int RS_NW = RS_NT / 32;

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <typename K>
__global__ void __launch_bounds__(RS_NT) k_rs_hist(const K* __restrict__ keys, uint64_t n, uint32_t shift,
                                                   uint32_t* __restrict__ hist, uint64_t ntiles) {
  __shared__ uint32_t cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const uint64_t base = (uint64_t)blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_ROUNDS; r++) {
    const uint64_t i = base + (uint64_t)r * RS_NT + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(uint32_t)(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(uint64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];  // digit-major
}

template <typename K>
__global__ void __launch_bounds__(RS_NT) k_rs_scatter(const K* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                      K* __restrict__ kout, uint32_t* __restrict__ vout, uint64_t n,
                                                      uint32_t shift, const uint64_t* __restrict__ off,
                                                      uint64_t ntiles) {
  __shared__ uint32_t wcnt[RS_NW][256];
  __shared__ uint64_t run[256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  run[threadIdx.x] = off[(uint64_t)threadIdx.x * ntiles + blockIdx.x];
  const uint64_t base = (uint64_t)blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_ROUNDS; r++) {
    for (int k = 0; k < RS_NW; k++) wcnt[k][threadIdx.x] = 0;
    __syncthreads();
    const uint64_t i = base + (uint64_t)r * RS_NT + threadIdx.x;
    const bool ok = i < n;
    K key = ok ? kin[i] : K(0);
    const uint32_t val = (ok && vin) ? vin[i] : 0u;
    const uint32_t dig = ok ? ((uint32_t)(key >> shift) & 255u) : 256u;
    const uint32_t peers = __match_any_sync(LG_FULL_MASK, dig);
    const uint32_t rank = __popc(peers & lanemask_lt());
    if (ok && rank == 0) wcnt[w][dig] = __popc(peers);
    __syncthreads();
    // thread t owns digit t: exclusive prefix over warps, then advance the run
    {
      uint32_t acc = 0;
      for (int k = 0; k < RS_NW; k++) {
        const uint32_t c = wcnt[k][threadIdx.x];
        wcnt[k][threadIdx.x] = acc;
        acc += c;
      }
      // read run before updating: positions use the old value
      __syncthreads();
      if (ok) {
        const uint64_t pos = run[dig] + wcnt[w][dig] + rank;
        kout[pos] = key;
        if (vin) vout[pos] = val;
      }
      __syncthreads();
      run[threadIdx.x] += acc;
    }
    __syncthreads();
  }
  (void)lane;
}

size_t radix_tmp_bytes(uint64_t n) {
  const uint64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
  const uint64_t cells = 256 * ntiles;
  return cells * sizeof(uint32_t) + (cells + 1) * sizeof(uint64_t) + scan_tmp_words(cells) * sizeof(uint64_t) + 256;
}

template <typename K>
static cudaError_t radix_impl(K* keys, uint32_t* vals, K* keys_alt, uint32_t* vals_alt, uint64_t n,
                              uint32_t key_bits, void* tmp, cudaStream_t st) {
  if (n <= 1 || key_bits == 0) return cudaSuccess;
  const uint64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
  const uint64_t cells = 256 * ntiles;
  uint32_t* hist = reinterpret_cast<uint32_t*>(tmp);
  uint64_t* off = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(tmp) + ((cells * 4 + 15) & ~15ull));
  uint64_t* stmp = off + cells + 2;
  K* ka = keys; K* kb = keys_alt;
  uint32_t* va = vals; uint32_t* vb = vals_alt;
  const uint32_t passes = (key_bits + 7) / 8;
  for (uint32_t p = 0; p < passes; p++) {
    const uint32_t shift = 8 * p;
    k_rs_hist<K><<<(unsigned)ntiles, RS_NT, 0, st>>>(ka, n, shift, hist, ntiles);
    count_launch();
    cudaError_t e = scan_excl_u32(hist, cells, off, stmp, st);
    if (e != cudaSuccess) return e;
    k_rs_scatter<K><<<(unsigned)ntiles, RS_NT, 0, st>>>(ka, va, kb, vb, n, shift, off, ntiles);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    K* t = ka; ka = kb; kb = t;
    uint32_t* tv = va; va = vb; vb = tv;
  }
  if (ka != keys) {
    cudaError_t e = cudaMemcpyAsync(keys, ka, n * sizeof(K), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    if (vals) e = cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

cudaError_t radix_sort_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt, uint64_t n,
                           uint32_t key_bits, void* tmp, cudaStream_t st) {
  return radix_impl<uint32_t>(keys, vals, keys_alt, vals_alt, n, key_bits, tmp, st);
}
cudaError_t radix_sort_u64(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt, uint64_t n,
                           uint32_t key_bits, void* tmp, cudaStream_t st) {
  return radix_impl<uint64_t>(keys, vals, keys_alt, vals_alt, n, key_bits, tmp, st);
}

// =========================================================================
// segmented sort of CSR rows
// =========================================================================
constexpr uint32_t SEG_SMALL = 32;    // one warp per row, bitonic network in registers
constexpr uint32_t SEG_MEDIUM = 8192; // one CTA per row, bitonic in shared memory

// bitonic sort of each aligned group of W lanes (ascending within the group)
template <int W, bool VALS>
__device__ __forceinline__ void warp_bitonic_w(uint32_t& key, uint32_t& val) {
  const int li = threadIdx.x & (W - 1);
#pragma unroll
  for (int k = 2; k <= W; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      const uint32_t ok = __shfl_xor_sync(LG_FULL_MASK, key, j);
      uint32_t ov = 0;
      if (VALS) ov = __shfl_xor_sync(LG_FULL_MASK, val, j);
      const bool up = ((li & k) == 0);
      const bool lower = ((li & j) == 0);
      const bool take_other = lower ? (up ? (ok < key) : (ok > key)) : (up ? (ok > key) : (ok < key));
      if (take_other) { key = ok; if (VALS) val = ov; }
    }
  }
}

// sort the rows whose bits are set in `todo` (each of <= W keys): 32 / W rows
// at a time, lane group g taking the g-th next row
template <int W, bool VALS>
__device__ __forceinline__ void sort_rows_w(uint32_t todo, uint64_t mlo, uint64_t md, uint32_t* keys,
                                            uint32_t* vals) {
  const int lane = threadIdx.x & 31;
  const int grp = lane / W, li = lane & (W - 1);
  while (todo) {
    int src = -1;  // the row of this lane's group in this round
#pragma unroll
    for (int g = 0; g < 32 / W; g++) {
      const int r = todo ? __ffs(todo) - 1 : -1;
      if (r >= 0) todo &= todo - 1;
      if (g == grp) src = r;
    }
    const uint64_t lo = __shfl_sync(LG_FULL_MASK, mlo, src < 0 ? 0 : src);
    uint64_t d = __shfl_sync(LG_FULL_MASK, md, src < 0 ? 0 : src);
    if (src < 0) d = 0;
    uint32_t key = (uint64_t)li < d ? keys[lo + li] : 0xffffffffu;
    uint32_t val = (VALS && (uint64_t)li < d) ? vals[lo + li] : 0u;
    warp_bitonic_w<W, VALS>(key, val);
    if ((uint64_t)li < d) {
      keys[lo + li] = key;
      if (VALS) vals[lo + li] = val;
    }
  }
}

// rows of <= 32 keys, 32 rows per warp batch: rows of <= 8 keys four at a
// time (8-lane networks), <= 16 two at a time, the rest one per warp
template <bool VALS>
__global__ void __launch_bounds__(256) k_seg_small(uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                                   const uint64_t* __restrict__ off, uint64_t rows) {
  const int lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t r0 = ((uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; r0 < rows; r0 += warps * 32) {
    const uint64_t mr = r0 + lane;
    uint64_t mlo = 0, md = 0;
    if (mr < rows) { mlo = off[mr]; md = off[mr + 1] - mlo; }
    sort_rows_w<8, VALS>(__ballot_sync(LG_FULL_MASK, md > 1 && md <= 8), mlo, md, keys, vals);
    sort_rows_w<16, VALS>(__ballot_sync(LG_FULL_MASK, md > 8 && md <= 16), mlo, md, keys, vals);
    sort_rows_w<32, VALS>(__ballot_sync(LG_FULL_MASK, md > 16 && md <= SEG_SMALL), mlo, md, keys, vals);
  }
}

// one CTA per row, bitonic network in shared memory over P = 2^k >= d keys
// (padded with UINT32_MAX); blockDim = min(P/2, 256), each thread owns pairs
__global__ void __launch_bounds__(256) k_seg_bitonic(uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                                     const uint64_t* __restrict__ off, const uint32_t* __restrict__ list,
                                                     uint32_t nlist, uint32_t P) {
  extern __shared__ uint32_t sm[];
  uint32_t* sk = sm;
  uint32_t* sv = sm + P;
  const uint32_t half = P >> 1;
  for (uint32_t li = blockIdx.x; li < nlist; li += gridDim.x) {
    const uint64_t r = list[li];
    const uint64_t lo = off[r];
    const uint32_t d = (uint32_t)(off[r + 1] - lo);
    for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
      sk[i] = i < d ? keys[lo + i] : 0xffffffffu;
      if (vals) sv[i] = i < d ? vals[lo + i] : 0u;
    }
    __syncthreads();
    for (uint32_t k = 2; k <= P; k <<= 1) {
      for (uint32_t j = k >> 1; j > 0; j >>= 1) {
        for (uint32_t t = threadIdx.x; t < half; t += blockDim.x) {
          const uint32_t i = ((t & ~(j - 1)) << 1) | (t & (j - 1));
          const uint32_t ixj = i + j;
          const bool up = (i & k) == 0;
          const uint32_t a = sk[i], b = sk[ixj];
          if (up ? (a > b) : (a < b)) {
            sk[i] = b; sk[ixj] = a;
            if (vals) { const uint32_t tv = sv[i]; sv[i] = sv[ixj]; sv[ixj] = tv; }
          }
        }
        __syncthreads();
      }
    }
    for (uint32_t i = threadIdx.x; i < d; i += blockDim.x) {
      keys[lo + i] = sk[i];
      if (vals) vals[lo + i] = sv[i];
    }
    __syncthreads();
  }
}

// size class of a row: 0 = warp path (d <= 32), 1..8 = P = 64..8192, 9 = radix
__device__ __forceinline__ int seg_class(uint64_t d) {
  if (d <= SEG_SMALL) return 0;
  if (d > SEG_MEDIUM) return 9;
  int c = 1;
  uint64_t P = 64;
  while (P < d) { P <<= 1; c++; }
  return c;
}

constexpr int SEG_NCLASS = 10;

__global__ void k_seg_count(const uint64_t* __restrict__ off, uint64_t rows, uint32_t* __restrict__ cnt) {
  __shared__ uint32_t c[SEG_NCLASS];
  if (threadIdx.x < SEG_NCLASS) c[threadIdx.x] = 0;
  __syncthreads();
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (uint64_t)gridDim.x * blockDim.x) {
    const int k = seg_class(off[r + 1] - off[r]);
    if (k) atomicAdd(&c[k], 1u);
  }
  __syncthreads();
  if (threadIdx.x < SEG_NCLASS && c[threadIdx.x]) atomicAdd(&cnt[threadIdx.x], c[threadIdx.x]);
}

__global__ void k_seg_fill(const uint64_t* __restrict__ off, uint64_t rows, const uint32_t* __restrict__ base,
                           uint32_t* __restrict__ cursor, uint32_t* __restrict__ list) {
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (uint64_t)gridDim.x * blockDim.x) {
    const int k = seg_class(off[r + 1] - off[r]);
    if (k) list[base[k] + atomicAdd(&cursor[k], 1u)] = (uint32_t)r;
  }
}

// large rows: gather (row rank, key) composite keys, radix sort, scatter back
__global__ void k_seg_big_gather(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                                 const uint64_t* __restrict__ off, const uint32_t* __restrict__ big,
                                 const uint64_t* __restrict__ boff, uint32_t nbig, uint64_t* __restrict__ ck,
                                 uint32_t* __restrict__ cv) {
  for (uint32_t b = blockIdx.x; b < nbig; b += gridDim.x) {
    const uint64_t lo = off[big[b]], d = off[big[b] + 1] - lo, o = boff[b];
    for (uint64_t i = threadIdx.x; i < d; i += blockDim.x) {
      ck[o + i] = ((uint64_t)b << 32) | keys[lo + i];
      cv[o + i] = vals ? vals[lo + i] : 0u;
    }
  }
}
__global__ void k_seg_big_scatter(uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                  const uint64_t* __restrict__ off, const uint32_t* __restrict__ big,
                                  const uint64_t* __restrict__ boff, uint32_t nbig, const uint64_t* __restrict__ ck,
                                  const uint32_t* __restrict__ cv) {
  for (uint32_t b = blockIdx.x; b < nbig; b += gridDim.x) {
    const uint64_t lo = off[big[b]], d = off[big[b] + 1] - lo, o = boff[b];
    for (uint64_t i = threadIdx.x; i < d; i += blockDim.x) {
      keys[lo + i] = (uint32_t)ck[o + i];
      if (vals) vals[lo + i] = cv[o + i];
    }
  }
}
__global__ void k_seg_big_sizes(const uint64_t* __restrict__ off, const uint32_t* __restrict__ big, uint32_t nbig,
                                uint64_t* __restrict__ sizes) {
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nbig; b += gridDim.x * blockDim.x)
    sizes[b] = off[big[b] + 1] - off[big[b]];
}

static cudaError_t seg_sort_big(uint32_t* keys, uint32_t* vals, const uint64_t* off, const uint32_t* big,
                                uint32_t nbig, cudaStream_t st) {
  uint64_t *sizes = nullptr, *boff = nullptr, *ck = nullptr, *ck2 = nullptr, *stmp = nullptr;
  uint32_t *cv = nullptr, *cv2 = nullptr;
  void* rtmp = nullptr;
  uint64_t nb_total = 0;
  cudaError_t e = cudaMallocAsync((void**)&sizes, nbig * sizeof(uint64_t), st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&boff, (nbig + 1) * sizeof(uint64_t), st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&stmp, scan_tmp_words(nbig) * sizeof(uint64_t), st);
  if (e == cudaSuccess) {
    k_seg_big_sizes<<<grid_for(nbig, 256, 1024), 256, 0, st>>>(off, big, nbig, sizes);
    count_launch();
    e = scan_excl_u64(sizes, nbig, boff, stmp, st);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&nb_total, boff + nbig, sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&ck, nb_total * sizeof(uint64_t), st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&ck2, nb_total * sizeof(uint64_t), st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&cv, nb_total * sizeof(uint32_t), st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&cv2, nb_total * sizeof(uint32_t), st);
  if (e == cudaSuccess) e = cudaMallocAsync(&rtmp, radix_tmp_bytes(nb_total), st);
  if (e == cudaSuccess) {
    k_seg_big_gather<<<grid_for(nbig, 1, 4096), 256, 0, st>>>(keys, vals, off, big, boff, nbig, ck, cv);
    count_launch();
    e = radix_sort_u64(ck, cv, ck2, cv2, nb_total, 32 + host_bits(nbig), rtmp, st);
  }
  if (e == cudaSuccess) {
    k_seg_big_scatter<<<grid_for(nbig, 1, 4096), 256, 0, st>>>(keys, vals, off, big, boff, nbig, ck, cv);
    count_launch();
    e = cudaGetLastError();
  }
  cudaFreeAsync(sizes, st); cudaFreeAsync(boff, st); cudaFreeAsync(stmp, st);
  cudaFreeAsync(ck, st); cudaFreeAsync(ck2, st); cudaFreeAsync(cv, st); cudaFreeAsync(cv2, st);
  cudaFreeAsync(rtmp, st);
  return e;
}

cudaError_t segmented_sort(uint32_t* keys, uint32_t* vals, const uint64_t* off, uint64_t rows, uint64_t total,
                           uint64_t max_row, cudaStream_t st, bool small_done) {
  if (rows == 0 || total == 0 || max_row <= 1) return cudaSuccess;
  cudaError_t e;
  if (!small_done) {
    if (vals) k_seg_small<true><<<grid_for(rows, 256, 152 * 16), 256, 0, st>>>(keys, vals, off, rows);
    else k_seg_small<false><<<grid_for(rows, 256, 152 * 16), 256, 0, st>>>(keys, vals, off, rows);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (max_row <= SEG_SMALL) return cudaSuccess;
  // rows by power-of-two size class
  uint32_t* meta = nullptr;  // cnt[10], base[10], cursor[10]
  if ((e = cudaMallocAsync((void**)&meta, 3 * SEG_NCLASS * sizeof(uint32_t), st)) != cudaSuccess) return e;
  cudaMemsetAsync(meta, 0, 3 * SEG_NCLASS * sizeof(uint32_t), st);
  k_seg_count<<<grid_for(rows, 256, 152 * 16), 256, 0, st>>>(off, rows, meta);
  count_launch();
  uint32_t cnt[SEG_NCLASS], base[SEG_NCLASS];
  cudaMemcpyAsync(cnt, meta, sizeof(cnt), cudaMemcpyDeviceToHost, st);
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) { cudaFreeAsync(meta, st); return e; }
  uint32_t tot = 0;
  for (int k = 0; k < SEG_NCLASS; k++) { base[k] = tot; tot += cnt[k]; }
  uint32_t* list = nullptr;
  if ((e = cudaMallocAsync((void**)&list, (tot ? tot : 1) * sizeof(uint32_t), st)) != cudaSuccess) {
    cudaFreeAsync(meta, st);
    return e;
  }
  cudaMemcpyAsync(meta + SEG_NCLASS, base, sizeof(base), cudaMemcpyHostToDevice, st);
  k_seg_fill<<<grid_for(rows, 256, 152 * 16), 256, 0, st>>>(off, rows, meta + SEG_NCLASS, meta + 2 * SEG_NCLASS, list);
  count_launch();
  for (int k = 1; k <= 8 && e == cudaSuccess; k++) {
    if (!cnt[k]) continue;
    const uint32_t P = 32u << k;
    const unsigned threads = P / 2 < 256 ? P / 2 : 256;
    const size_t smem = (size_t)P * sizeof(uint32_t) * (vals ? 2 : 1);
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_seg_bitonic, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_seg_bitonic<<<grid_for(cnt[k], 1, 152 * 32), threads, smem, st>>>(keys, vals, off, list + base[k], cnt[k], P);
    count_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && cnt[9]) e = seg_sort_big(keys, vals, off, list + base[9], cnt[9], st);
  cudaFreeAsync(list, st);
  cudaFreeAsync(meta, st);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

// =========================================================================
// DM permuter (Section 5.6): label i goes to the i-th vertex in the order
// (degree descending, original ID ascending); the relabeled CSR holds row
// P(v) = sorted { P(u) : u in N_v }.
// =========================================================================
__global__ void k_dm_keys(const uint64_t* __restrict__ rp, uint64_t n, uint64_t max_deg, uint32_t* __restrict__ keys,
                          uint32_t* __restrict__ vals) {
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
    keys[v] = (uint32_t)(max_deg - (rp[v + 1] - rp[v]));
    vals[v] = (uint32_t)v;
  }
}
__global__ void k_dm_perm(const uint32_t* __restrict__ inv, uint64_t n, uint32_t* __restrict__ perm,
                          const uint64_t* __restrict__ rp, uint32_t* __restrict__ newdeg) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t v = inv[i];
    perm[v] = (uint32_t)i;
    newdeg[i] = (uint32_t)(rp[v + 1] - rp[v]);
  }
}
// one warp per new row: copy the old row mapped through perm (rows are sorted
// afterwards; one row per warp keeps the most independent rows in flight).
// The rows stream through L2 (evict-first loads, streaming stores) so that the
// randomly gathered perm array stays resident (evict-last).
__global__ void __launch_bounds__(256) k_dm_scatter(const uint64_t* __restrict__ rp, const uint32_t* __restrict__ col,
                                                    const uint32_t* __restrict__ w, const uint32_t* __restrict__ inv,
                                                    const uint32_t* __restrict__ perm, const uint64_t* __restrict__ nrp,
                                                    uint32_t* __restrict__ ncol, uint32_t* __restrict__ nw, uint64_t n) {
  const int lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  const uint64_t pstream = policy_stream(), pkeep = policy_keep();
  for (uint64_t i = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
    const uint32_t v = inv[i];
    const uint64_t lo = rp[v], d = rp[v + 1] - lo, o = nrp[i];
    for (uint64_t k = lane; k < d; k += 32) {
      const uint32_t c = ldg_hint(col + lo + k, pstream);
      __stcs(ncol + o + k, ldg_hint(perm + c, pkeep));
      if (w) __stcs(nw + o + k, ldg_hint(w + lo + k, pstream));
    }
  }
}

// =========================================================================
// Greedy permuter for local IDs (Listing 1, Section 3.2.2).  The listing walks
// the vertices by increasing degree (ties by ID) and hands the next free label
// to each neighbor that has none; so a vertex's label is the rank of its FIRST
// appearance in the neighbor lists concatenated in that order, and vertices
// that never appear follow in ID order.  That rank is computed in parallel:
// every arc offers its position in the concatenation to its target with
// atomicMin, then one sort by (first position, ID) gives the labels.
// =========================================================================
__global__ void k_gr_keys(const uint64_t* __restrict__ rp, uint64_t n, uint32_t* __restrict__ keys,
                          uint32_t* __restrict__ vals) {
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
    keys[v] = (uint32_t)(rp[v + 1] - rp[v]);
    vals[v] = (uint32_t)v;
  }
}
__global__ void k_gr_degs(const uint64_t* __restrict__ rp, const uint32_t* __restrict__ order, uint64_t n,
                          uint32_t* __restrict__ sdeg, uint64_t* __restrict__ first, uint64_t none,
                          uint32_t* __restrict__ ids) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t v = order[i];
    sdeg[i] = (uint32_t)(rp[v + 1] - rp[v]);
    first[i] = none;
    ids[i] = (uint32_t)i;
  }
}
// one warp per vertex of the sorted order: its arcs offer positions pos0[i] + j
__global__ void __launch_bounds__(256) k_gr_first(const uint64_t* __restrict__ rp, const uint32_t* __restrict__ col,
                                                  const uint32_t* __restrict__ order, const uint64_t* __restrict__ pos0,
                                                  uint64_t n, unsigned long long* __restrict__ first) {
  const int lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t i = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
    const uint32_t v = order[i];
    const uint64_t lo = rp[v], d = rp[v + 1] - lo, p = pos0[i];
    for (uint64_t k = lane; k < d; k += 32) {
      const uint32_t u = col[lo + k];
      if ((unsigned long long)(p + k) < first[u]) atomicMin(first + u, (unsigned long long)(p + k));
    }
  }
}

cudaError_t enc_dm_relabel(const uint64_t* rp, const uint32_t* col, const uint32_t* w, uint64_t n, uint64_t arcs,
                           uint64_t max_deg, uint32_t mode, uint32_t* perm, uint32_t* inv_perm, uint64_t* nrp,
                           uint32_t* ncol, uint32_t* nw, cudaStream_t st) {
  cudaError_t e;
  uint32_t *keys = nullptr, *k2 = nullptr, *v2 = nullptr, *newdeg = nullptr;
  uint64_t* stmp = nullptr;
  void* rtmp = nullptr;
  e = cudaMallocAsync((void**)&keys, n * sizeof(uint32_t), st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&k2, n * sizeof(uint32_t), st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&v2, n * sizeof(uint32_t), st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&newdeg, n * sizeof(uint32_t), st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&stmp, scan_tmp_words(n) * sizeof(uint64_t), st);
  if (e == cudaSuccess) e = cudaMallocAsync(&rtmp, radix_tmp_bytes(n), st);
  if (e == cudaSuccess && mode == 2) {
    // greedy: order by (degree asc, ID asc), first appearances, sort by them
    uint64_t *pos0 = nullptr, *first = nullptr, *first2 = nullptr;
    e = cudaMallocAsync((void**)&pos0, (n + 1) * sizeof(uint64_t), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&first, n * sizeof(uint64_t), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&first2, n * sizeof(uint64_t), st);
    if (e == cudaSuccess) {
      k_gr_keys<<<grid_for(n, 256, 152 * 32), 256, 0, st>>>(rp, n, keys, inv_perm);  // inv_perm: the order
      count_launch();
      e = radix_sort_u32(keys, inv_perm, k2, v2, n, host_bits(max_deg), rtmp, st);
    }
    if (e == cudaSuccess) {
      // first[] indexed by vertex; keys reused as the sorted degrees, v2 as vertex IDs
      k_gr_degs<<<grid_for(n, 256, 152 * 32), 256, 0, st>>>(rp, inv_perm, n, keys, first, arcs, v2);
      count_launch();
      e = scan_excl_u32(keys, n, pos0, stmp, st);
    }
    if (e == cudaSuccess) {
      k_gr_first<<<grid_for(n, 8, 152 * 64), 256, 0, st>>>(rp, col, inv_perm, pos0, n,
                                                           reinterpret_cast<unsigned long long*>(first));
      count_launch();
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      // new label i goes to the vertex with the i-th smallest (first, ID): v2
      // holds 0..n-1, the radix sort is stable, never-seen vertices share key arcs
      e = radix_sort_u64(first, v2, first2, k2, n, host_bits(arcs), rtmp, st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(inv_perm, v2, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st);
    cudaFreeAsync(pos0, st);
    cudaFreeAsync(first, st);
    cudaFreeAsync(first2, st);
  } else if (e == cudaSuccess) {
    k_dm_keys<<<grid_for(n, 256, 152 * 32), 256, 0, st>>>(rp, n, max_deg, keys, inv_perm);
    count_launch();
    e = radix_sort_u32(keys, inv_perm, k2, v2, n, host_bits(max_deg), rtmp, st);
  }
  if (e == cudaSuccess) {
    k_dm_perm<<<grid_for(n, 256, 152 * 32), 256, 0, st>>>(inv_perm, n, perm, rp, newdeg);
    count_launch();
    e = scan_excl_u32(newdeg, n, nrp, stmp, st);
  }
  if (e == cudaSuccess) {
    k_dm_scatter<<<grid_for(n, 8, 152 * 64), 256, 0, st>>>(rp, col, w, inv_perm, perm, nrp, ncol, nw, n);
    count_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = segmented_sort(ncol, w ? nw : nullptr, nrp, n, arcs, max_deg, st);
  cudaFreeAsync(keys, st); cudaFreeAsync(k2, st); cudaFreeAsync(v2, st); cudaFreeAsync(newdeg, st);
  cudaFreeAsync(stmp, st); cudaFreeAsync(rtmp, st);
  return e;
}

}  // namespace lg
