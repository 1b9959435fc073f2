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

// Scatter of one tile of RS_TILE keys: the tile is first ranked stably by digit
// into shared memory (per round of RS_NT keys: a match among the warp's lanes,
// the counts of the warps before, the tile's keys of this digit in earlier
// rounds), then written out in that order, so the keys of one digit -- about
// RS_TILE / 256 of them -- go to consecutive addresses (coalesced writes).
template <typename K>
struct RsSmem {
  K keys[RS_TILE];
  uint32_t vals[RS_TILE];
  uint32_t wcnt[RS_NW][256];
  uint32_t loc[256];        // first position of each digit in the tile
  uint32_t seen[256];       // keys of each digit placed so far
  uint64_t glob[256];       // first global position of each digit for this tile
  uint32_t red[RS_NW];
};

template <typename K>
__global__ void __launch_bounds__(RS_NT) k_rs_scatter(const K* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                      K* __restrict__ kout, uint32_t* __restrict__ vout, uint64_t n,
                                                      uint32_t shift, const uint64_t* __restrict__ off,
                                                      const uint32_t* __restrict__ hist, uint64_t ntiles) {
  extern __shared__ __align__(16) unsigned char rs_raw[];
  RsSmem<K>& sm = *reinterpret_cast<RsSmem<K>*>(rs_raw);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint64_t cell = (uint64_t)threadIdx.x * ntiles + blockIdx.x;
  {
    uint32_t total;
    sm.loc[threadIdx.x] = block_excl_scan<uint32_t, RS_NT>(hist[cell], total, sm.red);
    sm.glob[threadIdx.x] = off[cell];
    sm.seen[threadIdx.x] = 0;
  }
  const uint64_t base = (uint64_t)blockIdx.x * RS_TILE;
  const uint32_t tn = (uint32_t)min((uint64_t)RS_TILE, n - base);
  for (int r = 0; r < RS_ROUNDS; r++) {
    for (int k = 0; k < RS_NW; k++) sm.wcnt[k][threadIdx.x] = 0;
    __syncthreads();
    const uint32_t li = (uint32_t)r * RS_NT + threadIdx.x;
    const bool ok = li < tn;
    const K key = ok ? kin[base + li] : K(0);
    const uint32_t val = (ok && vin) ? vin[base + li] : 0u;
    const uint32_t dig = ok ? ((uint32_t)(key >> shift) & 255u) : 256u;
    const uint32_t peers = __match_any_sync(LG_FULL_MASK, dig);
    const uint32_t rank = __popc(peers & lanemask_lt());
    if (ok && rank == 0) sm.wcnt[w][dig] = __popc(peers);
    __syncthreads();
    // thread t owns digit t: exclusive prefix over the warps of this round
    uint32_t acc = 0;
    for (int k = 0; k < RS_NW; k++) {
      const uint32_t c = sm.wcnt[k][threadIdx.x];
      sm.wcnt[k][threadIdx.x] = acc;
      acc += c;
    }
    __syncthreads();
    if (ok) {
      const uint32_t pos = sm.loc[dig] + sm.seen[dig] + sm.wcnt[w][dig] + rank;
      sm.keys[pos] = key;
      sm.vals[pos] = val;
    }
    __syncthreads();
    sm.seen[threadIdx.x] += acc;
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < tn; i += RS_NT) {
    const K key = sm.keys[i];
    const uint32_t dig = (uint32_t)(key >> shift) & 255u;
    const uint64_t pos = sm.glob[dig] + (i - sm.loc[dig]);
    kout[pos] = key;
    if (vin) vout[pos] = sm.vals[i];
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
  {
    const cudaError_t e = cudaFuncSetAttribute(k_rs_scatter<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)sizeof(RsSmem<K>));
    if (e != cudaSuccess) return e;
  }
  for (uint32_t p = 0; p < passes; p++) {
    const uint32_t shift = 8 * p;
    k_rs_hist<K><<<(unsigned)ntiles, RS_NT, 0, st>>>(ka, n, shift, hist, ntiles);
    count_launch();
    cudaError_t e = scan_excl_u32(hist, cells, off, stmp, st);
    if (e != cudaSuccess) return e;
    k_rs_scatter<K><<<(unsigned)ntiles, RS_NT, sizeof(RsSmem<K>), st>>>(ka, va, kb, vb, n, shift, off, hist, ntiles);
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
constexpr uint32_t SEG_SMALL = 32;    // one thread per row, sorting network in registers
constexpr uint32_t SEG_MEDIUM = 4096; // 16 keys per lane, 4 lanes .. 8 warps per row
constexpr int SROW = 33;              // shared slot stride of a small row (conflict-free lanes)

// compare-exchange into ascending order, without branches
template <bool VALS>
__device__ __forceinline__ void ce_asc(uint32_t& a, uint32_t& b, uint32_t& va, uint32_t& vb) {
  if (VALS) {
    const bool sw = a > b;
    const uint32_t ta = sw ? b : a, tb = sw ? a : b;
    const uint32_t tva = sw ? vb : va, tvb = sw ? va : vb;
    a = ta; b = tb; va = tva; vb = tvb;
  } else {
    const uint32_t lo = min(a, b), hi = max(a, b);
    a = lo; b = hi;
  }
}

// compare-exchange into ascending (up) or descending order
template <bool VALS>
__device__ __forceinline__ void ce_dir(uint32_t& a, uint32_t& b, uint32_t& va, uint32_t& vb, bool up) {
  if (VALS) {
    const bool sw = up ? (a > b) : (a < b);
    const uint32_t ta = sw ? b : a, tb = sw ? a : b;
    const uint32_t tva = sw ? vb : va, tvb = sw ? va : vb;
    a = ta; b = tb; va = tva; vb = tvb;
  } else {
    const uint32_t lo = min(a, b), hi = max(a, b);
    a = up ? lo : hi; b = up ? hi : lo;
  }
}

// Batcher's odd-even merge sort network on N = 2^m registers (19, 63 and 191
// comparators for N = 8, 16, 32): merges of sorted runs of length p into runs
// of 2p, each merge comparing elements k apart for k = p, p/2, .., 1 within
// the same 2p-run.  One instantiation per (p, k), so that every register
// index is a compile-time constant.
template <int N, bool VALS, int P, int K>
__device__ __forceinline__ void oem_pk(uint32_t (&x)[N], uint32_t (&y)[N]) {
  if constexpr (P < N) {
    if constexpr (K == 0) {
      oem_pk<N, VALS, 2 * P, 2 * P>(x, y);
    } else {
#pragma unroll
      for (int j = K % P; j + K < N; j += 2 * K) {
#pragma unroll
        for (int i = 0; i < K; i++) {
          if (i + j + K < N && (i + j) / (2 * P) == (i + j + K) / (2 * P))
            ce_asc<VALS>(x[i + j], x[i + j + K], y[i + j], y[i + j + K]);
        }
      }
      oem_pk<N, VALS, P, K / 2>(x, y);
    }
  }
}

template <int N, bool VALS>
__device__ __forceinline__ void oem_sort(uint32_t (&x)[N], uint32_t (&y)[N]) {
  oem_pk<N, VALS, 1, 1>(x, y);
}

// one thread sorts the d <= N keys of its shared slot (padded with UINT32_MAX)
template <int N, bool VALS>
__device__ __forceinline__ void slot_sort(uint32_t* sk, uint32_t* sv, uint32_t d) {
  uint32_t x[N], y[N];
#pragma unroll
  for (int t = 0; t < N; t++) {
    x[t] = (uint32_t)t < d ? sk[t] : 0xffffffffu;
    y[t] = (VALS && (uint32_t)t < d) ? sv[t] : 0u;
  }
  oem_sort<N, VALS>(x, y);
#pragma unroll
  for (int t = 0; t < N; t++) {
    if ((uint32_t)t < d) {
      sk[t] = x[t];
      if (VALS) sv[t] = y[t];
    }
  }
}

// Each lane sorts slot `lane` (d keys, d <= 32) of its warp's 32 shared slots.
// A warp runs at most two networks: 8 keys, and 16 or 32 (32 if any of its
// rows needs it).
template <bool VALS>
__device__ __forceinline__ void warp_sort_slots(uint32_t* sk, uint32_t* sv, uint32_t d, bool small, int lane) {
  const bool any32 = __any_sync(LG_FULL_MASK, small && d > 16);
  if (small && d > 1) {
    uint32_t* k = sk + lane * SROW;
    uint32_t* v = sv + lane * SROW;
    if (d <= 8) slot_sort<8, VALS>(k, v, d);
    else if (any32) slot_sort<32, VALS>(k, v, d);
    else slot_sort<16, VALS>(k, v, d);
  }
  __syncwarp();
}

// rows of <= 32 keys, in place: a warp takes 32 consecutive rows, copies the
// small ones into its shared slots (coalesced, a row per step), sorts a row
// per lane and copies them back.
template <bool VALS>
__global__ void __launch_bounds__(256) k_seg_small(uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                                   const uint64_t* __restrict__ off, uint64_t rows) {
  extern __shared__ uint32_t ssm[];  // 8 warps x 32 slots of keys, then of values
  const int lane = threadIdx.x & 31;
  uint32_t* sk = ssm + (threadIdx.x >> 5) * 32 * SROW;
  uint32_t* sv = ssm + 8 * 32 * SROW + (threadIdx.x >> 5) * 32 * SROW;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t r0 = ((uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; r0 < rows;
       r0 += warps * 32) {
    const uint64_t r = r0 + lane;
    uint64_t lo = 0;
    uint32_t d = 0;
    if (r < rows) {
      lo = off[r];
      d = (uint32_t)(off[r + 1] - lo);
    }
    const bool small = d > 1 && d <= SEG_SMALL;
    const uint32_t todo = __ballot_sync(LG_FULL_MASK, small);
    if (!todo) continue;
    for (uint32_t t = todo; t; t &= t - 1) {
      const int q = __ffs(t) - 1;
      const uint64_t lq = __shfl_sync(LG_FULL_MASK, lo, q);
      const uint32_t dq = __shfl_sync(LG_FULL_MASK, d, q);
      if ((uint32_t)lane < dq) {
        sk[q * SROW + lane] = keys[lq + lane];
        if (VALS) sv[q * SROW + lane] = vals[lq + lane];
      }
    }
    __syncwarp();
    warp_sort_slots<VALS>(sk, sv, d, small, lane);
    for (uint32_t t = todo; t; t &= t - 1) {
      const int q = __ffs(t) - 1;
      const uint64_t lq = __shfl_sync(LG_FULL_MASK, lo, q);
      const uint32_t dq = __shfl_sync(LG_FULL_MASK, d, q);
      if ((uint32_t)lane < dq) {
        keys[lq + lane] = sk[q * SROW + lane];
        if (VALS) vals[lq + lane] = sv[q * SROW + lane];
      }
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Rows of 32 < d <= 4096 keys from a size-class list, P = 16 G W >= d keys per
// row (padded with UINT32_MAX): G lanes per row in a warp (G <= 32), or W
// warps per row (G = 32).  Lane g of warp w holds keys 16 (32 w + g) + e,
// e < 16, so a bitonic compare-exchange at distance j is a register pair for
// j < 16, a shuffle with lane g ^ (j / 16) for 16 <= j < 512 and an exchange
// through shared memory with warp w ^ (j / 512) beyond.  The first four
// levels are unrolled; the rest run as a loop (an unrolled network of this
// size would outgrow the instruction cache).
// ---------------------------------------------------------------------------
template <int J, bool VALS>
__device__ __forceinline__ void blk_pairs(uint32_t (&x)[16], uint32_t (&y)[16], uint32_t base16, uint32_t k) {
#pragma unroll
  for (int e = 0; e < 16; e++) {
    if ((e & J) == 0) ce_dir<VALS>(x[e], x[e | J], y[e], y[e | J], ((base16 | (uint32_t)e) & k) == 0);
  }
}

// the four register stages j = 8, 4, 2, 1 of a level k >= 16 (direction set
// by the lane's block only)
template <bool VALS>
__device__ __forceinline__ void blk_tail(uint32_t (&x)[16], uint32_t (&y)[16], bool up) {
#pragma unroll
  for (int j = 8; j >= 1; j >>= 1) {
#pragma unroll
    for (int e = 0; e < 16; e++) {
      if ((e & j) == 0) ce_dir<VALS>(x[e], x[e | j], y[e], y[e | j], up);
    }
  }
}

template <bool VALS>
__device__ __forceinline__ void blk_shfl(uint32_t (&x)[16], uint32_t (&y)[16], uint32_t lanemask, bool keep_min) {
#pragma unroll
  for (int e = 0; e < 16; e++) {
    const uint32_t ok = __shfl_xor_sync(LG_FULL_MASK, x[e], lanemask);
    if (VALS) {
      const uint32_t ov = __shfl_xor_sync(LG_FULL_MASK, y[e], lanemask);
      const bool take = keep_min ? (ok < x[e]) : (ok > x[e]);
      x[e] = take ? ok : x[e];
      y[e] = take ? ov : y[e];
    } else {
      x[e] = keep_min ? min(x[e], ok) : max(x[e], ok);
    }
  }
}

template <int G, int W, bool VALS>
__global__ void __launch_bounds__(256) k_seg_blk(uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                                 const uint64_t* __restrict__ off, const uint32_t* __restrict__ list,
                                                 uint32_t nlist) {
  constexpr uint32_t P = 16u * G * W;
  constexpr int RPB = 256 / (G * W);  // rows per block pass
  extern __shared__ uint32_t bsm[];   // W > 1: RPB rows x P keys, then values
  const int lane = threadIdx.x & 31;
  const int g = lane % G;
  const int wv = W > 1 ? (threadIdx.x >> 5) % W : 0;
  const int grp = threadIdx.x / (G * W);
  const uint32_t base16 = 16u * (32u * wv + g);
  uint32_t* gk = bsm + grp * P;
  uint32_t* gv = bsm + RPB * P + grp * P;
  for (uint64_t base = (uint64_t)blockIdx.x * RPB; base < nlist; base += (uint64_t)gridDim.x * RPB) {
    const uint64_t li = base + grp;
    uint64_t lo = 0;
    uint32_t d = 0;
    if (li < nlist) {
      const uint64_t r = list[li];
      lo = off[r];
      d = (uint32_t)(off[r + 1] - lo);
    }
    uint32_t x[16], y[16];
#pragma unroll
    for (int e = 0; e < 16; e++) {
      const uint32_t i = base16 + e;
      x[e] = i < d ? keys[lo + i] : 0xffffffffu;
      y[e] = (VALS && i < d) ? vals[lo + i] : 0u;
    }
    // levels k = 2 .. 16 inside the lane's block
    blk_pairs<1, VALS>(x, y, base16, 2);
    blk_pairs<2, VALS>(x, y, base16, 4);
    blk_pairs<1, VALS>(x, y, base16, 4);
    blk_pairs<4, VALS>(x, y, base16, 8);
    blk_pairs<2, VALS>(x, y, base16, 8);
    blk_pairs<1, VALS>(x, y, base16, 8);
    blk_tail<VALS>(x, y, (base16 & 16u) == 0);
#pragma unroll 1
    for (uint32_t k = 32; k <= P; k <<= 1) {
      const bool up = (base16 & k) == 0;
#pragma unroll 1
      for (uint32_t j = k >> 1; j >= 16; j >>= 1) {
        if (W > 1 && j >= 512) {  // partner warp wv ^ (j / 512), same lane and register
          const int jw = (int)(j >> 9);
          __syncthreads();
#pragma unroll
          for (int e = 0; e < 16; e++) {
            gk[wv * 512 + e * 32 + lane] = x[e];
            if (VALS) gv[wv * 512 + e * 32 + lane] = y[e];
          }
          __syncthreads();
          const bool keep_min = (((wv & jw) == 0) == up);
#pragma unroll
          for (int e = 0; e < 16; e++) {
            const int at = (wv ^ jw) * 512 + e * 32 + lane;
            const uint32_t ok = gk[at];
            const bool take = keep_min ? (ok < x[e]) : (ok > x[e]);
            if (VALS) y[e] = take ? gv[at] : y[e];
            x[e] = take ? ok : x[e];
          }
        } else {
          const uint32_t m = j >> 4;
          blk_shfl<VALS>(x, y, m, ((g & m) == 0) == up);
        }
      }
      blk_tail<VALS>(x, y, up);
    }
#pragma unroll
    for (int e = 0; e < 16; e++) {
      const uint32_t i = base16 + e;
      if (i < d) {
        keys[lo + i] = x[e];
        if (VALS) vals[lo + i] = y[e];
      }
    }
  }
}

// size class of a row: 0 = warp path (d <= 32), 1..7 = P = 64..4096, 9 = radix
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

__global__ void __launch_bounds__(256) k_seg_fill(const uint64_t* __restrict__ off, uint64_t rows,
                                                  const uint32_t* __restrict__ base, uint32_t* __restrict__ cursor,
                                                  uint32_t* __restrict__ list) {
  const int lane = threadIdx.x & 31;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t r0 = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); r0 < rows; r0 += stride) {
    const uint64_t r = r0 + lane;
    const int k = r < rows ? seg_class(off[r + 1] - off[r]) : 0;
    // one cursor atomic per class present in the warp
    const uint32_t peers = __match_any_sync(LG_FULL_MASK, k);
    const int leader = __ffs(peers) - 1;
    uint32_t at = 0;
    if (k && lane == leader) at = base[k] + atomicAdd(&cursor[k], (uint32_t)__popc(peers));
    at = __shfl_sync(LG_FULL_MASK, at, leader);
    if (k) list[at + __popc(peers & ((1u << lane) - 1u))] = (uint32_t)r;
  }
}

// large rows: gather (row rank, key) composite keys, radix sort, scatter back
__global__ void k_seg_big_gather(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                                 const uint64_t* __restrict__ off, const uint32_t* __restrict__ big,
                                 const uint64_t* __restrict__ boff, uint32_t nbig, uint32_t* __restrict__ ck,
                                 uint32_t* __restrict__ cv) {
  for (uint32_t b = blockIdx.x; b < nbig; b += gridDim.x) {
    const uint64_t lo = off[big[b]], d = off[big[b] + 1] - lo, o = boff[b];
    for (uint64_t i = threadIdx.x; i < d; i += blockDim.x) {
      ck[o + i] = keys[lo + i];
      cv[o + i] = vals ? vals[lo + i] : 0u;
    }
  }
}
__global__ void k_seg_big_scatter(uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                  const uint64_t* __restrict__ off, const uint32_t* __restrict__ big,
                                  const uint64_t* __restrict__ boff, uint32_t nbig, const uint32_t* __restrict__ ck,
                                  const uint32_t* __restrict__ cv) {
  for (uint32_t b = blockIdx.x; b < nbig; b += gridDim.x) {
    const uint64_t lo = off[big[b]], d = off[big[b] + 1] - lo, o = boff[b];
    for (uint64_t i = threadIdx.x; i < d; i += blockDim.x) {
      keys[lo + i] = ck[o + i];
      if (vals) vals[lo + i] = cv[o + i];
    }
  }
}
__global__ void k_seg_big_sizes(const uint64_t* __restrict__ off, const uint32_t* __restrict__ big, uint32_t nbig,
                                uint64_t* __restrict__ sizes) {
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nbig; b += gridDim.x * blockDim.x)
    sizes[b] = off[big[b] + 1] - off[big[b]];
}

// -------------------------------------------------------------------------
// One stable split of a tile of up to RS_TILE keys by a 9-bit digit, for the
// segmented radix sorts.  Warp w holds the consecutive chunk of keys
// [c0, c0 + 32 G) with c0 = 32 G w, key c0 + 32 g + lane in x[g]: the warp
// counts its chunk's digits into its own row of `wc` (one match per 32 keys,
// the lowest lane of each digit adds its group's count), one block scan turns
// the (digit, warp) counts into positions, and the warp writes its chunk in
// order.  Three block barriers per pass, whatever the tile's length.
// -------------------------------------------------------------------------
constexpr int SPL_BITS = 9;
constexpr uint32_t SPL_NB = 1u << SPL_BITS;  // digits per pass
constexpr int SPL_G = RS_TILE / RS_NT;       // groups of 32 keys per warp, at most

struct SplitSmem {
  uint32_t wc[RS_NW][SPL_NB];  // per warp: its count, then its next position, of each digit
  uint32_t dstart[SPL_NB];     // first position of each digit in the tile
  uint32_t red[RS_NW];
};

__host__ __device__ constexpr uint32_t spl_passes(uint32_t key_bits) { return (key_bits + SPL_BITS - 1) / SPL_BITS; }

template <bool VALS>
__device__ __forceinline__ void split_pass(const uint32_t (&x)[SPL_G], const uint32_t (&y)[SPL_G], uint32_t c0,
                                           uint32_t len, int G, uint32_t shift, uint32_t* __restrict__ dk,
                                           uint32_t* __restrict__ dv, SplitSmem& sp) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t lt = lanemask_lt();
  for (uint32_t b = lane; b < SPL_NB; b += 32) sp.wc[w][b] = 0;
  __syncwarp();
  uint32_t pm[SPL_G];
#pragma unroll
  for (int g = 0; g < SPL_G; g++) {
    pm[g] = 0;
    if (g < G) {
      const bool ok = c0 + 32u * g + lane < len;
      const uint32_t dig = ok ? (x[g] >> shift) & (SPL_NB - 1) : SPL_NB;
      pm[g] = __match_any_sync(LG_FULL_MASK, dig);
      if (ok && (pm[g] & lt) == 0) sp.wc[w][dig] += __popc(pm[g]);
      __syncwarp();
    }
  }
  __syncthreads();
  constexpr int DPT = SPL_NB / RS_NT;  // digits per thread, consecutive
  uint32_t tot[DPT], sum = 0;
#pragma unroll
  for (int q = 0; q < DPT; q++) {
    const uint32_t b = threadIdx.x * DPT + q;
    uint32_t acc = 0;
#pragma unroll
    for (int v = 0; v < RS_NW; v++) {
      const uint32_t c = sp.wc[v][b];
      sp.wc[v][b] = acc;
      acc += c;
    }
    tot[q] = acc;
    sum += acc;
  }
  uint32_t total;
  uint32_t pre = block_excl_scan<uint32_t, RS_NT>(sum, total, sp.red);
#pragma unroll
  for (int q = 0; q < DPT; q++) {
    const uint32_t b = threadIdx.x * DPT + q;
    sp.dstart[b] = pre;
#pragma unroll
    for (int v = 0; v < RS_NW; v++) sp.wc[v][b] += pre;
    pre += tot[q];
  }
  __syncthreads();
#pragma unroll
  for (int g = 0; g < SPL_G; g++) {
    if (g < G) {
      const bool ok = c0 + 32u * g + lane < len;
      const uint32_t dig = (x[g] >> shift) & (SPL_NB - 1);
      if (ok) {
        const uint32_t pos = sp.wc[w][dig] + __popc(pm[g] & lt);
        dk[pos] = x[g];
        if (VALS) dv[pos] = y[g];
      }
      __syncwarp();
      if (ok && (pm[g] & lt) == 0) sp.wc[w][dig] += __popc(pm[g]);
      __syncwarp();
    }
  }
  __syncthreads();
}

template <bool VALS>
__device__ __forceinline__ void split_load(const uint32_t* __restrict__ k, const uint32_t* __restrict__ v,
                                           uint32_t c0, uint32_t len, int G, uint32_t (&x)[SPL_G],
                                           uint32_t (&y)[SPL_G]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int g = 0; g < SPL_G; g++) {
    const uint32_t i = c0 + 32u * g + lane;
    const bool ok = g < G && i < len;
    x[g] = ok ? k[i] : 0u;
    y[g] = (VALS && ok) ? v[i] : 0u;
  }
}

// Rows above SEG_MEDIUM keys: a segmented LSD radix sort of the rows gathered
// into one buffer.  Tiles of RS_TILE keys never straddle two rows; the
// histogram cells are laid out row by row, digit-major within a row, so one
// exclusive scan over all cells gives every (row, digit, tile) its output
// position inside its own row -- no row index in the keys, ceil(key_bits / 9)
// passes over 4-byte keys.
struct SrsTile {
  uint64_t start;     // first key of the tile in the gathered buffer
  uint64_t cellbase;  // first histogram cell of the tile's row
  uint32_t len;       // keys in the tile (<= RS_TILE)
  uint32_t stride;    // tiles in the row
  uint32_t tl;        // index of the tile within its row
  uint32_t pad;
};

__global__ void k_srs_tile_count(const uint64_t* __restrict__ boff, uint32_t nbig, uint32_t* __restrict__ nt) {
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nbig; b += gridDim.x * blockDim.x)
    nt[b] = (uint32_t)((boff[b + 1] - boff[b] + RS_TILE - 1) / RS_TILE);
}
__global__ void k_srs_tile_fill(const uint64_t* __restrict__ boff, const uint64_t* __restrict__ tbase, uint32_t nbig,
                                SrsTile* __restrict__ tiles) {
  for (uint32_t b = blockIdx.x; b < nbig; b += gridDim.x) {
    const uint64_t size = boff[b + 1] - boff[b], t0 = tbase[b];
    const uint32_t nt = (uint32_t)(tbase[b + 1] - t0);
    for (uint32_t tl = threadIdx.x; tl < nt; tl += blockDim.x) {
      SrsTile d;
      d.start = boff[b] + (uint64_t)tl * RS_TILE;
      d.cellbase = (uint64_t)SPL_NB * t0;
      d.len = (uint32_t)min((uint64_t)RS_TILE, size - (uint64_t)tl * RS_TILE);
      d.stride = nt;
      d.tl = tl;
      d.pad = 0;
      tiles[t0 + tl] = d;
    }
  }
}
__global__ void __launch_bounds__(RS_NT) k_srs_hist(const uint32_t* __restrict__ keys, const SrsTile* __restrict__ tiles,
                                                    uint32_t shift, uint32_t* __restrict__ hist) {
  __shared__ uint32_t cnt[SPL_NB];
  const SrsTile d = tiles[blockIdx.x];
  for (uint32_t b = threadIdx.x; b < SPL_NB; b += RS_NT) cnt[b] = 0;
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < d.len; i += RS_NT)
    atomicAdd(&cnt[(keys[d.start + i] >> shift) & (SPL_NB - 1)], 1u);
  __syncthreads();
  for (uint32_t b = threadIdx.x; b < SPL_NB; b += RS_NT) hist[d.cellbase + (uint64_t)b * d.stride + d.tl] = cnt[b];
}

struct SrsSmem {
  uint32_t k[RS_TILE];
  uint32_t v[RS_TILE];
  uint64_t glob[SPL_NB];  // first output position of each digit of this tile
  SplitSmem sp;
};

// One pass: the tile is split by digit in shared memory, then each key goes to
// its digit's run for this tile (runs of one digit are consecutive in kout).
template <bool VALS>
__global__ void __launch_bounds__(RS_NT) k_srs_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                       uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                       const SrsTile* __restrict__ tiles, uint32_t shift,
                                                       const uint64_t* __restrict__ off) {
  extern __shared__ __align__(16) unsigned char srs_raw[];
  SrsSmem& sm = *reinterpret_cast<SrsSmem*>(srs_raw);
  const SrsTile d = tiles[blockIdx.x];
  for (uint32_t b = threadIdx.x; b < SPL_NB; b += RS_NT) sm.glob[b] = off[d.cellbase + (uint64_t)b * d.stride + d.tl];
  const int G = (int)((d.len + RS_NT - 1) / RS_NT);
  const uint32_t c0 = 32u * G * (threadIdx.x >> 5);
  uint32_t x[SPL_G], y[SPL_G];
  split_load<VALS>(kin + d.start, vin + (VALS ? d.start : 0), c0, d.len, G, x, y);
  split_pass<VALS>(x, y, c0, d.len, G, shift, sm.k, sm.v, sm.sp);
  for (uint32_t i = threadIdx.x; i < d.len; i += RS_NT) {
    const uint32_t key = sm.k[i];
    const uint32_t dig = (key >> shift) & (SPL_NB - 1);
    const uint64_t pos = sm.glob[dig] + (i - sm.sp.dstart[dig]);
    kout[pos] = key;
    if (VALS) vout[pos] = sm.v[i];
  }
}

// The segmented radix passes over rows held back to back in (ka, va), row b at
// [boff[b], boff[b+1]) with boff on the device; kb, vb hold as much.  On
// return *result_in_b says whether the sorted rows ended in (kb, vb).
static cudaError_t srs_sort(uint32_t* ka, uint32_t* va, uint32_t* kb, uint32_t* vb, const uint64_t* boff,
                            uint32_t nbig, uint32_t key_bits, bool* result_in_b, cudaStream_t st) {
  uint64_t *tbase = nullptr, *stmp = nullptr, *coff = nullptr, *ctmp = nullptr;
  uint32_t *nt = nullptr, *hist = nullptr;
  SrsTile* tiles = nullptr;
  uint64_t ntiles = 0;
  *result_in_b = false;
  cudaError_t e = lg::pool_alloc((void**)&tbase, (nbig + 1) * sizeof(uint64_t), st);
  if (e == cudaSuccess) e = lg::pool_alloc((void**)&nt, nbig * sizeof(uint32_t), st);
  if (e == cudaSuccess) e = lg::pool_alloc((void**)&stmp, scan_tmp_words(nbig) * sizeof(uint64_t), st);
  if (e == cudaSuccess) {
    k_srs_tile_count<<<grid_for(nbig, 256, 1024), 256, 0, st>>>(boff, nbig, nt);
    count_launch();
    e = scan_excl_u32(nt, nbig, tbase, stmp, st);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&ntiles, tbase + nbig, sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  const uint64_t cells = (uint64_t)SPL_NB * ntiles;
  if (e == cudaSuccess) e = lg::pool_alloc((void**)&tiles, (ntiles ? ntiles : 1) * sizeof(SrsTile), st);
  if (e == cudaSuccess) e = lg::pool_alloc((void**)&hist, (cells ? cells : 1) * sizeof(uint32_t), st);
  if (e == cudaSuccess) e = lg::pool_alloc((void**)&coff, (cells + 1) * sizeof(uint64_t), st);
  if (e == cudaSuccess) e = lg::pool_alloc((void**)&ctmp, scan_tmp_words(cells) * sizeof(uint64_t), st);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(va ? k_srs_scatter<true> : k_srs_scatter<false>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SrsSmem));
  if (e == cudaSuccess) {
    k_srs_tile_fill<<<grid_for(nbig, 1, 4096), 256, 0, st>>>(boff, tbase, nbig, tiles);
    count_launch();
    e = cudaGetLastError();
  }
  const uint32_t passes = spl_passes(key_bits);
  for (uint32_t p = 0; p < passes && e == cudaSuccess && ntiles; p++) {
    const uint32_t shift = SPL_BITS * p;
    k_srs_hist<<<(unsigned)ntiles, RS_NT, 0, st>>>(ka, tiles, shift, hist);
    count_launch();
    e = scan_excl_u32(hist, cells, coff, ctmp, st);
    if (e != cudaSuccess) break;
    if (va)
      k_srs_scatter<true><<<(unsigned)ntiles, RS_NT, sizeof(SrsSmem), st>>>(ka, va, kb, vb, tiles, shift, coff);
    else
      k_srs_scatter<false><<<(unsigned)ntiles, RS_NT, sizeof(SrsSmem), st>>>(ka, va, kb, vb, tiles, shift, coff);
    count_launch();
    e = cudaGetLastError();
    uint32_t* t = ka; ka = kb; kb = t;
    t = va; va = vb; vb = t;
    *result_in_b = !*result_in_b;
  }
  cudaFreeAsync(tbase, st); cudaFreeAsync(nt, st); cudaFreeAsync(stmp, st);
  cudaFreeAsync(tiles, st); cudaFreeAsync(hist, st); cudaFreeAsync(coff, st); cudaFreeAsync(ctmp, st);
  return e;
}

// Rows above SEG_MEDIUM keys listed in `big`: gathered back to back, sorted,
// scattered back.
static cudaError_t seg_sort_big(uint32_t* keys, uint32_t* vals, const uint64_t* off, const uint32_t* big,
                                uint32_t nbig, uint32_t key_bits, cudaStream_t st) {
  uint64_t *sizes = nullptr, *boff = nullptr, *stmp = nullptr;
  uint32_t *ka = nullptr, *kb = nullptr, *va = nullptr, *vb = nullptr;
  uint64_t nb_total = 0;
  cudaError_t e = lg::pool_alloc((void**)&sizes, nbig * sizeof(uint64_t), st);
  if (e == cudaSuccess) e = lg::pool_alloc((void**)&boff, (nbig + 1) * sizeof(uint64_t), st);
  if (e == cudaSuccess) e = lg::pool_alloc((void**)&stmp, scan_tmp_words(nbig) * sizeof(uint64_t), st);
  if (e == cudaSuccess) {
    k_seg_big_sizes<<<grid_for(nbig, 256, 1024), 256, 0, st>>>(off, big, nbig, sizes);
    count_launch();
    e = scan_excl_u64(sizes, nbig, boff, stmp, st);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&nb_total, boff + nbig, sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = lg::pool_alloc((void**)&ka, nb_total * sizeof(uint32_t), st);
  if (e == cudaSuccess) e = lg::pool_alloc((void**)&kb, nb_total * sizeof(uint32_t), st);
  if (e == cudaSuccess) e = lg::pool_alloc((void**)&va, nb_total * sizeof(uint32_t), st);
  if (e == cudaSuccess) e = lg::pool_alloc((void**)&vb, nb_total * sizeof(uint32_t), st);
  if (e == cudaSuccess) {
    k_seg_big_gather<<<grid_for(nbig, 1, 4096), 256, 0, st>>>(keys, vals, off, big, boff, nbig, ka, va);
    count_launch();
    e = cudaGetLastError();
  }
  bool in_b = false;
  if (e == cudaSuccess) e = srs_sort(ka, vals ? va : nullptr, kb, vals ? vb : nullptr, boff, nbig, key_bits, &in_b, st);
  if (e == cudaSuccess) {
    k_seg_big_scatter<<<grid_for(nbig, 1, 4096), 256, 0, st>>>(keys, vals, off, big, boff, nbig, in_b ? kb : ka,
                                                                in_b ? vb : va);
    count_launch();
    e = cudaGetLastError();
  }
  cudaFreeAsync(sizes, st); cudaFreeAsync(boff, st); cudaFreeAsync(stmp, st);
  cudaFreeAsync(ka, st); cudaFreeAsync(kb, st); cudaFreeAsync(va, st); cudaFreeAsync(vb, st);
  return e;
}

// The first nbig rows are the rows above SEG_MEDIUM keys (degree-descending
// order) and lie back to back from off[0] = 0: sorted in place, with one
// buffer of the same size beside them.
static cudaError_t seg_sort_big_prefix(uint32_t* keys, uint32_t* vals, const uint64_t* off, uint32_t nbig,
                                       uint32_t key_bits, cudaStream_t st) {
  uint64_t nb_total = 0;
  cudaError_t e = cudaMemcpyAsync(&nb_total, off + nbig, sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  uint32_t *kb = nullptr, *vb = nullptr;
  if (e == cudaSuccess) e = lg::pool_alloc((void**)&kb, nb_total * sizeof(uint32_t), st);
  if (e == cudaSuccess && vals) e = lg::pool_alloc((void**)&vb, nb_total * sizeof(uint32_t), st);
  bool in_b = false;
  if (e == cudaSuccess) e = srs_sort(keys, vals, kb, vb, off, nbig, key_bits, &in_b, st);
  if (e == cudaSuccess && in_b) {
    e = cudaMemcpyAsync(keys, kb, nb_total * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && vals) e = cudaMemcpyAsync(vals, vb, nb_total * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st);
  }
  if (kb) cudaFreeAsync(kb, st);
  if (vb) cudaFreeAsync(vb, st);
  return e;
}

// Rows of 513..4096 keys: a CTA per row, a stable LSD radix sort with 9-bit
// digits (ceil(key_bits / 9) passes of split_pass) -- a few compare-free steps
// per key and pass instead of a bitonic network's log2(d) (log2(d) + 1) / 2
// stages.
constexpr uint32_t SEG_RADIX_MAX = 4096;
static_assert(SEG_RADIX_MAX <= (uint32_t)RS_TILE, "a row must fit one split tile");

template <bool VALS>
struct SegRadixSmem {
  uint32_t k[SEG_RADIX_MAX];
  uint32_t v[VALS ? SEG_RADIX_MAX : 1];
  SplitSmem sp;
};

// Rows of SEG_SMALL < d <= SEG_RADIX_MAX keys, one row per block: the keys
// stay in registers (warp chunks), each pass splits them into shared memory
// and reads them back; the last pass's order is written out coalesced.
template <bool VALS>
__global__ void __launch_bounds__(RS_NT) k_seg_radix(uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                                     const uint64_t* __restrict__ off,
                                                     const uint32_t* __restrict__ list, uint32_t nlist,
                                                     uint32_t passes) {
  extern __shared__ __align__(16) unsigned char sr_raw[];
  SegRadixSmem<VALS>& sm = *reinterpret_cast<SegRadixSmem<VALS>*>(sr_raw);
  for (uint32_t li = blockIdx.x; li < nlist; li += gridDim.x) {
    const uint64_t lo = off[list[li]];
    const uint32_t d = (uint32_t)(off[list[li] + 1] - lo);
    const int G = (int)((d + RS_NT - 1) / RS_NT);
    const uint32_t c0 = 32u * G * (threadIdx.x >> 5);
    uint32_t x[SPL_G], y[SPL_G];
    split_load<VALS>(keys + lo, vals + (VALS ? lo : 0), c0, d, G, x, y);
    for (uint32_t p = 0; p < passes; p++) {
      if (p) split_load<VALS>(sm.k, sm.v, c0, d, G, x, y);
      split_pass<VALS>(x, y, c0, d, G, SPL_BITS * p, sm.k, sm.v, sm.sp);
    }
    for (uint32_t i = threadIdx.x; i < d; i += RS_NT) {
      keys[lo + i] = sm.k[i];
      if (VALS) vals[lo + i] = sm.v[i];
    }
    __syncthreads();
  }
}

template <bool VALS>
static cudaError_t seg_radix_launch(uint32_t* keys, uint32_t* vals, const uint64_t* off, const uint32_t* list,
                                    uint32_t nlist, uint32_t key_bits, cudaStream_t st) {
  const size_t smem = sizeof(SegRadixSmem<VALS>);
  cudaError_t e = cudaFuncSetAttribute(k_seg_radix<VALS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_seg_radix<VALS><<<grid_for(nlist, 1, 152 * 8), RS_NT, smem, st>>>(keys, vals, off, list, nlist,
                                                                      spl_passes(key_bits));
  count_launch();
  return cudaGetLastError();
}

template <int G, int W, bool VALS>
static cudaError_t seg_blk_launch(uint32_t* keys, uint32_t* vals, const uint64_t* off, const uint32_t* list,
                                  uint32_t nlist, cudaStream_t st) {
  constexpr int RPB = 256 / (G * W);
  const size_t smem = W > 1 ? (size_t)RPB * 16 * G * W * sizeof(uint32_t) * (VALS ? 2 : 1) : 0;
  k_seg_blk<G, W, VALS><<<grid_for(nlist, RPB, 152 * 16), 256, smem, st>>>(keys, vals, off, list, nlist);
  count_launch();
  return cudaGetLastError();
}

// size class k holds rows of 2^(4+k) < d <= 2^(5+k) keys
template <bool VALS>
static cudaError_t seg_blk_class(int k, uint32_t* keys, uint32_t* vals, const uint64_t* off, const uint32_t* list,
                                 uint32_t nlist, cudaStream_t st) {
  switch (k) {
    case 1: return seg_blk_launch<4, 1, VALS>(keys, vals, off, list, nlist, st);
    case 2: return seg_blk_launch<8, 1, VALS>(keys, vals, off, list, nlist, st);
    case 3: return seg_blk_launch<16, 1, VALS>(keys, vals, off, list, nlist, st);
    case 4: return seg_blk_launch<32, 1, VALS>(keys, vals, off, list, nlist, st);
    case 5: return seg_blk_launch<32, 2, VALS>(keys, vals, off, list, nlist, st);
    case 6: return seg_blk_launch<32, 4, VALS>(keys, vals, off, list, nlist, st);
    case 7: return seg_blk_launch<32, 8, VALS>(keys, vals, off, list, nlist, st);
    default: return cudaErrorInvalidValue;
  }
}

static cudaError_t seg_small_launch(uint32_t* keys, uint32_t* vals, const uint64_t* off, uint64_t rows,
                                    cudaStream_t st) {
  const size_t smem = (size_t)8 * 32 * SROW * sizeof(uint32_t) * (vals ? 2 : 1);
  if (vals) {
    const cudaError_t e = cudaFuncSetAttribute(k_seg_small<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (vals) k_seg_small<true><<<grid_for(rows, 256, 152 * 16), 256, smem, st>>>(keys, vals, off, rows);
  else k_seg_small<false><<<grid_for(rows, 256, 152 * 16), 256, smem, st>>>(keys, vals, off, rows);
  count_launch();
  return cudaGetLastError();
}

cudaError_t segmented_sort(uint32_t* keys, uint32_t* vals, const uint64_t* off, uint64_t rows, uint64_t total,
                           uint64_t max_row, cudaStream_t st, bool small_done, uint32_t key_bits, bool big_prefix) {
  if (rows == 0 || total == 0 || max_row <= 1) return cudaSuccess;
  cudaError_t e;
  if (!small_done && (e = seg_small_launch(keys, vals, off, rows, st)) != cudaSuccess) return e;
  if (max_row <= SEG_SMALL) return cudaSuccess;
  // rows by power-of-two size class
  uint32_t* meta = nullptr;  // cnt[10], base[10], cursor[10]
  if ((e = lg::pool_alloc((void**)&meta, 3 * SEG_NCLASS * sizeof(uint32_t), st)) != cudaSuccess) return e;
  cudaMemsetAsync(meta, 0, 3 * SEG_NCLASS * sizeof(uint32_t), st);
  k_seg_count<<<grid_for(rows, 256, 152 * 16), 256, 0, st>>>(off, rows, meta);
  count_launch();
  uint32_t cnt[SEG_NCLASS], base[SEG_NCLASS];
  cudaMemcpyAsync(cnt, meta, sizeof(cnt), cudaMemcpyDeviceToHost, st);
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) { cudaFreeAsync(meta, st); return e; }
  uint32_t tot = 0;
  for (int k = 0; k < SEG_NCLASS; k++) { base[k] = tot; tot += cnt[k]; }
  uint32_t* list = nullptr;
  if ((e = lg::pool_alloc((void**)&list, (tot ? tot : 1) * sizeof(uint32_t), st)) != cudaSuccess) {
    cudaFreeAsync(meta, st);
    return e;
  }
  cudaMemcpyAsync(meta + SEG_NCLASS, base, sizeof(base), cudaMemcpyHostToDevice, st);
  k_seg_fill<<<grid_for(rows, 256, 152 * 16), 256, 0, st>>>(off, rows, meta + SEG_NCLASS, meta + 2 * SEG_NCLASS, list);
  count_launch();
  for (int k = 1; k <= 4 && e == cudaSuccess; k++)
    if (cnt[k]) e = vals ? seg_blk_class<true>(k, keys, vals, off, list + base[k], cnt[k], st)
                         : seg_blk_class<false>(k, keys, vals, off, list + base[k], cnt[k], st);
  // rows of 513..4096 keys: one radix sort per row in shared memory
  const uint32_t mid = cnt[5] + cnt[6] + cnt[7];  // classes 5..7 are adjacent in `list`
  if (e == cudaSuccess && mid)
    e = vals ? seg_radix_launch<true>(keys, vals, off, list + base[5], mid, key_bits, st)
             : seg_radix_launch<false>(keys, vals, off, list + base[5], mid, key_bits, st);
  if (e == cudaSuccess && cnt[9])
    e = big_prefix ? seg_sort_big_prefix(keys, vals, off, cnt[9], key_bits, st)
                   : seg_sort_big(keys, vals, off, list + base[9], cnt[9], key_bits, st);
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
// New rows P(v) = { P(u) : u in N_v }.  A warp takes 32 consecutive new rows.
// Rows of <= 32 arcs are gathered into the warp's shared slots (a row per
// step, coalesced reads of the old row, DM_INFLIGHT rows' perm lookups in
// flight),
// sorted one per lane in registers and written out coalesced, so they are
// final here.  Longer rows are copied unsorted (the size-class sorts follow).
// Rows stream through L2 (evict-first loads, streaming stores) so that the
// randomly gathered perm array stays resident (evict-last).
constexpr int DM_INFLIGHT = 8;  // rows whose loads and perm lookups are in flight together

template <bool VALS>
__global__ void __launch_bounds__(256) k_dm_rows(const uint64_t* __restrict__ rp, const uint32_t* __restrict__ col,
                                                 const uint32_t* __restrict__ w, const uint32_t* __restrict__ inv,
                                                 const uint32_t* __restrict__ perm, const uint64_t* __restrict__ nrp,
                                                 uint32_t* __restrict__ ncol, uint32_t* __restrict__ nw, uint64_t n,
                                                 int skip_big) {
  extern __shared__ uint32_t dsm[];  // 8 warps x 32 slots of keys, then of weights
  const int lane = threadIdx.x & 31;
  uint32_t* sk = dsm + (threadIdx.x >> 5) * 32 * SROW;
  uint32_t* sv = dsm + 8 * 32 * SROW + (threadIdx.x >> 5) * 32 * SROW;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  const uint64_t pstream = policy_stream(), pkeep = policy_keep();
  for (uint64_t i0 = ((uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; i0 < n;
       i0 += warps * 32) {
    const uint64_t i = i0 + lane;
    uint64_t lo = 0, o = 0;
    uint32_t d = 0;
    if (i < n) {
      const uint32_t v = inv[i];
      lo = rp[v];
      d = (uint32_t)(rp[v + 1] - lo);
      o = nrp[i];
    }
    const bool small = d <= SEG_SMALL;
    const uint32_t todo = __ballot_sync(LG_FULL_MASK, small && d > 0);
    for (uint32_t t = todo; t;) {
      int q[DM_INFLIGHT];
      uint32_t c[DM_INFLIGHT];
      bool on[DM_INFLIGHT];
#pragma unroll
      for (int z = 0; z < DM_INFLIGHT; z++) {
        q[z] = t ? __ffs(t) - 1 : 0;
        on[z] = t != 0;
        if (t) t &= t - 1;
      }
#pragma unroll
      for (int z = 0; z < DM_INFLIGHT; z++) {
        const uint64_t lq = __shfl_sync(LG_FULL_MASK, lo, q[z]);
        const uint32_t dq = __shfl_sync(LG_FULL_MASK, d, q[z]);
        on[z] = on[z] && (uint32_t)lane < dq;
        c[z] = on[z] ? ldg_hint(col + lq + lane, pstream) : 0u;
        if (VALS && on[z]) sv[q[z] * SROW + lane] = ldg_hint(w + lq + lane, pstream);
      }
#pragma unroll
      for (int z = 0; z < DM_INFLIGHT; z++) {
        if (on[z]) sk[q[z] * SROW + lane] = ldg_hint(perm + c[z], pkeep);
      }
    }
    __syncwarp();
    warp_sort_slots<VALS>(sk, sv, d, small, lane);
    for (uint32_t t = todo; t; t &= t - 1) {
      const int q = __ffs(t) - 1;
      const uint64_t oq = __shfl_sync(LG_FULL_MASK, o, q);
      const uint32_t dq = __shfl_sync(LG_FULL_MASK, d, q);
      if ((uint32_t)lane < dq) {
        __stcs(ncol + oq + lane, sk[q * SROW + lane]);
        if (VALS) __stcs(nw + oq + lane, sv[q * SROW + lane]);
      }
    }
    __syncwarp();
    if (skip_big) continue;  // k_dm_big copies the rows of more than SEG_SMALL arcs
    for (uint32_t t = __ballot_sync(LG_FULL_MASK, !small); t; t &= t - 1) {
      const int q = __ffs(t) - 1;
      const uint64_t lq = __shfl_sync(LG_FULL_MASK, lo, q);
      const uint64_t oq = __shfl_sync(LG_FULL_MASK, o, q);
      const uint32_t dq = __shfl_sync(LG_FULL_MASK, d, q);
      for (uint32_t k = lane; k < dq; k += 32) {
        const uint32_t cc = ldg_hint(col + lq + k, pstream);
        __stcs(ncol + oq + k, ldg_hint(perm + cc, pkeep));
        if (VALS) __stcs(nw + oq + k, ldg_hint(w + lq + k, pstream));
      }
    }
  }
}

// Rows of more than SEG_SMALL arcs in DM order.  Labels go by degree
// descending, so these rows are the first K new rows and their arcs the prefix
// [0, nrp[K]) of the new CSR: the prefix is cut into chunks of DM_CHUNK arcs
// spread evenly over the grid (a hub no longer rests on one warp).  chunk_row[c]
// is the row holding arc c * DM_CHUNK; a lane walks 8 arcs 32 apart, all their
// loads and perm lookups in flight together.
constexpr uint32_t DM_CHUNK = 256;

// K = the number of rows of more than SEG_SMALL arcs (degrees are descending)
__global__ void k_dm_count_big(const uint32_t* __restrict__ newdeg, uint64_t n, unsigned long long* __restrict__ K) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    if (newdeg[i] > SEG_SMALL && (i + 1 == n || newdeg[i + 1] <= SEG_SMALL)) *K = i + 1;
}
__global__ void k_dm_chunk_rows(const uint64_t* __restrict__ nrp, uint64_t n, const unsigned long long* __restrict__ K,
                                uint32_t* __restrict__ chunk_row) {
  const uint64_t k = *K;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k && i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t c0 = (nrp[i] + DM_CHUNK - 1) / DM_CHUNK, c1 = (nrp[i + 1] + DM_CHUNK - 1) / DM_CHUNK;
    for (uint64_t c = c0; c < c1; c++) chunk_row[c] = (uint32_t)i;
  }
}
template <bool VALS>
__global__ void __launch_bounds__(256) k_dm_big(const uint64_t* __restrict__ rp, const uint32_t* __restrict__ col,
                                                const uint32_t* __restrict__ w, const uint32_t* __restrict__ inv,
                                                const uint32_t* __restrict__ perm, const uint64_t* __restrict__ nrp,
                                                const unsigned long long* __restrict__ K,
                                                const uint32_t* __restrict__ chunk_row, uint32_t* __restrict__ ncol,
                                                uint32_t* __restrict__ nw) {
  constexpr int T = DM_CHUNK / 32;
  const int lane = threadIdx.x & 31;
  const uint64_t E = nrp[*K];
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  const uint64_t pstream = policy_stream(), pkeep = policy_keep();
  for (uint64_t c = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c * DM_CHUNK < E; c += warps) {
    uint32_t i = chunk_row[c];
    uint64_t rs = nrp[i], re = nrp[i + 1], old = rp[inv[i]];
    uint32_t cc[T], wv[T];
#pragma unroll
    for (int t = 0; t < T; t++) {
      const uint64_t p = c * DM_CHUNK + lane + 32u * t;
      cc[t] = 0;
      wv[t] = 0;
      if (p < E) {
        while (re <= p) {  // next row (each holds more than SEG_SMALL arcs)
          i++;
          rs = re;
          re = nrp[i + 1];
          old = rp[inv[i]];
        }
        cc[t] = ldg_hint(col + old + (p - rs), pstream);
        if (VALS) wv[t] = ldg_hint(w + old + (p - rs), pstream);
      }
    }
    uint32_t pv[T];
#pragma unroll
    for (int t = 0; t < T; t++) {
      const uint64_t p = c * DM_CHUNK + lane + 32u * t;
      pv[t] = p < E ? ldg_hint(perm + cc[t], pkeep) : 0u;
    }
#pragma unroll
    for (int t = 0; t < T; t++) {
      const uint64_t p = c * DM_CHUNK + lane + 32u * t;
      if (p < E) {
        __stcs(ncol + p, pv[t]);
        if (VALS) __stcs(nw + p, wv[t]);
      }
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
  e = lg::pool_alloc((void**)&keys, n * sizeof(uint32_t), st);
  if (e == cudaSuccess) e = lg::pool_alloc((void**)&k2, n * sizeof(uint32_t), st);
  if (e == cudaSuccess) e = lg::pool_alloc((void**)&v2, n * sizeof(uint32_t), st);
  if (e == cudaSuccess) e = lg::pool_alloc((void**)&newdeg, n * sizeof(uint32_t), st);
  if (e == cudaSuccess) e = lg::pool_alloc((void**)&stmp, scan_tmp_words(n) * sizeof(uint64_t), st);
  if (e == cudaSuccess) e = lg::pool_alloc(&rtmp, radix_tmp_bytes(n), st);
  if (e == cudaSuccess && mode == 2) {
    // greedy: order by (degree asc, ID asc), first appearances, sort by them
    uint64_t *pos0 = nullptr, *first = nullptr, *first2 = nullptr;
    e = lg::pool_alloc((void**)&pos0, (n + 1) * sizeof(uint64_t), st);
    if (e == cudaSuccess) e = lg::pool_alloc((void**)&first, n * sizeof(uint64_t), st);
    if (e == cudaSuccess) e = lg::pool_alloc((void**)&first2, n * sizeof(uint64_t), st);
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
  // DM order (degree descending): the rows of more than SEG_SMALL arcs form a
  // prefix and go to k_dm_big; the greedy order mixes sizes, so k_dm_rows
  // copies its big rows itself
  const int split_big = mode != 2;
  unsigned long long* dK = nullptr;
  uint32_t* chunk_row = nullptr;
  if (e == cudaSuccess && split_big) {
    e = lg::pool_alloc((void**)&dK, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = lg::pool_alloc((void**)&chunk_row, (arcs / DM_CHUNK + 2) * sizeof(uint32_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dK, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) {
      k_dm_count_big<<<grid_for(n, 256, 152 * 32), 256, 0, st>>>(newdeg, n, dK);
      count_launch();
      k_dm_chunk_rows<<<grid_for(n, 256, 152 * 32), 256, 0, st>>>(nrp, n, dK, chunk_row);
      count_launch();
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) {
    const size_t smem = (size_t)8 * 32 * SROW * sizeof(uint32_t) * (w ? 2 : 1);
    if (w) {
      e = cudaFuncSetAttribute(k_dm_rows<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess)
        k_dm_rows<true><<<grid_for(n, 256, 152 * 16), 256, smem, st>>>(rp, col, w, inv_perm, perm, nrp, ncol, nw, n,
                                                                       split_big);
    } else {
      k_dm_rows<false><<<grid_for(n, 256, 152 * 16), 256, smem, st>>>(rp, col, w, inv_perm, perm, nrp, ncol, nw, n,
                                                                      split_big);
    }
    count_launch();
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  if (e == cudaSuccess && split_big) {
    if (w) k_dm_big<true><<<152 * 8, 256, 0, st>>>(rp, col, w, inv_perm, perm, nrp, dK, chunk_row, ncol, nw);
    else k_dm_big<false><<<152 * 8, 256, 0, st>>>(rp, col, w, inv_perm, perm, nrp, dK, chunk_row, ncol, nw);
    count_launch();
    e = cudaGetLastError();
  }
  if (dK) cudaFreeAsync(dK, st);
  if (chunk_row) cudaFreeAsync(chunk_row, st);
  // rows of <= 32 arcs left k_dm_rows sorted
  // DM order is degree-descending, so its rows above SEG_MEDIUM keys are the first rows
  if (e == cudaSuccess)
    e = segmented_sort(ncol, w ? nw : nullptr, nrp, n, arcs, max_deg, st, true, host_bits(n - 1), split_big != 0);
  cudaFreeAsync(keys, st); cudaFreeAsync(k2, st); cudaFreeAsync(v2, st); cudaFreeAsync(newdeg, st);
  cudaFreeAsync(stmp, st); cudaFreeAsync(rtmp, st);
  return e;
}

}  // namespace lg
