// Encoder kernels: input validation, per-neighborhood widths (Sections 3.2.2
// and 3.6), the prefix sum of bit lengths, bit packing of A (Sections 3.2-3.3,
// bit order of Listing 2) and of the offsets (Section 3.4, packed; Section 4.3,
// Elias-Fano with select samples).
//
// Packing is word-owned: every output word is assembled by exactly one thread
// (fixed-width streams) or one CTA (variable-width local streams, assembled in
// shared memory), so no global atomics touch A and the result is deterministic.
#include "lg_internal.h"

namespace lg {

// =========================================================================
// exclusive scan (u32 or u64 input, u64 output with the total at out[n])
// =========================================================================
constexpr int SCAN_NT = 256;
constexpr int SCAN_IPT = 8;
constexpr int SCAN_TILE = SCAN_NT * SCAN_IPT;

uint64_t scan_tmp_words(uint64_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 2; }

template <typename T>
__global__ void __launch_bounds__(SCAN_NT) k_scan_reduce(const T* __restrict__ in, uint64_t n,
                                                         uint64_t* __restrict__ part) {
  __shared__ uint64_t tmp[SCAN_NT / 32];
  const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE;
  uint64_t s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_IPT; k++) {
    const uint64_t i = base + (uint64_t)k * SCAN_NT + threadIdx.x;
    if (i < n) s += (uint64_t)in[i];
  }
  uint64_t total;
  block_excl_scan<uint64_t, SCAN_NT>(s, total, tmp);
  if (threadIdx.x == 0) part[blockIdx.x] = total;
}

// single block: exclusive scan of the tile partials in place, total at part[np]
__global__ void __launch_bounds__(SCAN_NT) k_scan_partials(uint64_t* part, uint64_t np) {
  __shared__ uint64_t tmp[SCAN_NT / 32];
  uint64_t carry = 0;
  for (uint64_t base = 0; base < np; base += SCAN_TILE) {
    uint64_t v[SCAN_IPT];
    uint64_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_IPT; k++) {
      const uint64_t i = base + (uint64_t)threadIdx.x * SCAN_IPT + k;
      v[k] = i < np ? part[i] : 0;
      s += v[k];
    }
    uint64_t total;
    uint64_t pre = block_excl_scan<uint64_t, SCAN_NT>(s, total, tmp) + carry;
#pragma unroll
    for (int k = 0; k < SCAN_IPT; k++) {
      const uint64_t i = base + (uint64_t)threadIdx.x * SCAN_IPT + k;
      if (i < np) part[i] = pre;
      pre += v[k];
    }
    carry += total;
  }
  if (threadIdx.x == 0) part[np] = carry;
}

template <typename T>
__global__ void __launch_bounds__(SCAN_NT) k_scan_down(const T* __restrict__ in, uint64_t n,
                                                       const uint64_t* __restrict__ part,
                                                       uint64_t np, uint64_t* __restrict__ out) {
  __shared__ uint64_t tmp[SCAN_NT / 32];
  const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE;
  uint64_t v[SCAN_IPT];
  uint64_t s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_IPT; k++) {
    const uint64_t i = base + (uint64_t)threadIdx.x * SCAN_IPT + k;
    v[k] = i < n ? (uint64_t)in[i] : 0;
    s += v[k];
  }
  uint64_t total;
  uint64_t pre = block_excl_scan<uint64_t, SCAN_NT>(s, total, tmp) + part[blockIdx.x];
#pragma unroll
  for (int k = 0; k < SCAN_IPT; k++) {
    const uint64_t i = base + (uint64_t)threadIdx.x * SCAN_IPT + k;
    if (i < n) out[i] = pre;
    pre += v[k];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = part[np];
}

template <typename T>
static cudaError_t scan_impl(const T* in, uint64_t n, uint64_t* out, uint64_t* tmp, cudaStream_t st) {
  const uint64_t np = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (np == 0) return cudaMemsetAsync(out, 0, sizeof(uint64_t), st);
  k_scan_reduce<T><<<(unsigned)np, SCAN_NT, 0, st>>>(in, n, tmp);
  count_launch();
  k_scan_partials<<<1, SCAN_NT, 0, st>>>(tmp, np);
  count_launch();
  k_scan_down<T><<<(unsigned)np, SCAN_NT, 0, st>>>(in, n, tmp, np, out);
  count_launch();
  return cudaGetLastError();
}
cudaError_t scan_excl_u64(const uint64_t* in, uint64_t n, uint64_t* out, uint64_t* tmp, cudaStream_t st) {
  return scan_impl<uint64_t>(in, n, out, tmp, st);
}
cudaError_t scan_excl_u32(const uint32_t* in, uint64_t n, uint64_t* out, uint64_t* tmp, cudaStream_t st) {
  return scan_impl<uint32_t>(in, n, out, tmp, st);
}

// =========================================================================
// validation (never reads outside the given arrays)
// =========================================================================
// Streaming validation.  Rows are strictly increasing iff every "break"
// (a position j > 0 with col[j-1] >= col[j]) is the first arc of a row, i.e.
// iff the number of breaks equals the number of breaks at the starts of
// nonempty rows (each such row has its own start).  A row pass checks the
// bounds, takes the largest degree and counts breaks at row starts; an arc
// pass (16-byte loads when aligned) checks ID ranges and weights and counts
// all breaks; a last thread compares the two counts.
__global__ void __launch_bounds__(256) k_validate_rows(const uint64_t* __restrict__ rp, const uint32_t* __restrict__ col,
                                                       uint64_t n, uint64_t arcs, int* err,
                                                       unsigned long long* max_deg, unsigned long long* start_breaks) {
  uint64_t dmax = 0, sb = 0;
  int flags = 0;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t lo = rp[v], hi = rp[v + 1];
    if (hi < lo || hi > arcs || (v == 0 && lo != 0) || (v == n - 1 && hi != arcs) || hi - lo > n) {
      flags |= DERR_ROWPTR;
      continue;
    }
    dmax = max(dmax, hi - lo);
    if (hi > lo && lo > 0 && col[lo - 1] >= col[lo]) sb++;
  }
  flags = __reduce_or_sync(LG_FULL_MASK, flags);
  for (int o = 16; o > 0; o >>= 1) {
    dmax = max(dmax, (uint64_t)__shfl_xor_sync(LG_FULL_MASK, dmax, o));
    sb += __shfl_xor_sync(LG_FULL_MASK, sb, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (flags) atomicOr(err, flags);
    if (dmax) atomicMax(max_deg, (unsigned long long)dmax);
    if (sb) atomicAdd(start_breaks, (unsigned long long)sb);
  }
}

template <bool VEC>
__global__ void __launch_bounds__(256) k_validate_arcs(const uint32_t* __restrict__ col, const uint32_t* __restrict__ w,
                                                       uint64_t n, uint64_t arcs, uint32_t wbits, int* err,
                                                       uint32_t* max_w, unsigned long long* breaks) {
  uint64_t nb = 0;
  uint32_t wmax = 0;
  int flags = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i * 4 < arcs; i += stride) {
    const uint64_t j0 = i * 4;
    uint32_t c[4], x[4] = {0, 0, 0, 0};
    if (VEC && j0 + 4 <= arcs) {
      const uint4 q = __ldcs(reinterpret_cast<const uint4*>(col) + i);
      c[0] = q.x; c[1] = q.y; c[2] = q.z; c[3] = q.w;
      if (w) {
        const uint4 r = __ldcs(reinterpret_cast<const uint4*>(w) + i);
        x[0] = r.x; x[1] = r.y; x[2] = r.z; x[3] = r.w;
      }
    } else {
#pragma unroll
      for (int k = 0; k < 4; k++) {
        c[k] = j0 + k < arcs ? col[j0 + k] : 0xffffffffu;
        if (w && j0 + k < arcs) x[k] = w[j0 + k];
      }
    }
    uint32_t prev = j0 > 0 ? col[j0 - 1] : 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
      if (j0 + k >= arcs) break;
      if (c[k] >= n) flags |= DERR_COL_RANGE;
      if (j0 + k > 0 && prev >= c[k]) nb++;
      prev = c[k];
      wmax = max(wmax, x[k]);
      if (w && wbits && wbits < 32 && (x[k] >> wbits)) flags |= DERR_WEIGHT;
    }
  }
  flags = __reduce_or_sync(LG_FULL_MASK, flags);
  wmax = __reduce_max_sync(LG_FULL_MASK, wmax);
  for (int o = 16; o > 0; o >>= 1) nb += __shfl_xor_sync(LG_FULL_MASK, nb, o);
  if ((threadIdx.x & 31) == 0) {
    if (flags) atomicOr(err, flags);
    if (w && wmax) atomicMax(max_w, wmax);
    if (nb) atomicAdd(breaks, (unsigned long long)nb);
  }
}

__global__ void k_validate_sorted(const unsigned long long* breaks, const unsigned long long* start_breaks, int* err) {
  if (threadIdx.x == 0 && breaks[0] != start_breaks[0]) atomicOr(err, DERR_UNSORTED);
}

cudaError_t enc_validate(const uint64_t* rp, const uint32_t* col, const uint32_t* w, uint64_t n, uint64_t arcs,
                         uint32_t wbits, int* err, unsigned long long* max_deg, uint32_t* max_w, cudaStream_t st) {
  // two counters after max_w in the caller's zeroed 64-byte block
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(err) + 24);
  k_validate_rows<<<grid_for(n, 256, 152 * 16), 256, 0, st>>>(rp, col, n, arcs, err, max_deg, cnt + 1);
  count_launch();
  const bool vec = ((reinterpret_cast<uintptr_t>(col) | reinterpret_cast<uintptr_t>(w)) & 15) == 0;
  const unsigned grid = grid_for((arcs + 3) / 4, 256, 152 * 16);
  if (vec) k_validate_arcs<true><<<grid, 256, 0, st>>>(col, w, n, arcs, wbits, err, max_w, cnt);
  else k_validate_arcs<false><<<grid, 256, 0, st>>>(col, w, n, arcs, wbits, err, max_w, cnt);
  count_launch();
  k_validate_sorted<<<1, 32, 0, st>>>(cnt, cnt + 1, err);
  count_launch();
  return cudaGetLastError();
}

// every arc (v, u) needs the arc (u, v): binary search of v in row u
__global__ void __launch_bounds__(256) k_check_sym(const uint64_t* __restrict__ rp, const uint32_t* __restrict__ col,
                                                   uint64_t n, int* err) {
  const int lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  int flags = 0;
  for (uint64_t v = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); v < n; v += warps) {
    for (uint64_t j = rp[v] + lane; j < rp[v + 1]; j += 32) {
      const uint32_t u = col[j];
      uint64_t lo = rp[u], hi = rp[u + 1];
      while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (col[mid] < v) lo = mid + 1; else hi = mid;
      }
      if (lo == rp[u + 1] || col[lo] != v) flags |= DERR_ASYM;
    }
  }
  flags = __reduce_or_sync(LG_FULL_MASK, flags);
  if (lane == 0 && flags) atomicOr(err, flags);
}

cudaError_t enc_check_symmetric(const uint64_t* rp, const uint32_t* col, uint64_t n, int* err, cudaStream_t st) {
  k_check_sym<<<grid_for(n, 8, 152 * 64), 256, 0, st>>>(rp, col, n, err);
  count_launch();
  return cudaGetLastError();
}

// =========================================================================
// local widths: w_v = max(1, bits(maxN_v)) (Section 3.2.2) or
// g_v = max(1, bits(max gap)) (Section 3.6); len_v = bits of the neighborhood
// =========================================================================
// One warp takes 32 consecutive rows (bounds loaded one per lane).  Local IDs:
// a row's width is that of its last (largest) ID.  Gaps: when the 32 rows hold
// at most LL_STAGE arcs (contiguous in col) the warp copies them to shared
// memory with coalesced loads and each lane scans its own row there; warps
// with a longer row (near the hubs) reduce row by row over the warp.
constexpr int LL_STAGE = 1024;
__global__ void __launch_bounds__(256) k_local_lengths(const uint64_t* __restrict__ rp,
                                                       const uint32_t* __restrict__ col, uint64_t n, int gap,
                                                       uint32_t s, uint32_t H, uint8_t* __restrict__ wid,
                                                       uint64_t* __restrict__ len) {
  __shared__ uint32_t stage[8][LL_STAGE];
  const int lane = threadIdx.x & 31;
  uint32_t* sk = stage[threadIdx.x >> 5];
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t v0 = ((uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; v0 < n; v0 += warps * 32) {
    const int rows = (int)min((uint64_t)32, n - v0);
    const uint64_t mv = v0 + lane;
    uint64_t mlo = 0, mhi = 0;
    if (lane < rows) { mlo = rp[mv]; mhi = rp[mv + 1]; }
    uint32_t mw = 0;  // lane l ends with the width of row v0 + l
    if (!gap && lane < rows && mhi > mlo) mw = max(1u, bits_u32(col[mhi - 1]));
    if (gap) {
      const uint64_t r0 = __shfl_sync(LG_FULL_MASK, mlo, 0);
      const uint64_t r1 = __shfl_sync(LG_FULL_MASK, mhi, rows - 1);
      if (r1 - r0 <= (uint64_t)LL_STAGE) {
        const uint32_t tot = (uint32_t)(r1 - r0);
        for (uint32_t q = lane; q < tot; q += 32) sk[q] = col[r0 + q];
        __syncwarp();
        if (lane < rows && mhi - mlo >= 2) {
          const uint32_t* row = sk + (mlo - r0);
          const uint32_t d = (uint32_t)(mhi - mlo);
          uint32_t prev = row[0], mg = 0;
          for (uint32_t t = 1; t < d; t++) {
            const uint32_t x = row[t];
            mg = max(mg, x - prev);
            prev = x;
          }
          mw = max(1u, bits_u32(mg));
        }
        __syncwarp();
      } else {
        for (int r = 0; r < rows; r++) {
          const uint64_t lo = __shfl_sync(LG_FULL_MASK, mlo, r), hi = __shfl_sync(LG_FULL_MASK, mhi, r);
          if (hi - lo < 2) continue;
          uint32_t mg = 0;
          for (uint64_t j = lo + 1 + lane; j < hi; j += 32) mg = max(mg, col[j] - col[j - 1]);
          mg = __reduce_max_sync(LG_FULL_MASK, mg);
          if (lane == r) mw = max(1u, bits_u32(mg));
        }
      }
    }
    if (lane < rows) {
      const uint64_t d = mhi - mlo;
      wid[mv] = (uint8_t)mw;
      len[mv] = gap ? (uint64_t)H + (d >= 1 ? s : 0) + (d >= 2 ? (d - 1) * (uint64_t)mw : 0)
                    : (uint64_t)H + d * (uint64_t)mw;
    }
  }
}

cudaError_t enc_local_lengths(const uint64_t* rp, const uint32_t* col, uint64_t n, int gap, uint32_t s, uint32_t H,
                              uint8_t* wid, uint64_t* len, cudaStream_t st) {
  k_local_lengths<<<grid_for(n, 256, 152 * 16), 256, 0, st>>>(rp, col, n, gap, s, H, wid, len);
  count_launch();
  return cudaGetLastError();
}

// =========================================================================
// fixed-width packing: record j = [id : s][weight : omega] at bit j * r
// (Sections 3.2.1 and 3.3; the weight directly after the ID).  One thread
// assembles one output word from the (at most 64/r + 2) records touching it.
// =========================================================================
// 64 records fill exactly r words: a warp takes one such chunk at a time,
// loads its 64 records coalesced into shared memory (ID | weight << s), then
// each lane assembles whole output words q = lane, lane + 32, ... of the chunk
// from the records overlapping them (the same records for every chunk, from a
// per-block table) and the r words go out as one coalesced store.
constexpr int PG_WARPS = 8;
__global__ void __launch_bounds__(PG_WARPS * 32) k_pack_global(const uint32_t* __restrict__ col,
                                                               const uint32_t* __restrict__ w, uint64_t arcs,
                                                               uint32_t s, uint32_t omega, uint64_t* __restrict__ out,
                                                               uint64_t data_words) {
  const uint32_t r = s + omega;  // 1..64
  __shared__ uint8_t tj0[64], tj1[64];  // first and last record of word q within a chunk of 64 records
  __shared__ uint64_t recs[PG_WARPS][64];
  if (threadIdx.x < r) {
    tj0[threadIdx.x] = (uint8_t)(threadIdx.x * 64u / r);
    tj1[threadIdx.x] = (uint8_t)((threadIdx.x * 64u + 63u) / r);
  }
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
  uint64_t* rec = recs[wid];
  const uint64_t nchunks = (arcs + 63) / 64;
  for (uint64_t c = (uint64_t)blockIdx.x * PG_WARPS + wid; c < nchunks; c += (uint64_t)gridDim.x * PG_WARPS) {
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const uint64_t j = c * 64 + 32u * h + lane;
      uint64_t x = 0;
      if (j < arcs) {
        x = (uint64_t)col[j];
        if (w) x |= (uint64_t)w[j] << s;
      }
      rec[32 * h + lane] = x;  // records past the last arc are zero
    }
    __syncwarp();
    for (uint32_t q = lane; q < r; q += 32) {
      const uint64_t k = c * r + q;
      if (k < data_words) {
        uint64_t acc = 0;
        for (uint32_t j = tj0[q]; j <= tj1[q]; j++) {
          const int off = (int)(j * r) - (int)(q * 64u);
          acc |= off >= 0 ? (rec[j] << off) : (rec[j] >> (-off));
        }
        out[k] = acc;
      }
    }
    __syncwarp();
  }
}

cudaError_t enc_pack_global(const uint32_t* col, const uint32_t* w, uint64_t arcs, uint32_t s, uint32_t omega,
                            uint64_t* out, uint64_t data_words, cudaStream_t st) {
  if (data_words == 0) return cudaSuccess;
  k_pack_global<<<grid_for((arcs + 63) / 64, PG_WARPS, 152 * 12), PG_WARPS * 32, 0, st>>>(col, w, arcs, s, omega,
                                                                                          out, data_words);
  count_launch();
  return cudaGetLastError();
}

// value j (u64, w <= 64 bits) at bit j * w
__global__ void __launch_bounds__(256) k_pack_u64(const uint64_t* __restrict__ vals, uint64_t count, uint32_t wbits,
                                                  uint64_t* __restrict__ out, uint64_t data_words) {
  const uint64_t mask = wbits >= 64 ? ~0ull : ((1ull << wbits) - 1ull);
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < data_words;
       k += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t b0 = k * 64;
    const uint64_t j0 = b0 / wbits;
    uint64_t j1 = (b0 + 63) / wbits;
    if (j1 >= count) j1 = count - 1;
    uint64_t acc = 0;
    for (uint64_t j = j0; j <= j1; j++) {
      const uint64_t rec = vals[j] & mask;
      const int64_t off = (int64_t)(j * wbits) - (int64_t)b0;
      acc |= off >= 0 ? (rec << off) : (rec >> (-off));
    }
    out[k] = acc;
  }
}

cudaError_t enc_pack_u64(const uint64_t* vals, uint64_t count, uint32_t w, uint64_t* out, uint64_t data_words,
                         cudaStream_t st) {
  if (data_words == 0 || w == 0) return cudaSuccess;
  k_pack_u64<<<grid_for(data_words, 256, 152 * 32), 256, 0, st>>>(vals, count, w, out, data_words);
  count_launch();
  return cudaGetLastError();
}

// =========================================================================
// variable-width local packing (Sections 3.2.2 / 3.6): vertex v's record
// [w_v : H][first : s][(d-1) gaps : w_v] (gaps) or [w_v : H][d IDs : w_v]
// starts at bit x[v].  A warp takes PK_ROWS consecutive rows.  If they hold at
// most PK_ARCS arcs, their arcs are staged in shared memory with coalesced
// loads and each lane emits its row's record into a shared copy of the
// group's bit range (shared atomicOr, as neighbouring records share words).
// Otherwise the warp packs the rows one at a time, in windows of up to
// PK_ARCS fields, a lane per field.  Either way the warp then writes the bit
// range out coalesced: its inner 64-bit words are its own, its first and last
// word may be shared with the neighbouring range and are OR-ed into A (zeroed
// at allocation).
// =========================================================================
constexpr int PK_ROWS = 32;
constexpr int PK_ARCS = 1024;
constexpr int PK_STAGE = PK_ARCS + 8;  // a window's fields, plus the ID before them (gaps)
constexpr int PK_W32 = 1104;           // >= 2 * ceil((PK_ARCS * 32 + PK_ROWS * 64 + 63) / 64), even
constexpr int PK_WARPS = 4;

__device__ __forceinline__ void pk_emit(uint32_t* ob, uint64_t p, uint32_t w, uint32_t val) {
  if (w == 0) return;
  const uint32_t i = (uint32_t)(p >> 5), sh = (uint32_t)p & 31u;
  atomicOr(&ob[i], val << sh);
  if (sh + w > 32) atomicOr(&ob[i + 1], val >> (32 - sh));
}

// bits [b0, b1) of A, held in ob from bit (b0 & ~63): inner words stored,
// the first and last OR-ed in
__device__ __forceinline__ void pk_flush(const uint32_t* ob, uint64_t b0, uint64_t b1, uint64_t* out, int lane) {
  const uint64_t base = b0 & ~63ull;
  const uint32_t nw64 = (uint32_t)((b1 - base + 63) >> 6);
  for (uint32_t j = lane; j < nw64; j += 32) {
    const uint64_t val = (uint64_t)ob[2 * j] | ((uint64_t)ob[2 * j + 1] << 32);
    uint64_t* dst = out + (base >> 6) + j;
    if (j == 0 || j + 1 == nw64) atomicOr(reinterpret_cast<unsigned long long*>(dst), (unsigned long long)val);
    else __stcs(dst, val);
  }
}

__device__ __forceinline__ void pk_clear(uint32_t* ob, uint64_t b0, uint64_t b1, int lane) {
  const uint32_t n32 = 2 * (uint32_t)((b1 - (b0 & ~63ull) + 63) >> 6);
  for (uint32_t q = lane; q < n32; q += 32) ob[q] = 0;
}

template <bool GAP>
__global__ void __launch_bounds__(PK_WARPS * 32) k_pack_local(const uint64_t* __restrict__ rp,
                                                             const uint32_t* __restrict__ col,
                                                             const uint64_t* __restrict__ x,
                                                             const uint8_t* __restrict__ wid, uint64_t n, uint32_t s,
                                                             uint32_t H, uint64_t* __restrict__ out) {
  __shared__ uint32_t stg_all[PK_WARPS][PK_STAGE];
  __shared__ uint32_t ob_all[PK_WARPS][PK_W32];
  const int lane = threadIdx.x & 31;
  uint32_t* stg = stg_all[threadIdx.x >> 5];
  uint32_t* ob = ob_all[threadIdx.x >> 5];
  const uint64_t groups = (n + PK_ROWS - 1) / PK_ROWS;
  const uint64_t warps = (uint64_t)gridDim.x * PK_WARPS;
  for (uint64_t gi = (uint64_t)blockIdx.x * PK_WARPS + (threadIdx.x >> 5); gi < groups; gi += warps) {
    const uint64_t v0 = gi * PK_ROWS;
    const int rows = (int)min((uint64_t)PK_ROWS, n - v0);
    uint64_t mlo = 0, mhi = 0, xb = 0, xe = 0;
    uint32_t wv = 0;
    if (lane < rows) {
      mlo = rp[v0 + lane];
      mhi = rp[v0 + lane + 1];
      xb = x[v0 + lane];
      xe = x[v0 + lane + 1];
      wv = wid[v0 + lane];
    }
    const uint64_t r0 = __shfl_sync(LG_FULL_MASK, mlo, 0);
    const uint64_t r1 = __shfl_sync(LG_FULL_MASK, mhi, rows - 1);
    if (r1 - r0 <= (uint64_t)PK_ARCS) {  // the whole group at once, a lane per row
      const uint64_t B0 = __shfl_sync(LG_FULL_MASK, xb, 0);
      const uint64_t B1 = __shfl_sync(LG_FULL_MASK, xe, rows - 1);
      const uint64_t base = B0 & ~63ull;
      const uint32_t tot = (uint32_t)(r1 - r0);
      for (uint32_t q = lane; q < tot; q += 32) stg[q] = col[r0 + q];
      pk_clear(ob, B0, B1, lane);
      __syncwarp();
      if (lane < rows) {
        const uint32_t* row = stg + (mlo - r0);
        const uint32_t d = (uint32_t)(mhi - mlo);
        uint64_t p = xb - base;
        pk_emit(ob, p, H, wv);
        p += H;
        if (GAP) {
          if (d >= 1) {
            pk_emit(ob, p, s, row[0]);
            p += s;
            uint32_t prev = row[0];
            for (uint32_t t = 1; t < d; t++) {
              const uint32_t cur = row[t];
              pk_emit(ob, p, wv, cur - prev);
              prev = cur;
              p += wv;
            }
          }
        } else {
          for (uint32_t t = 0; t < d; t++) {
            pk_emit(ob, p, wv, row[t]);
            p += wv;
          }
        }
      }
      __syncwarp();
      pk_flush(ob, B0, B1, out, lane);
      __syncwarp();
      continue;
    }
    // long rows present: one row at a time, windows of up to PK_ARCS fields
    for (int r = 0; r < rows; r++) {
      const uint64_t lo = __shfl_sync(LG_FULL_MASK, mlo, r), hi = __shfl_sync(LG_FULL_MASK, mhi, r);
      const uint64_t rb = __shfl_sync(LG_FULL_MASK, xb, r), re = __shfl_sync(LG_FULL_MASK, xe, r);
      const uint32_t w = __shfl_sync(LG_FULL_MASK, wv, r);
      const uint64_t d = hi - lo;
      const uint64_t f0 = rb + H + (GAP && d >= 1 ? s : 0);  // bit of data field 0
      const uint64_t nf = GAP ? (d >= 1 ? d - 1 : 0) : d;    // data fields
      // data field k: gaps col[lo+k+1] - col[lo+k], or IDs col[lo+k]
      for (uint64_t k0 = 0; k0 == 0 || k0 < nf; k0 += PK_ARCS) {
        const uint32_t kn = (uint32_t)min((uint64_t)PK_ARCS, nf - min(nf, k0));
        const uint64_t b0 = k0 == 0 ? rb : f0 + k0 * w;
        const uint64_t b1 = k0 + kn >= nf ? re : f0 + (k0 + kn) * w;
        const uint64_t base = b0 & ~63ull;
        // staged IDs: the window's fields, plus the ID before the first gap
        const uint32_t ns = GAP ? (d >= 1 ? kn + 1u : 0u) : kn;
        for (uint32_t q = lane; q < ns; q += 32) stg[q] = col[lo + k0 + q];
        pk_clear(ob, b0, b1, lane);
        __syncwarp();
        if (k0 == 0 && lane == 0) {
          pk_emit(ob, rb - base, H, w);
          if (GAP && d >= 1) pk_emit(ob, rb + H - base, s, stg[0]);
        }
        for (uint32_t q = lane; q < kn; q += 32) {
          const uint32_t val = GAP ? stg[q + 1] - stg[q] : stg[q];
          pk_emit(ob, f0 + (k0 + q) * w - base, w, val);
        }
        __syncwarp();
        pk_flush(ob, b0, b1, out, lane);
        __syncwarp();
      }
    }
  }
}

cudaError_t enc_pack_local(const uint64_t* rp, const uint32_t* col, const uint64_t* x, const uint8_t* wid, uint64_t n,
                           int gap, uint32_t s, uint32_t H, uint64_t* out, uint64_t data_words, cudaStream_t st) {
  if (data_words == 0 || n == 0) return cudaSuccess;
  const unsigned grid = grid_for((n + PK_ROWS - 1) / PK_ROWS, PK_WARPS, 152 * 16);
  if (gap) k_pack_local<true><<<grid, PK_WARPS * 32, 0, st>>>(rp, col, x, wid, n, s, H, out);
  else k_pack_local<false><<<grid, PK_WARPS * 32, 0, st>>>(rp, col, x, wid, n, s, H, out);
  count_launch();
  return cudaGetLastError();
}

// =========================================================================
// Elias-Fano (Section 4.3): one set bit per value at (x_i >> l) + i, and the
// select samples S[k] = (x_{k*sample} >> l) + k*sample.  Each warp combines
// the bits that fall into the same word before one atomicOr per word.
// =========================================================================
__global__ void __launch_bounds__(256) k_ef_high(const uint64_t* __restrict__ x, uint64_t N, uint32_t l,
                                                 unsigned long long* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  for (uint64_t base = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~31ull; base < N;
       base += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = base + lane;
    const bool ok = i < N;
    const uint64_t pos = ok ? (x[i] >> l) + i : 0;
    const uint64_t word = ok ? pos >> 6 : ~0ull;
    unsigned long long bit = ok ? (1ull << (pos & 63)) : 0ull;
    // positions increase with i, so equal words are adjacent lanes: segmented OR
    const uint64_t prev_word = __shfl_up_sync(LG_FULL_MASK, word, 1);
    const bool head = lane == 0 || prev_word != word;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long b = __shfl_down_sync(LG_FULL_MASK, bit, o);
      const uint64_t wd = __shfl_down_sync(LG_FULL_MASK, word, o);
      if (lane + o < 32 && wd == word) bit |= b;
    }
    if (ok && head) atomicOr(&out[word], bit);
  }
}

cudaError_t enc_ef_high(const uint64_t* x, uint64_t N, uint32_t l, uint64_t* out, cudaStream_t st) {
  k_ef_high<<<grid_for(N, 256, 152 * 32), 256, 0, st>>>(x, N, l, reinterpret_cast<unsigned long long*>(out));
  count_launch();
  return cudaGetLastError();
}

__global__ void k_ef_samples(const uint64_t* __restrict__ x, uint64_t N, uint32_t l, uint32_t sample,
                             uint64_t* __restrict__ out, uint64_t ns) {
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < ns; k += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = k * sample;
    if (i < N) out[k] = (x[i] >> l) + i;
  }
}

cudaError_t enc_ef_samples(const uint64_t* x, uint64_t N, uint32_t l, uint32_t sample, uint64_t* out, uint64_t ns,
                           cudaStream_t st) {
  if (ns == 0) return cudaSuccess;
  k_ef_samples<<<grid_for(ns, 256, 4096), 256, 0, st>>>(x, N, l, sample, out, ns);
  count_launch();
  return cudaGetLastError();
}

}  // namespace lg
