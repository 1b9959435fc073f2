// Device-side building blocks shared by the encoder and the traversal kernels.
//
// Bit order (Listing 2, Section 3.7.2 of the Log(Graph) paper): a stream is an
// array of little-endian words; a w-bit field at bit position p holds value
// bit k at stream bit p + k.  On a little-endian GPU the same memory read as
// 32-bit or 64-bit words gives the same bit positions, so the decoders read
// 32-bit words and use one funnel shift per field.
//
// Every stream allocation is padded to an even number of u64 words and
// followed by four zero guard words (32 bytes), so a read of the word after a
// data word, or of the aligned 32-byte sector holding it, stays inside the
// allocation.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#define LG_FULL_MASK 0xffffffffu

namespace lg {

enum IdMode : int { ID_GLOBAL = 0, ID_LOCAL = 1, ID_LOCAL_GAP = 2, ID_CSR32 = 3 };
enum OffMode : int { OFF_PACKED = 0, OFF_EF = 1, OFF_ROWPTR = 2 };

// Device error flag bits (combined with atomicOr; read back by the host).
enum DevErr : int {
  DERR_ROWPTR = 1,      // row_ptr not monotone / out of range
  DERR_COL_RANGE = 2,   // neighbor id >= n
  DERR_UNSORTED = 4,    // row not strictly increasing
  DERR_WEIGHT = 8,      // weight does not fit the requested width
  DERR_ASYM = 16,       // an arc without its reverse
  DERR_QUERY = 32,      // query vertex >= n
  DERR_INTERNAL = 64,   // a structural invariant did not hold (bounded loop ran out)
};

constexpr int LG_TILE_V = 512;  // vertices per tile of the pull kernels

// One unit of the heavy-vertex schedule: fields [f0, f0 + nf) of vertex v.
// Vertices whose degree exceeds the light limit are split into items of at
// most heavy_seg fields so that no single warp walks a whole hub; `carry` is
// the absolute neighbor ID just before field f0 (gap-coded IDs only).
struct HeavyItem {
  uint64_t bit;        // stream bit of the vertex's first field
  uint32_t v;          // stored label
  uint32_t f0, nf;     // field range
  uint32_t carry;      // running ID before f0 (local-gap mode)
  uint32_t deg;        // degree of v
  uint32_t first;      // index of the vertex's first item
  uint32_t nitems;     // items of this vertex
  uint32_t w;          // field width (gap width for local-gap)
  uint32_t slot;       // index among the split vertices (0xffffffff if not split)
};

// Read-only view of an encoded graph, passed by value to kernels.
struct GView {
  const uint32_t* A32;        // A stream as 32-bit words (CSR32: the col array)
  const uint64_t* A64;        // same memory as 64-bit words
  const uint64_t* O;          // packed offsets (PACKED) or row_ptr (ROWPTR)
  const uint64_t* ef_low;
  const uint32_t* ef_high32;  // EF high bits as 32-bit words
  const uint64_t* ef_samples;
  const uint32_t* perm;       // original -> stored (nullptr without relabel)
  const uint32_t* inv_perm;   // stored -> original
  const uint32_t* W32;        // CSR32 only: 32-bit weights beside the IDs (nullptr if none)
  const HeavyItem* items;     // heavy-vertex schedule (nullptr if none)
  const uint32_t* multi;      // first item of every vertex split into > 1 item
  uint64_t n, arcs;
  uint64_t ef_high_words32;   // number of valid 32-bit words of the high vector
  uint64_t n_items, n_multi;
  uint32_t s, H, omega, r, w_O, ef_l, sample_log2;
  uint32_t heavy_min;         // degrees above this are in the schedule
  uint32_t heavy_seg;         // max fields per schedule item
};

__device__ __forceinline__ uint32_t bits_u32(uint32_t x) { return 32u - __clz(x); }
__device__ __forceinline__ uint32_t bits_u64(uint64_t x) { return 64u - __clzll(x); }

__device__ __forceinline__ uint32_t mask_lo(uint32_t w) { return w >= 32 ? 0xffffffffu : ((1u << w) - 1u); }

// w <= 32 bit field at bit p of a 32-bit word stream.
__device__ __forceinline__ uint32_t ext32(const uint32_t* __restrict__ A, uint64_t p, uint32_t w) {
  const uint64_t wi = p >> 5;
  const uint32_t lo = __ldg(A + wi);
  const uint32_t hi = __ldg(A + wi + 1);
  return __funnelshift_r(lo, hi, (uint32_t)p & 31u) & mask_lo(w);
}

// w <= 64 bit field at bit p of a 64-bit word stream.
__device__ __forceinline__ uint64_t ext64(const uint64_t* __restrict__ A, uint64_t p, uint32_t w) {
  const uint64_t wi = p >> 6;
  const uint32_t sh = (uint32_t)p & 63u;
  const uint64_t lo = __ldg(A + wi);
  const uint64_t hi = __ldg(A + wi + 1);
  const uint64_t v = sh ? ((lo >> sh) | (hi << (64u - sh))) : lo;
  return w >= 64 ? v : (v & ((1ull << w) - 1ull));
}

// Position (0..31) of the r-th set bit (0-based) of x; requires r < popc(x).
__device__ __forceinline__ uint32_t select_in_u32(uint32_t x, uint32_t r) {
  uint32_t pos = 0, c;
  c = __popc(x & 0xffffu); if (r >= c) { r -= c; x >>= 16; pos += 16; }
  c = __popc(x & 0xffu);   if (r >= c) { r -= c; x >>= 8;  pos += 8; }
  c = __popc(x & 0xfu);    if (r >= c) { r -= c; x >>= 4;  pos += 4; }
  c = __popc(x & 0x3u);    if (r >= c) { r -= c; x >>= 2;  pos += 2; }
  c = x & 1u;              if (r >= c) { pos += 1; }
  return pos;
}

// 128-bit read-only load (address must be 16-byte aligned).
__device__ __forceinline__ uint4 ldg128(const uint32_t* p) { return __ldg(reinterpret_cast<const uint4*>(p)); }

// ---------------------------------------------------------------------------
// L2 eviction priority (a per-instruction cache policy, no device state): the
// compressed stream is read once per sweep and marked evict-first, so it does
// not push the gathered per-vertex arrays out of L2.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t policy_stream() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_keep() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// one whole 32-byte sector (p 32-byte aligned) in a single request
__device__ __forceinline__ void ldg256_stream(const uint32_t* p, uint64_t pol, uint4& a, uint4& b) {
  asm("ld.global.nc.L2::cache_hint.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8], %9;"
      : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
      : "l"(p), "l"(pol));
}
// Gathers of per-vertex arrays keep the default L1 allocation (on this GPU a
// no-allocate L1 hint made 392M random 4-byte gathers 3.5x slower, measured)
// and mark their L2 lines evict-last, so the stream and the freshly written
// next-iteration array are evicted before them.
__device__ __forceinline__ float ldg_gather(const float* p, uint64_t pol) {
  float v;
  asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
  return v;
}
// one 32-bit word with an L2 cache policy
__device__ __forceinline__ uint32_t ldg_hint(const uint32_t* p, uint64_t pol) {
  uint32_t v;
  asm("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
// four consecutive floats (16-byte aligned), same policy
__device__ __forceinline__ float4 ldg_gather4(const float* p, uint64_t pol) {
  float4 v;
  asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
      : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
      : "l"(p), "l"(pol));
  return v;
}
// BFS frontier masks (2, 4 or 8 bytes per vertex), same policy argument
__device__ __forceinline__ uint16_t ldg_gather(const uint16_t* p, uint64_t pol) {
  uint16_t v;
  asm("ld.global.nc.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ uint32_t ldg_gather(const uint32_t* p, uint64_t pol) {
  uint32_t v;
  asm("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ uint64_t ldg_gather(const uint64_t* p, uint64_t pol) {
  uint64_t v;
  asm("ld.global.nc.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(pol));
  return v;
}

// ---------------------------------------------------------------------------
// Sequential bit reader: one thread walks a run of fields (w <= 32 bits).  The
// window lo:hi holds the 64 stream bits starting at word `wnext - 2`; a field
// at bit offset o (< 32) of lo is one funnel shift and a mask, and advancing
// past lo shifts the window by one word.  Words come from whole 32-byte
// sectors (two 128-bit loads of one aligned sector) held in registers, so a
// warp whose lanes walk different runs issues one sector request per lane per
// 256 bits.  The window runs one word ahead of the last field read, which the
// 32-byte zero guard after every stream keeps inside the allocation.
// ---------------------------------------------------------------------------
struct BitReader {
  const uint32_t* A;
  uint64_t pol;       // L2 policy of the stream loads
  uint64_t wnext;     // index of the next word to enter the window
  uint32_t lo, hi;    // the window
  uint32_t o;         // bit offset of the next field in lo, 0..31
  uint4 q0, q1;       // next words of the current sector, q0 first (shifted down)
  uint32_t n0, n1;    // valid words in q0, q1

  __device__ __forceinline__ void load_sector() {
    const uint64_t c = wnext & ~7ull;  // the stream is 32-byte aligned (alloc_words)
    uint4 a, b;
    ldg256_stream(A + c, pol, a, b);
    uint32_t skip = (uint32_t)(wnext - c);
    if (skip >= 4) { a = b; n1 = 0; skip -= 4; } else { n1 = 4; }
    if (skip >= 1) { a.x = a.y; a.y = a.z; a.z = a.w; }
    if (skip >= 2) { a.x = a.y; a.y = a.z; }
    if (skip >= 3) { a.x = a.y; }
    q0 = a;
    q1 = b;
    n0 = 4u - skip;
  }
  __device__ __forceinline__ uint32_t next_word() {
    if (n0 == 0) {
      if (n1) { q0 = q1; n0 = n1; n1 = 0; }
      else load_sector();
    }
    const uint32_t x = q0.x;
    q0.x = q0.y; q0.y = q0.z; q0.z = q0.w;
    n0--;
    wnext++;
    return x;
  }
  __device__ __forceinline__ void init(const uint32_t* base, uint64_t bit, uint64_t policy) {
    A = base;
    pol = policy;
    wnext = bit >> 5;
    n0 = 0; n1 = 0;
    lo = next_word();
    hi = next_word();
    o = (uint32_t)bit & 31u;
  }
  // w <= 32
  __device__ __forceinline__ uint32_t get(uint32_t w) {
    const uint32_t v = __funnelshift_r(lo, hi, o) & mask_lo(w);
    o += w;
    if (o >= 32) {
      o -= 32;
      lo = hi;
      hi = next_word();
    }
    return v;
  }
  __device__ __forceinline__ void skip(uint32_t w) { (void)get(w); }
};

// ---------------------------------------------------------------------------
// warp / block scans
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_incl_scan(T x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(LG_FULL_MASK, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(LG_FULL_MASK, x, o);
  return x;
}

template <typename T>
__device__ __forceinline__ T warp_or(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x |= __shfl_xor_sync(LG_FULL_MASK, x, o);
  return x;
}

// Exclusive scan over a block of NT threads; `tmp` holds NT/32 elements of
// shared memory.  Returns the exclusive prefix and the block total.
template <typename T, int NT>
__device__ __forceinline__ T block_excl_scan(T v, T& total, T* tmp) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int NW = NT / 32;
  T x = warp_incl_scan(v);
  if (lane == 31) tmp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    T w = lane < NW ? tmp[lane] : T(0);
    w = warp_incl_scan(w);
    if (lane < NW) tmp[lane] = w;
  }
  __syncthreads();
  const T pre = (wid > 0 ? tmp[wid - 1] : T(0)) + x - v;
  total = tmp[NW - 1];
  __syncthreads();
  return pre;
}

// Two exclusive scans over a block of NT threads in one pass (one tree, two
// values); `tmp` holds 2 * NT/32 elements of shared memory.
template <typename T, int NT>
__device__ __forceinline__ void block_excl_scan2(T a, T b, T& pa, T& pb, T& ta, T& tb, T* tmp) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int NW = NT / 32;
  const T xa = warp_incl_scan(a), xb = warp_incl_scan(b);
  if (lane == 31) { tmp[wid] = xa; tmp[NW + wid] = xb; }
  __syncthreads();
  if (wid == 0) {
    T ya = lane < NW ? tmp[lane] : T(0), yb = lane < NW ? tmp[NW + lane] : T(0);
    ya = warp_incl_scan(ya);
    yb = warp_incl_scan(yb);
    if (lane < NW) { tmp[lane] = ya; tmp[NW + lane] = yb; }
  }
  __syncthreads();
  pa = (wid > 0 ? tmp[wid - 1] : T(0)) + xa - a;
  pb = (wid > 0 ? tmp[NW + wid - 1] : T(0)) + xb - b;
  ta = tmp[NW - 1];
  tb = tmp[2 * NW - 1];
  __syncthreads();
}

__device__ __forceinline__ void set_err(int* err, int bit) { atomicOr(err, bit); }

// ---------------------------------------------------------------------------
// Warp-flattened walk over the entries of 32 consecutive rows: lane r holds
// row r's entry count; lane l then visits flattened entries l, l + 32, ...
// (entry f of row r with pre[r] <= f < pre[r+1]), so every lane is busy
// whatever the row lengths and the loads of different rows overlap.
// `pre` is 33 words of per-warp shared memory.
// ---------------------------------------------------------------------------
template <class Body>
__device__ __forceinline__ void warp_flat(uint64_t* pre, uint64_t my_count, Body body) {
  const int lane = threadIdx.x & 31;
  const uint64_t incl = warp_incl_scan<uint64_t>(my_count);
  pre[lane + 1] = incl;
  if (lane == 0) pre[0] = 0;
  __syncwarp();
  const uint64_t total = __shfl_sync(LG_FULL_MASK, incl, 31);
#pragma unroll 2
  for (uint64_t base = 0; base < total; base += 32) {
    const uint64_t f = base + lane;
    if (f < total) {
      int r = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1)
        if (pre[r + step] <= f) r += step;
      body(r, f - pre[r]);
    }
  }
  __syncwarp();
}

}  // namespace lg
