// Graph kernels with the Log(Graph) decoder fused in (Sections 3.7.2-3.7.3 for
// the access path, Section 7.1.2 for BFS and PageRank).
//
// Pull sweeps (PageRank, bottom-up BFS) are one launch with two kinds of CTA:
//   * heavy CTAs walk the heavy-vertex schedule built at encode time: vertices
//     of degree > heavy_min split into items of <= heavy_seg fields, one warp per
//     item, lane i decoding field i of each 32-field chunk with 4 chunks in
//     flight (gap-coded IDs by a warp prefix sum from the item's carry);
//   * tile CTAs take 512 consecutive stored labels each:
//     1. offsets x_v of the tile (packed fields, CSR row_ptr, or an
//        Elias-Fano block decode: the tile starts on a select sample, the CTA
//        popcounts the high-bit words it spans and every thread selects one
//        vertex's one);
//     2. per vertex: degree and field width from the offsets and the
//        neighborhood header;
//     3. light vertices (degree <= heavy_min) are split over the threads in
//        contiguous runs of nearly equal field counts, each thread decoding
//        its run with a sequential bit reader (one 32-byte sector per 256 bits,
//        a shift and a mask per field, a running sum for gap-coded IDs, four
//        gathers in flight).
// Vertices split into several items are finished by a small second kernel.
// Push steps and neighbor queries decode one random vertex per warp.
#pragma once

#include "lg_internal.h"

namespace lg {

constexpr int TV = LG_TILE_V;  // vertices per tile
constexpr int TNT = 256;       // threads per tile CTA
// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t udiv_small(uint64_t a, uint32_t b) {
  return a < 0x100000000ull ? (uint64_t)((uint32_t)a / b) : a / b;
}
__device__ __forceinline__ uint32_t lane_lt_mask() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <typename M> __device__ __forceinline__ M atomic_or_mask(M* p, M m);
template <> __device__ __forceinline__ uint16_t atomic_or_mask<uint16_t>(uint16_t* p, uint16_t m) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  uint32_t* w = reinterpret_cast<uint32_t*>(a & ~(uintptr_t)3);
  const uint32_t sh = (uint32_t)(a & 2) * 8u;
  return (uint16_t)(atomicOr(w, (uint32_t)m << sh) >> sh);
}
template <> __device__ __forceinline__ uint32_t atomic_or_mask<uint32_t>(uint32_t* p, uint32_t m) {
  return atomicOr(p, m);
}
template <> __device__ __forceinline__ uint64_t atomic_or_mask<uint64_t>(uint64_t* p, uint64_t m) {
  return (uint64_t)atomicOr(reinterpret_cast<unsigned long long*>(p), (unsigned long long)m);
}

// depth of v for every source in bitsv: row s of the S x n array, or row
// rows[s] when the caller keeps one separate row per source (a source that
// joined a running sweep at level row_base[s] counts depths from there)
template <typename M>
__device__ __forceinline__ void write_depths(const BfsArgs& a, uint64_t n, uint64_t v, M bitsv, uint32_t d) {
  uint64_t b = (uint64_t)bitsv;
  while (b) {
    const int s = __ffsll((long long)b) - 1;
    b &= b - 1;
    if (a.rows) a.rows[s][a.row_perm ? (uint64_t)a.row_perm[v] : v] = d - a.row_base[s];
    else if (a.vmajor) a.depth[v * a.S + s] = d;
    else a.depth[(uint64_t)s * n + v] = d;
  }
}

// ---------------------------------------------------------------------------
// offsets of a tile: xs[i] = x_{v0+i}, i = 0..cnt (cnt+1 values)
// ---------------------------------------------------------------------------
struct TileScratch {
  uint32_t cum[TNT];
  uint32_t w[TNT];
  uint32_t red[TNT / 32];
};

template <int OFF>
__device__ __forceinline__ void tile_offsets(const GView& g, uint64_t v0, int cnt, uint64_t* xs, TileScratch& ts);

template <>
__device__ __forceinline__ void tile_offsets<OFF_PACKED>(const GView& g, uint64_t v0, int cnt, uint64_t* xs,
                                                         TileScratch&) {
  for (int i = threadIdx.x; i <= cnt; i += TNT) xs[i] = ext64(g.O, (v0 + i) * g.w_O, g.w_O);
}

template <>
__device__ __forceinline__ void tile_offsets<OFF_ROWPTR>(const GView& g, uint64_t v0, int cnt, uint64_t* xs,
                                                         TileScratch&) {
  for (int i = threadIdx.x; i <= cnt; i += TNT) xs[i] = __ldg(g.O + v0 + i);
}

// Elias-Fano block decode (Section 4.3): ones number v0 .. v0+cnt of the high
// vector, starting from the sample at or below v0.
template <>
__device__ __forceinline__ void tile_offsets<OFF_EF>(const GView& g, uint64_t v0, int cnt, uint64_t* xs,
                                                     TileScratch& ts) {
  const uint64_t k = v0 >> g.sample_log2;
  const uint64_t p0 = __ldg(g.ef_samples + k);
  const uint64_t skip = v0 - (k << g.sample_log2);
  const uint64_t need_end = skip + (uint64_t)cnt + 1;
  uint64_t wbase = p0 >> 5;
  uint64_t carry = 0;
  bool first = true;
  while (carry < need_end && wbase < g.ef_high_words32) {
    const uint64_t wi = wbase + threadIdx.x;
    uint32_t w = wi < g.ef_high_words32 ? __ldg(g.ef_high32 + wi) : 0u;
    if (first && threadIdx.x == 0) w &= (0xffffffffu << ((uint32_t)p0 & 31u));
    uint32_t total;
    const uint32_t pre = block_excl_scan<uint32_t, TNT>((uint32_t)__popc(w), total, ts.red);
    ts.cum[threadIdx.x] = pre;
    ts.w[threadIdx.x] = w;
    __syncthreads();
    const uint64_t r_lo = carry > skip ? carry : skip;
    const uint64_t r_hi = (carry + total) < need_end ? (carry + total) : need_end;
    for (uint64_t r = r_lo + threadIdx.x; r < r_hi; r += TNT) {
      const uint32_t local = (uint32_t)(r - carry);
      int lo = 0, hi = TNT - 1;
      while (lo < hi) {
        const int m = (lo + hi + 1) >> 1;
        if (ts.cum[m] <= local) lo = m; else hi = m - 1;
      }
      const uint64_t pos = (wbase + (uint64_t)lo) * 32u + select_in_u32(ts.w[lo], local - ts.cum[lo]);
      const uint64_t i = r - skip;
      xs[i] = (pos - (v0 + i)) << g.ef_l;
    }
    carry += total;
    wbase += TNT;
    first = false;
    __syncthreads();
  }
  if (g.ef_l)
    for (int i = threadIdx.x; i <= cnt; i += TNT) xs[i] |= ext64(g.ef_low, (v0 + i) * g.ef_l, g.ef_l);
}

// ---------------------------------------------------------------------------
// random-access offsets x_v, x_{v+1}; called by all 32 lanes of a warp
// ---------------------------------------------------------------------------
template <int OFF>
__device__ __forceinline__ void offset_pair(const GView& g, uint64_t v, uint64_t& x0, uint64_t& x1);

template <>
__device__ __forceinline__ void offset_pair<OFF_PACKED>(const GView& g, uint64_t v, uint64_t& x0, uint64_t& x1) {
  x0 = ext64(g.O, v * g.w_O, g.w_O);
  x1 = ext64(g.O, (v + 1) * g.w_O, g.w_O);
}
template <>
__device__ __forceinline__ void offset_pair<OFF_ROWPTR>(const GView& g, uint64_t v, uint64_t& x0, uint64_t& x1) {
  x0 = __ldg(g.O + v);
  x1 = __ldg(g.O + v + 1);
}
// warp select of ones number v and v+1 (Section 4.1: O_v = select_O(v))
template <>
__device__ __forceinline__ void offset_pair<OFF_EF>(const GView& g, uint64_t v, uint64_t& x0, uint64_t& x1) {
  const int lane = threadIdx.x & 31;
  const uint64_t k = v >> g.sample_log2;
  const uint64_t p0 = __ldg(g.ef_samples + k);
  const uint64_t rem = v - (k << g.sample_log2);
  uint64_t wbase = p0 >> 5;
  uint64_t carry = 0;
  uint64_t pos[2] = {0, 0};
  uint32_t found = 0;
  bool first = true;
  while (found != 3u && wbase < g.ef_high_words32) {
    const uint64_t wi = wbase + lane;
    uint32_t w = wi < g.ef_high_words32 ? __ldg(g.ef_high32 + wi) : 0u;
    if (first && lane == 0) w &= (0xffffffffu << ((uint32_t)p0 & 31u));
    const uint32_t c = __popc(w);
    const uint32_t incl = warp_incl_scan<uint32_t>(c);
    const uint32_t excl = incl - c;
    const uint32_t total = __shfl_sync(LG_FULL_MASK, incl, 31);
#pragma unroll
    for (int t = 0; t < 2; t++) {
      const uint64_t target = rem + t;
      const bool here = !(found >> t & 1u) && carry + excl <= target && target < carry + incl;
      const uint32_t b = __ballot_sync(LG_FULL_MASK, here);
      uint64_t p = here ? wi * 32u + select_in_u32(w, (uint32_t)(target - carry - excl)) : 0;
      if (b) {
        p = __shfl_sync(LG_FULL_MASK, p, __ffs(b) - 1);
        pos[t] = p;
        found |= 1u << t;
      }
    }
    carry += total;
    wbase += 32;
    first = false;
  }
  const uint64_t lo0 = g.ef_l ? ext64(g.ef_low, v * g.ef_l, g.ef_l) : 0;
  const uint64_t lo1 = g.ef_l ? ext64(g.ef_low, (v + 1) * g.ef_l, g.ef_l) : 0;
  x0 = ((pos[0] - v) << g.ef_l) | lo0;
  x1 = ((pos[1] - (v + 1)) << g.ef_l) | lo1;
}

// ---------------------------------------------------------------------------
// neighborhood geometry from consecutive offsets (Section 3.7.3: d_v from
// O[v+1] - O[v]; in the local modes from the bit length and the header)
//   start: bit of the first field; w: field width (IDs, or gaps for LOCAL_GAP)
// ---------------------------------------------------------------------------
template <int IDM>
__device__ __forceinline__ void vgeo(const GView& g, uint64_t x0, uint64_t x1, uint64_t& start, uint32_t& deg,
                                     uint32_t& w) {
  if (IDM == ID_GLOBAL) {
    start = x0 * g.r; deg = (uint32_t)(x1 - x0); w = g.s;
  } else if (IDM == ID_CSR32) {
    start = x0 * 32u; deg = (uint32_t)(x1 - x0); w = 32;
  } else if (IDM == ID_LOCAL) {
    w = ext32(g.A32, x0, g.H);
    deg = w ? (uint32_t)udiv_small(x1 - x0 - g.H, w) : 0u;
    start = x0 + g.H;
  } else {
    w = ext32(g.A32, x0, g.H);
    const uint64_t len = x1 - x0;
    deg = len == g.H ? 0u : (w == 0 ? 1u : 1u + (uint32_t)udiv_small(len - g.H - g.s, w));
    start = x0 + g.H;
  }
}

// sequential decoder for one neighborhood (light path)
template <int IDM>
struct SeqDec {
  BitReader br;
  uint32_t w, s, omega, id;
  bool first;
  __device__ __forceinline__ void init(const GView& g, uint64_t start, uint32_t width, uint64_t pol) {
    br.init(g.A32, start, pol);
    w = width; s = g.s; omega = g.omega; id = 0; first = true;
  }
  __device__ __forceinline__ uint32_t next() {
    if (IDM == ID_GLOBAL) {
      const uint32_t v = br.get(s);
      if (omega) br.skip(omega);
      return v;
    } else if (IDM == ID_CSR32) {
      return br.get(32);
    } else if (IDM == ID_LOCAL) {
      return br.get(w);
    } else {
      id = first ? br.get(s) : id + br.get(w);
      first = false;
      return id;
    }
  }
};

// value of field i for the warp path (not yet prefix-summed for gaps)
template <int IDM>
__device__ __forceinline__ uint32_t field_at(const GView& g, uint64_t start, uint32_t w, uint64_t i) {
  if (IDM == ID_GLOBAL) return ext32(g.A32, start + i * g.r, g.s);
  if (IDM == ID_CSR32) return __ldg(g.A32 + (start >> 5) + i);
  if (IDM == ID_LOCAL) return ext32(g.A32, start + i * w, w);
  // the first field holds the absolute ID in s bits, the others gaps in w bits
  const uint64_t p = i == 0 ? start : start + g.s + (i - 1) * (uint64_t)w;
  return ext32(g.A32, p, i == 0 ? g.s : w);
}
__device__ __forceinline__ uint32_t weight_at(const GView& g, uint64_t start, uint64_t i) {
  return ext32(g.A32, start + i * g.r + g.s, g.omega);
}

// Lane-parallel decode of U chunks of 32 fields starting at field `base`
// (fields >= f1 read as 0).  Gap-coded IDs are prefix-summed across the warp
// with `carry` = the absolute ID before field `base`; carry is advanced.  All
// field loads of the U chunks are independent, so they are in flight together.
template <int IDM, int U>
__device__ __forceinline__ void warp_ids(const GView& g, uint64_t start, uint32_t w, uint32_t base, uint32_t f1,
                                         uint32_t& carry, uint32_t (&val)[U]) {
  const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
  for (int u = 0; u < U; u++) {
    const uint32_t idx = base + 32u * u + lane;
    val[u] = idx < f1 ? field_at<IDM>(g, start, w, idx) : 0u;
  }
  if (IDM == ID_LOCAL_GAP) {
#pragma unroll
    for (int u = 0; u < U; u++) {
      val[u] = warp_incl_scan<uint32_t>(val[u]) + carry;
      carry = __shfl_sync(LG_FULL_MASK, val[u], 31);
    }
  }
}

constexpr int HEAVY_U = 4;  // chunks of 32 fields in flight per warp

// ---------------------------------------------------------------------------
// tile phases shared by the pull kernels
// ---------------------------------------------------------------------------
struct TileSmem {
  uint64_t xs[TV + 1];     // offsets
  uint64_t st[TV];         // first-field bit of each vertex
  uint32_t deg[TV];
  uint32_t fpre[TV + 1];   // field prefix over the compacted light list
  uint16_t clist[TV];      // compacted light vertices (local index)
  uint8_t wid[TV];
  uint32_t nlight, nfields;
  uint64_t red64[TNT / 32];
  TileScratch ts;
};

// Phase 2: geometry of each vertex; light vertices (0 < degree <= heavy_min)
// that `keep(i)` accepts form the compacted, field-prefix-summed list.
// Heavier vertices are left to the heavy schedule.
template <int IDM, typename Keep>
__device__ __forceinline__ void tile_classify(const GView& g, TileSmem& sm, int cnt, Keep keep) {
  uint32_t lc = 0, lf = 0;
  bool light[TV / TNT];
#pragma unroll
  for (int q = 0; q < TV / TNT; q++) {
    const int i = threadIdx.x * (TV / TNT) + q;
    light[q] = false;
    if (i < cnt) {
      uint64_t start; uint32_t d, w;
      vgeo<IDM>(g, sm.xs[i], sm.xs[i + 1], start, d, w);
      sm.st[i] = start; sm.deg[i] = d; sm.wid[i] = (uint8_t)w;
      if (d > 0 && d <= g.heavy_min && keep(i)) { light[q] = true; lc++; lf += d; }
    }
  }
  uint64_t total;
  const uint64_t pre = block_excl_scan<uint64_t, TNT>(((uint64_t)lc << 32) | lf, total, sm.red64);
  uint32_t ci = (uint32_t)(pre >> 32), cf = (uint32_t)pre;
#pragma unroll
  for (int q = 0; q < TV / TNT; q++) {
    const int i = threadIdx.x * (TV / TNT) + q;
    if (light[q]) {
      sm.clist[ci] = (uint16_t)i;
      sm.fpre[ci] = cf;
      ci++;
      cf += sm.deg[i];
    }
  }
  if (threadIdx.x == 0) {
    sm.nlight = (uint32_t)(total >> 32);
    sm.nfields = (uint32_t)total;
    sm.fpre[sm.nlight] = (uint32_t)total;
  }
  __syncthreads();
}

// range of compacted light vertices owned by this thread (balanced by fields)
__device__ __forceinline__ void light_range(const TileSmem& sm, uint32_t& jb, uint32_t& je) {
  const uint64_t F = sm.nfields;
  const uint32_t flo = (uint32_t)((F * threadIdx.x) / TNT);
  const uint32_t fhi = (uint32_t)((F * (threadIdx.x + 1)) / TNT);
  const uint32_t nl = sm.nlight;
  uint32_t a = 0, b = nl;
  while (a < b) { const uint32_t m = (a + b) >> 1; if (sm.fpre[m] < flo) a = m + 1; else b = m; }
  jb = a;
  b = nl;
  while (a < b) { const uint32_t m = (a + b) >> 1; if (sm.fpre[m] < fhi) a = m + 1; else b = m; }
  je = a;
}

// number of CTAs that work on the heavy schedule (one item per warp)
__host__ __device__ inline unsigned heavy_blocks(uint64_t n_items) {
  return (unsigned)((n_items + (TNT / 32) - 1) / (TNT / 32));
}

// ===========================================================================
// PageRank
// ===========================================================================
template <int IDM, int OFF>
__global__ void __launch_bounds__(TNT) k_pr_init(GView g, PrArgs a) {
  __shared__ TileSmem sm;
  const uint64_t v0 = (uint64_t)blockIdx.x * TV;
  const int cnt = (int)min((uint64_t)TV, g.n - v0);
  tile_offsets<OFF>(g, v0, cnt, sm.xs, sm.ts);
  __syncthreads();
  for (int i = threadIdx.x; i < cnt; i += TNT) {
    uint64_t start; uint32_t d, w;
    vgeo<IDM>(g, sm.xs[i], sm.xs[i + 1], start, d, w);
    const uint64_t v = v0 + i;
    const float r0 = a.personal < 0 ? a.r0_all : ((int64_t)v == a.personal ? 1.0f : 0.0f);
    a.contrib_out[v] = d ? r0 / (float)d : 0.0f;
  }
}

__device__ __forceinline__ void pr_finish(const GView& g, const PrArgs& a, uint64_t v, uint32_t d, float sum) {
  const float base = a.personal < 0 ? a.base_all : ((int64_t)v == a.personal ? a.base_all : 0.0f);
  const float r = base + a.damp * sum;
  __stcs(a.contrib_out + v, d ? r / (float)d : 0.0f);  // streamed: read again only next iteration
  if (a.last) __stcs(a.ranks_out + (g.inv_perm ? (uint64_t)g.inv_perm[v] : v), r);
}

// One launch = one iteration.  Blocks [0, HB) take the heavy schedule (a warp
// per item); the other blocks take one tile of 512 vertices each.
template <int IDM, int OFF>
__global__ void __launch_bounds__(TNT, (IDM == ID_LOCAL || IDM == ID_CSR32) ? 5 : 6) k_pr_pull(GView g, PrArgs a) {
  __shared__ TileSmem sm;
  const float* __restrict__ c = a.contrib_in;
  const unsigned hb = heavy_blocks(g.n_items);
  const int lane = threadIdx.x & 31;
  const uint64_t pstream = policy_stream(), pkeep = policy_keep();
  if (blockIdx.x < hb) {
    const uint64_t it = (uint64_t)blockIdx.x * (TNT / 32) + (threadIdx.x >> 5);
    if (it >= g.n_items) return;
    const HeavyItem h = g.items[it];
    const uint32_t f1 = h.f0 + h.nf;
    uint32_t carry = h.carry;
    float acc = 0.f, comp = 0.f;
    for (uint32_t base = h.f0; base < f1; base += 32 * HEAVY_U) {
      uint32_t id[HEAVY_U];
      warp_ids<IDM, HEAVY_U>(g, h.bit, h.w, base, f1, carry, id);
      float x[HEAVY_U];
#pragma unroll
      for (int u = 0; u < HEAVY_U; u++) x[u] = (base + 32u * u + lane < f1) ? ldg_gather(c + id[u], id[u] < a.hot ? pkeep : pstream) : 0.f;
#pragma unroll
      for (int u = 0; u < HEAVY_U; u++) {  // compensated (Kahan) lane sums
        const float y = x[u] - comp;
        const float t = acc + y;
        comp = (t - acc) - y;
        acc = t;
      }
    }
    acc = warp_sum<float>(acc);
    if (lane == 0) {
      if (h.nitems == 1) pr_finish(g, a, h.v, h.deg, acc);
      else a.part[it] = acc;
    }
    return;
  }
  const uint64_t v0 = (uint64_t)(blockIdx.x - hb) * TV;
  const int cnt = (int)min((uint64_t)TV, g.n - v0);
  tile_offsets<OFF>(g, v0, cnt, sm.xs, sm.ts);
  __syncthreads();
  tile_classify<IDM>(g, sm, cnt, [](int) { return true; });

  // zero-degree vertices keep the teleport term only
  for (int i = threadIdx.x; i < cnt; i += TNT)
    if (sm.deg[i] == 0) pr_finish(g, a, v0 + i, 0, 0.0f);

  if (IDM == ID_LOCAL_GAP) {
    // gap-coded IDs cannot start mid-neighborhood: runs of whole vertices,
    // sequential decode, 4 gathers in flight
    uint32_t jb, je;
    light_range(sm, jb, je);
    for (uint32_t j = jb; j < je; j++) {
      const int i = sm.clist[j];
      const uint32_t d = sm.deg[i];
      SeqDec<IDM> dec;
      dec.init(g, sm.st[i], sm.wid[i], pstream);
      float s0 = 0.f, s1 = 0.f;
      uint32_t k = 0;
      for (; k + 4 <= d; k += 4) {
        const uint32_t u0 = dec.next(), u1 = dec.next(), u2 = dec.next(), u3 = dec.next();
        const float f0 = ldg_gather(c + u0, u0 < a.hot ? pkeep : pstream), f1 = ldg_gather(c + u1, u1 < a.hot ? pkeep : pstream);
        const float f2 = ldg_gather(c + u2, u2 < a.hot ? pkeep : pstream), f3 = ldg_gather(c + u3, u3 < a.hot ? pkeep : pstream);
        s0 += f0 + f1;
        s1 += f2 + f3;
      }
      for (; k < d; k++) {
        const uint32_t u = dec.next();
        s0 += ldg_gather(c + u, u < a.hot ? pkeep : pstream);
      }
      pr_finish(g, a, v0 + i, d, s0 + s1);
    }
    return;
  }
  // Fields-balanced light phase (as in k_ppr_pull): thread t decodes fields
  // [F*t/TNT, F*(t+1)/TNT) of the tile's light fields, entering its first
  // vertex mid-neighborhood if need be; per-vertex sums go to vsum, the
  // partial sum of a vertex entered mid-way to carry[t]; a uniform phase adds
  // them per vertex in thread order and finishes the vertex.
  __shared__ float vsum[TV];
  __shared__ float carry[TNT];
  float* ps = nullptr;
  const uint32_t F = sm.nfields, nl = sm.nlight;
  const uint32_t flo = (uint32_t)((uint64_t)F * threadIdx.x / TNT);
  const uint32_t fhi = (uint32_t)((uint64_t)F * (threadIdx.x + 1) / TNT);
  carry[threadIdx.x] = 0.f;
  if (flo < fhi) {
    uint32_t lo = 0, hi = nl - 1;  // the vertex holding field flo: last j with fpre[j] <= flo
    while (lo < hi) {
      const uint32_t m = (lo + hi + 1) >> 1;
      if (sm.fpre[m] <= flo) lo = m; else hi = m - 1;
    }
    uint32_t j = lo, f = flo;
    ps = sm.fpre[j] < flo ? &carry[threadIdx.x] : &vsum[j];
    while (f < fhi) {
      const int i = sm.clist[j];
      const uint32_t vend = min(sm.fpre[j + 1], fhi);
      const uint32_t fw = IDM == ID_GLOBAL ? g.r : (IDM == ID_CSR32 ? 32u : (uint32_t)sm.wid[i]);
      SeqDec<IDM> dec;
      dec.init(g, sm.st[i] + (uint64_t)(f - sm.fpre[j]) * fw, sm.wid[i], pstream);
      const uint32_t d = vend - f;
      float s0 = 0.f, s1 = 0.f;
      uint32_t k = 0;
      for (; k + 4 <= d; k += 4) {  // four gathers in flight
        const uint32_t u0 = dec.next(), u1 = dec.next(), u2 = dec.next(), u3 = dec.next();
        const float f0 = ldg_gather(c + u0, u0 < a.hot ? pkeep : pstream), f1 = ldg_gather(c + u1, u1 < a.hot ? pkeep : pstream);
        const float f2 = ldg_gather(c + u2, u2 < a.hot ? pkeep : pstream), f3 = ldg_gather(c + u3, u3 < a.hot ? pkeep : pstream);
        s0 += f0 + f1;
        s1 += f2 + f3;
      }
      for (; k < d; k++) {
        const uint32_t u = dec.next();
        s0 += ldg_gather(c + u, u < a.hot ? pkeep : pstream);
      }
      *ps = s0 + s1;
      f = vend;
      j++;
      ps = &vsum[j];
    }
  }
  __syncthreads();
  for (uint32_t j = threadIdx.x; j < nl; j += TNT) {
    const uint32_t fs = sm.fpre[j], fe = sm.fpre[j + 1];
    float sum = vsum[j];
    uint32_t q = (uint32_t)((uint64_t)fs * TNT / (F ? F : 1));  // the thread holding the first field
    while (q + 1 < TNT && (uint32_t)((uint64_t)F * (q + 1) / TNT) <= fs) q++;
    while (q > 0 && (uint32_t)((uint64_t)F * q / TNT) > fs) q--;
    for (q = q + 1; q < TNT && (uint32_t)((uint64_t)F * q / TNT) < fe; q++) sum += carry[q];
    const int i = sm.clist[j];
    pr_finish(g, a, v0 + i, sm.deg[i], sum);
  }
}

// ===========================================================================
// Personalized PageRank, PPR_K requests per sweep (serving engine).  Slot k
// iterates r_t[v] = (1-d_k)[v == s_k] + d_k * sum_{u in N_v} r_{t-1}[u] / d_u;
// the same tile / heavy-item structure as k_pr_pull, with PPR_K sums per
// vertex and one 32-byte gather per arc for all slots.
// ===========================================================================
__device__ __forceinline__ void ppr_finish(const PprArgs& a, uint64_t v, uint32_t d, const float (&sum)[PPR_K]) {
  float out[PPR_K];
#pragma unroll
  for (int k = 0; k < PPR_K; k++) {
    const bool act = (a.active >> k) & 1u;
    const float r = ((uint64_t)a.src[k] == v ? 1.0f - a.damp[k] : 0.0f) + a.damp[k] * sum[k];
    out[k] = (act && d) ? r / (float)d : 0.0f;
    if (act && ((a.last >> k) & 1u)) a.result[k][a.result_perm ? (uint64_t)a.result_perm[v] : v] = r;
  }
  float4* o = reinterpret_cast<float4*>(a.cout + v * PPR_K);
  __stcs(o, make_float4(out[0], out[1], out[2], out[3]));
  __stcs(o + 1, make_float4(out[4], out[5], out[6], out[7]));
}

// half h of the slots (4 of them) for vertex v, written by one lane of a pair
__device__ __forceinline__ void ppr_finish_half(const PprArgs& a, uint64_t v, uint32_t d, const float4& sum, int h) {
  const float sv[4] = {sum.x, sum.y, sum.z, sum.w};
  float out[4];
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const int k = h * 4 + q;
    const bool act = (a.active >> k) & 1u;
    const float r = ((uint64_t)a.src[k] == v ? 1.0f - a.damp[k] : 0.0f) + a.damp[k] * sv[q];
    out[q] = (act && d) ? r / (float)d : 0.0f;
    if (act && ((a.last >> k) & 1u)) a.result[k][a.result_perm ? (uint64_t)a.result_perm[v] : v] = r;
  }
  __stcs(reinterpret_cast<float4*>(a.cout + v * PPR_K + h * 4), make_float4(out[0], out[1], out[2], out[3]));
}

// one 16-byte half row of slot contributions; rows of the first `hot`
// vertices (the hubs, after DM relabeling) stay in L2, the rest stream through
__device__ __forceinline__ float4 gather_row(const float* ch, uint32_t u, uint32_t hot, uint64_t keep, uint64_t stream) {
  return ldg_gather4(ch + (uint64_t)u * PPR_K, u < hot ? keep : stream);
}

__device__ __forceinline__ void add4(float4& s, const float4& x) {
  s.x += x.x; s.y += x.y; s.z += x.z; s.w += x.w;
}

// range of compacted light vertices owned by lane pair `p` of `np` pairs
__device__ __forceinline__ void light_range_of(const TileSmem& sm, uint32_t p, uint32_t np, uint32_t& jb,
                                               uint32_t& je) {
  const uint64_t F = sm.nfields;
  const uint32_t flo = (uint32_t)((F * p) / np);
  const uint32_t fhi = (uint32_t)((F * (p + 1)) / np);
  const uint32_t nl = sm.nlight;
  uint32_t lo = 0, hi = nl;
  while (lo < hi) { const uint32_t m = (lo + hi) >> 1; if (sm.fpre[m] < flo) lo = m + 1; else hi = m; }
  jb = lo;
  hi = nl;
  while (lo < hi) { const uint32_t m = (lo + hi) >> 1; if (sm.fpre[m] < fhi) lo = m + 1; else hi = m; }
  je = lo;
}

// Light vertices are decoded by lane PAIRS: both lanes of a pair walk the
// same run of neighborhoods, lane h gathering the 16-byte half h of each
// neighbor's 32-byte slot row, so a pair's two loads of one arc coalesce into
// one sector and every thread keeps four arcs in flight.
template <int IDM, int OFF>
__global__ void __launch_bounds__(TNT, 4) k_ppr_pull(GView g, PprArgs a) {
  __shared__ TileSmem sm;
  const float* __restrict__ c = a.cin;
  const unsigned hb = heavy_blocks(g.n_items);
  const int lane = threadIdx.x & 31;
  const uint64_t pstream = policy_stream(), pkeep = policy_keep();
  if (blockIdx.x < hb) {
    // heavy item: lane pairs again -- the pair (2i, 2i+1) gathers both halves
    // of field i of each 16-field round; Kahan-compensated lane sums
    const uint64_t it = (uint64_t)blockIdx.x * (TNT / 32) + (threadIdx.x >> 5);
    if (it >= g.n_items) return;
    const HeavyItem hv = g.items[it];
    const uint32_t f1 = hv.f0 + hv.nf;
    const int h = lane & 1;
    const float* ch = c + h * 4;
    uint32_t carry = hv.carry;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f), comp = acc;
    for (uint32_t base = hv.f0; base < f1; base += 64) {
      uint32_t id[2];
      warp_ids<IDM, 2>(g, hv.bit, hv.w, base, f1, carry, id);
      float4 x[4];
#pragma unroll
      for (int u = 0; u < 2; u++) {
#pragma unroll
        for (int r = 0; r < 2; r++) {
          const uint32_t from = (uint32_t)(r * 16 + (lane >> 1));
          const uint32_t fid = __shfl_sync(LG_FULL_MASK, id[u], from);
          x[u * 2 + r] = (base + 32u * u + from < f1) ? gather_row(ch, fid, a.hot, pkeep, pstream)
                                                      : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
#pragma unroll
      for (int q = 0; q < 4; q++) {
        float* ap = &acc.x;
        float* cp = &comp.x;
        const float* xp = &x[q].x;
#pragma unroll
        for (int e = 0; e < 4; e++) {
          const float y = xp[e] - cp[e];
          const float t = ap[e] + y;
          cp[e] = (t - ap[e]) - y;
          ap[e] = t;
        }
      }
    }
    // sum the 16 lanes of each parity (offsets 16, 8, 4, 2 keep the parity)
#pragma unroll
    for (int o = 16; o >= 2; o >>= 1) {
      acc.x += __shfl_xor_sync(LG_FULL_MASK, acc.x, o);
      acc.y += __shfl_xor_sync(LG_FULL_MASK, acc.y, o);
      acc.z += __shfl_xor_sync(LG_FULL_MASK, acc.z, o);
      acc.w += __shfl_xor_sync(LG_FULL_MASK, acc.w, o);
    }
    if (lane < 2) {
      if (hv.nitems == 1) {
        ppr_finish_half(a, hv.v, hv.deg, acc, h);
      } else {
        float* pp = a.part + it * PPR_K + h * 4;
        pp[0] = acc.x; pp[1] = acc.y; pp[2] = acc.z; pp[3] = acc.w;
      }
    }
    return;
  }
  const uint64_t v0 = (uint64_t)(blockIdx.x - hb) * TV;
  const int cnt = (int)min((uint64_t)TV, g.n - v0);
  tile_offsets<OFF>(g, v0, cnt, sm.xs, sm.ts);
  __syncthreads();
  tile_classify<IDM>(g, sm, cnt, [](int) { return true; });
  const float zero[PPR_K] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int i = threadIdx.x; i < cnt; i += TNT)
    if (sm.deg[i] == 0) ppr_finish(a, v0 + i, 0, zero);
  const int h = threadIdx.x & 1;
  const float* ch = c + h * 4;
  if (IDM == ID_LOCAL_GAP) {
    // gap-coded IDs cannot start mid-neighborhood: runs of whole vertices
    uint32_t jb, je;
    light_range_of(sm, threadIdx.x >> 1, TNT / 2, jb, je);
    for (uint32_t j = jb; j < je; j++) {
      const int i = sm.clist[j];
      const uint32_t d = sm.deg[i];
      SeqDec<IDM> dec;
      dec.init(g, sm.st[i], sm.wid[i], pstream);
      float4 s0 = make_float4(0.f, 0.f, 0.f, 0.f), s1 = s0;
      uint32_t k = 0;
      for (; k + 4 <= d; k += 4) {
        const uint32_t u0 = dec.next(), u1 = dec.next(), u2 = dec.next(), u3 = dec.next();
        const float4 x0 = ldg_gather4(ch + (uint64_t)u0 * PPR_K, u0 < a.hot ? pkeep : pstream);
        const float4 x1 = ldg_gather4(ch + (uint64_t)u1 * PPR_K, u1 < a.hot ? pkeep : pstream);
        const float4 x2 = ldg_gather4(ch + (uint64_t)u2 * PPR_K, u2 < a.hot ? pkeep : pstream);
        const float4 x3 = ldg_gather4(ch + (uint64_t)u3 * PPR_K, u3 < a.hot ? pkeep : pstream);
        add4(s0, x0); add4(s1, x1); add4(s0, x2); add4(s1, x3);
      }
      for (; k < d; k++) add4(s0, gather_row(ch, dec.next(), a.hot, pkeep, pstream));
      add4(s0, s1);
      ppr_finish_half(a, v0 + i, d, s0, h);
    }
    return;
  }
  // Fields-balanced light phase: pair w takes fields [F*w/NW, F*(w+1)/NW) of
  // the tile's compacted light fields, starting mid-neighborhood if need be.
  // A vertex's sum over the range that contains its first field goes to
  // vsum[j]; a pair that entered its first vertex mid-way leaves that partial
  // in carry[w].  A uniform phase then adds, per vertex, vsum and the carries
  // of the following pairs in pair order (deterministic) and finishes it.
  __shared__ float4 vsum[TV][2];
  __shared__ float4 carry[TNT / 2][2];
  constexpr uint32_t NW = TNT / 2;
  const uint32_t w = threadIdx.x >> 1;
  const uint32_t F = sm.nfields, nl = sm.nlight;
  const uint32_t flo = (uint32_t)((uint64_t)F * w / NW), fhi = (uint32_t)((uint64_t)F * (w + 1) / NW);
  carry[w][h] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (flo < fhi) {
    uint32_t lo = 0, hi = nl - 1;  // the vertex holding field flo: last j with fpre[j] <= flo
    while (lo < hi) {
      const uint32_t m = (lo + hi + 1) >> 1;
      if (sm.fpre[m] <= flo) lo = m; else hi = m - 1;
    }
    uint32_t j = lo, f = flo;
    bool head = sm.fpre[j] < flo;
    while (f < fhi) {
      const int i = sm.clist[j];
      const uint32_t vend = min(sm.fpre[j + 1], fhi);
      const uint32_t off = f - sm.fpre[j];
      const uint32_t fw = IDM == ID_GLOBAL ? g.r : (IDM == ID_CSR32 ? 32u : (uint32_t)sm.wid[i]);
      SeqDec<IDM> dec;
      dec.init(g, sm.st[i] + (uint64_t)off * fw, sm.wid[i], pstream);
      float4 s0 = make_float4(0.f, 0.f, 0.f, 0.f), s1 = s0;
      const uint32_t d = vend - f;
      uint32_t k = 0;
      for (; k + 4 <= d; k += 4) {  // four arcs in flight
        const uint32_t u0 = dec.next(), u1 = dec.next(), u2 = dec.next(), u3 = dec.next();
        const float4 x0 = ldg_gather4(ch + (uint64_t)u0 * PPR_K, u0 < a.hot ? pkeep : pstream);
        const float4 x1 = ldg_gather4(ch + (uint64_t)u1 * PPR_K, u1 < a.hot ? pkeep : pstream);
        const float4 x2 = ldg_gather4(ch + (uint64_t)u2 * PPR_K, u2 < a.hot ? pkeep : pstream);
        const float4 x3 = ldg_gather4(ch + (uint64_t)u3 * PPR_K, u3 < a.hot ? pkeep : pstream);
        add4(s0, x0); add4(s1, x1); add4(s0, x2); add4(s1, x3);
      }
      for (; k < d; k++) add4(s0, gather_row(ch, dec.next(), a.hot, pkeep, pstream));
      add4(s0, s1);
      if (head) carry[w][h] = s0;
      else vsum[j][h] = s0;
      head = false;
      f = vend;
      j++;
    }
  }
  __syncthreads();
  for (uint32_t t = threadIdx.x; t < nl * 2; t += TNT) {
    const uint32_t j = t >> 1;
    const int hh = (int)(t & 1);
    const uint32_t fs = sm.fpre[j], fe = sm.fpre[j + 1];
    float4 sum = vsum[j][hh];
    // pairs after the owner whose ranges start inside this vertex
    uint32_t q = (uint32_t)((uint64_t)fs * NW / (F ? F : 1));
    while (q + 1 < NW && (uint32_t)((uint64_t)F * (q + 1) / NW) <= fs) q++;
    while (q > 0 && (uint32_t)((uint64_t)F * q / NW) > fs) q--;
    for (q = q + 1; q < NW && (uint32_t)((uint64_t)F * q / NW) < fe; q++) add4(sum, carry[q][hh]);
    const int i = sm.clist[j];
    ppr_finish_half(a, v0 + i, sm.deg[i], sum, hh);
  }
}

// a slot joins: its column of `cin` is all zero (the slot was idle for a
// whole sweep, or the array is fresh); r_0 = e_src gives cin[src] = 1 / d_src
template <int IDM, int OFF>
__global__ void __launch_bounds__(32) k_ppr_join(GView g, float* cin, uint32_t slot, uint32_t src) {
  uint64_t x0, x1, start;
  uint32_t d, w;
  offset_pair<OFF>(g, src, x0, x1);
  vgeo<IDM>(g, x0, x1, start, d, w);
  if (threadIdx.x == 0) cin[(uint64_t)src * PPR_K + slot] = d ? 1.0f / (float)d : 0.0f;
}

// ===========================================================================
// BFS (multi-source, bit-parallel): bit s of a mask is source s
// ===========================================================================
template <typename M>
__device__ __forceinline__ void bfs_finish(const GView& g, const BfsArgs& a, uint64_t v, M need, M found,
                                           uint32_t* qbuf, uint32_t* qn, uint32_t* pairs) {
  M* vis = reinterpret_cast<M*>(a.vis);
  M* fout = reinterpret_cast<M*>(a.front_out);
  const M nb = (M)(found & need);
  fout[v] = nb;
  if (nb) {
    vis[v] = (M)(vis[v] | nb);
    write_depths<M>(a, g.n, v, nb, a.level + 1);
    if (qbuf) {
      qbuf[atomicAdd(qn, 1u)] = (uint32_t)v;
      atomicAdd(pairs, (uint32_t)__popcll((unsigned long long)nb));
    } else {
      a.queue_out[atomicAdd(&a.counters[0], 1u)] = (uint32_t)v;
      atomicAdd(&a.counters[1], (uint32_t)__popcll((unsigned long long)nb));
    }
  }
}

template <int IDM, int OFF, typename M>
__global__ void __launch_bounds__(TNT, IDM == ID_LOCAL_GAP ? 6 : 5) k_bfs_pull(GView g, BfsArgs a) {
  __shared__ TileSmem sm;
  __shared__ M need_sm[TV];
  __shared__ uint32_t qbuf[TV];
  __shared__ uint32_t qn, newpairs, qbase;
  const M* vis = reinterpret_cast<const M*>(a.vis);
  const M* __restrict__ fin = reinterpret_cast<const M*>(a.front_in);
  M* fout = reinterpret_cast<M*>(a.front_out);
  const M all = (M)a.all_mask;
  const unsigned hb = heavy_blocks(g.n_items);
  const int lane = threadIdx.x & 31;
  const uint64_t pstream = policy_stream(), pkeep = policy_keep();
  if (blockIdx.x < hb) {
    const uint64_t it = (uint64_t)blockIdx.x * (TNT / 32) + (threadIdx.x >> 5);
    if (it >= g.n_items) return;
    const HeavyItem h = g.items[it];
    const M need = (M)(all & (M)~vis[h.v]);
    if (need == 0) {
      if (h.nitems == 1 && lane == 0) fout[h.v] = 0;
      return;
    }
    const uint32_t f1 = h.f0 + h.nf;
    uint32_t carry = h.carry;
    M acc = 0;
    for (uint32_t base = h.f0; base < f1; base += 32 * HEAVY_U) {
      uint32_t id[HEAVY_U];
      warp_ids<IDM, HEAVY_U>(g, h.bit, h.w, base, f1, carry, id);
      M x[HEAVY_U];
#pragma unroll
      for (int u = 0; u < HEAVY_U; u++) x[u] = (base + 32u * u + lane < f1) ? ldg_gather(fin + id[u], id[u] < a.hot ? pkeep : pstream) : (M)0;
#pragma unroll
      for (int u = 0; u < HEAVY_U; u++) acc |= x[u];
      acc = warp_or<M>(acc);
      if ((M)(acc & need) == need) break;
    }
    if (lane == 0) {
      if (h.nitems == 1) bfs_finish<M>(g, a, h.v, need, acc, nullptr, nullptr, nullptr);
      else atomic_or_mask<M>(reinterpret_cast<M*>(a.hacc) + h.slot, acc);
    }
    return;
  }
  if (threadIdx.x == 0) { qn = 0; newpairs = 0; }
  const uint64_t v0 = (uint64_t)(blockIdx.x - hb) * TV;
  const int cnt = (int)min((uint64_t)TV, g.n - v0);
  for (int i = threadIdx.x; i < cnt; i += TNT) need_sm[i] = (M)(all & (M)~vis[v0 + i]);
  tile_offsets<OFF>(g, v0, cnt, sm.xs, sm.ts);
  __syncthreads();
  tile_classify<IDM>(g, sm, cnt, [&](int i) { return need_sm[i] != 0; });

  for (int i = threadIdx.x; i < cnt; i += TNT)
    if (sm.deg[i] == 0 || (sm.deg[i] <= g.heavy_min && need_sm[i] == 0)) fout[v0 + i] = 0;

  if (IDM == ID_LOCAL_GAP) {
    // gap-coded IDs: runs of whole vertices (no mid-neighborhood start)
    uint32_t jb, je;
    light_range(sm, jb, je);
    for (uint32_t j = jb; j < je; j++) {
      const int i = sm.clist[j];
      const uint32_t d = sm.deg[i];
      const M need = need_sm[i];
      SeqDec<IDM> dec;
      dec.init(g, sm.st[i], sm.wid[i], pstream);
      M acc = 0;
      uint32_t k = 0;
      for (; k + 4 <= d; k += 4) {  // early exit once every unvisited source is found
        const uint32_t u0 = dec.next(), u1 = dec.next(), u2 = dec.next(), u3 = dec.next();
        acc |= (M)(ldg_gather(fin + u0, u0 < a.hot ? pkeep : pstream) | ldg_gather(fin + u1, u1 < a.hot ? pkeep : pstream) | ldg_gather(fin + u2, u2 < a.hot ? pkeep : pstream) |
                   ldg_gather(fin + u3, u3 < a.hot ? pkeep : pstream));
        if ((M)(acc & need) == need) break;
      }
      if ((M)(acc & need) != need)
        for (; k < d; k++) {
          const uint32_t u = dec.next();
          acc |= ldg_gather(fin + u, u < a.hot ? pkeep : pstream);
        }
      bfs_finish<M>(g, a, v0 + i, need, acc, qbuf, &qn, &newpairs);
    }
  } else {
    // fields-balanced (as in k_pr_pull): partial ORs of a vertex split over
    // threads are combined exactly in a uniform phase
    __shared__ M vor[TV];
    __shared__ M carry[TNT];
    const uint32_t F = sm.nfields, nl = sm.nlight;
    const uint32_t flo = (uint32_t)((uint64_t)F * threadIdx.x / TNT);
    const uint32_t fhi = (uint32_t)((uint64_t)F * (threadIdx.x + 1) / TNT);
    carry[threadIdx.x] = 0;
    if (flo < fhi) {
      uint32_t lo = 0, hi = nl - 1;
      while (lo < hi) {
        const uint32_t m = (lo + hi + 1) >> 1;
        if (sm.fpre[m] <= flo) lo = m; else hi = m - 1;
      }
      uint32_t j = lo, f = flo;
      M* ps = sm.fpre[j] < flo ? &carry[threadIdx.x] : &vor[j];
      while (f < fhi) {
        const int i = sm.clist[j];
        const M need = need_sm[i];
        const uint32_t vend = min(sm.fpre[j + 1], fhi);
        const uint32_t fw = IDM == ID_GLOBAL ? g.r : (IDM == ID_CSR32 ? 32u : (uint32_t)sm.wid[i]);
        SeqDec<IDM> dec;
        dec.init(g, sm.st[i] + (uint64_t)(f - sm.fpre[j]) * fw, sm.wid[i], pstream);
        const uint32_t d = vend - f;
        M acc = 0;
        uint32_t k = 0;
        for (; k + 4 <= d; k += 4) {
          const uint32_t u0 = dec.next(), u1 = dec.next(), u2 = dec.next(), u3 = dec.next();
          acc |= (M)(ldg_gather(fin + u0, u0 < a.hot ? pkeep : pstream) | ldg_gather(fin + u1, u1 < a.hot ? pkeep : pstream) | ldg_gather(fin + u2, u2 < a.hot ? pkeep : pstream) |
                     ldg_gather(fin + u3, u3 < a.hot ? pkeep : pstream));
          if ((M)(acc & need) == need) break;
        }
        if ((M)(acc & need) != need)
          for (; k < d; k++) {
          const uint32_t u = dec.next();
          acc |= ldg_gather(fin + u, u < a.hot ? pkeep : pstream);
        }
        *ps = acc;
        f = vend;
        j++;
        ps = &vor[j];
      }
    }
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < nl; j += TNT) {
      const uint32_t fs = sm.fpre[j], fe = sm.fpre[j + 1];
      M acc = vor[j];
      uint32_t q = (uint32_t)((uint64_t)fs * TNT / (F ? F : 1));
      while (q + 1 < TNT && (uint32_t)((uint64_t)F * (q + 1) / TNT) <= fs) q++;
      while (q > 0 && (uint32_t)((uint64_t)F * q / TNT) > fs) q--;
      for (q = q + 1; q < TNT && (uint32_t)((uint64_t)F * q / TNT) < fe; q++) acc |= carry[q];
      const int i = sm.clist[j];
      bfs_finish<M>(g, a, v0 + i, need_sm[i], acc, qbuf, &qn, &newpairs);
    }
  }

  __syncthreads();
  if (threadIdx.x == 0 && qn) {
    qbase = atomicAdd(&a.counters[0], qn);
    atomicAdd(&a.counters[1], newpairs);
  }
  __syncthreads();
  for (uint32_t t = threadIdx.x; t < qn; t += TNT) a.queue_out[qbase + t] = qbuf[t];
}

// top-down step over fields [f0, f1) of a frontier vertex with source mask m:
// every neighbor not yet visited by some of m's sources joins the next
// frontier for them (a warp, 32 * HEAVY_U fields per step)
template <int IDM, typename M>
__device__ __forceinline__ void push_fields(const GView& g, const BfsArgs& a, M m, uint64_t start, uint32_t w,
                                            uint32_t f0, uint32_t f1, uint32_t carry, uint32_t& pairs) {
  M* vis = reinterpret_cast<M*>(a.vis);
  M* fout = reinterpret_cast<M*>(a.front_out);
  const int lane = threadIdx.x & 31;
  const uint32_t nd = a.level + 1;
  for (uint32_t base = f0; base < f1; base += 32 * HEAVY_U) {
    uint32_t id[HEAVY_U];
    warp_ids<IDM, HEAVY_U>(g, start, w, base, f1, carry, id);
    M cur[HEAVY_U];
#pragma unroll
    for (int u = 0; u < HEAVY_U; u++) cur[u] = (base + 32u * u + lane < f1) ? vis[id[u]] : (M)~(M)0;
#pragma unroll
    for (int u = 0; u < HEAVY_U; u++) {
      const uint32_t u_id = id[u];
      bool app = false;
      M nb = (M)(m & (M)~cur[u]);
      if (nb) {
        const M old = atomic_or_mask<M>(vis + u_id, nb);
        nb = (M)(nb & (M)~old);
        if (nb) {
          const M oldf = atomic_or_mask<M>(fout + u_id, nb);
          app = (oldf == 0);
          write_depths<M>(a, g.n, u_id, nb, nd);
          pairs += __popcll((unsigned long long)nb);
        }
      }
      const uint32_t bal = __ballot_sync(LG_FULL_MASK, app);
      if (bal) {
        uint32_t basepos = 0;
        if (lane == 0) basepos = atomicAdd(&a.counters[0], (uint32_t)__popc(bal));
        basepos = __shfl_sync(LG_FULL_MASK, basepos, 0);
        if (app) a.queue_out[basepos + __popc(bal & lane_lt_mask())] = u_id;
      }
    }
  }
}

// Top-down step.  Blocks [0, hb) take the heavy-vertex schedule, a warp per
// item, working when the item's vertex is in the frontier (a hub's arcs are
// spread over as many warps as it has items); the other blocks take the
// frontier queue, a warp per vertex of degree <= heavy_min.
template <int IDM, int OFF, typename M>
__global__ void __launch_bounds__(256) k_bfs_push(GView g, BfsArgs a, unsigned hb) {
  const M* __restrict__ fin = reinterpret_cast<const M*>(a.front_in);
  const int lane = threadIdx.x & 31;
  uint32_t pairs = 0;
  if (blockIdx.x < hb) {
    const uint64_t it = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (it < g.n_items) {
      const HeavyItem h = g.items[it];
      const M m = fin[h.v];
      if (m) push_fields<IDM, M>(g, a, m, h.bit, h.w, h.f0, h.f0 + h.nf, h.carry, pairs);
    }
  } else {
    const uint64_t warps = (uint64_t)(gridDim.x - hb) * (blockDim.x >> 5);
    for (uint64_t q = (uint64_t)(blockIdx.x - hb) * (blockDim.x >> 5) + (threadIdx.x >> 5); q < a.queue_in_len;
         q += warps) {
      const uint32_t v = a.queue_in[q];
      const M m = fin[v];
      uint64_t x0, x1, start;
      uint32_t d, w;
      offset_pair<OFF>(g, v, x0, x1);
      vgeo<IDM>(g, x0, x1, start, d, w);
      if (d > g.heavy_min && g.n_items) continue;  // in the heavy schedule
      push_fields<IDM, M>(g, a, m, start, w, 0, d, 0, pairs);
    }
  }
  pairs = warp_sum<uint32_t>(pairs);
  if (lane == 0 && pairs) atomicAdd(&a.counters[1], pairs);
}

// ===========================================================================
// neighbor queries (getNeighbors of Listing 3): one warp per query
// ===========================================================================
template <int IDM, int OFF>
__global__ void __launch_bounds__(256) k_nbr_degrees(GView g, NbrArgs a) {
  const int lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t q = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < a.k; q += warps) {
    const uint32_t vo = a.vertices[q];
    if (vo >= g.n) {
      if (lane == 0) { set_err(a.err, DERR_QUERY); a.out_offsets[q] = 0; }
      continue;
    }
    const uint64_t v = g.perm ? (uint64_t)g.perm[vo] : vo;
    uint64_t x0, x1, start;
    uint32_t d, w;
    offset_pair<OFF>(g, v, x0, x1);
    vgeo<IDM>(g, x0, x1, start, d, w);
    if (lane == 0) a.out_offsets[q] = d;
  }
}

template <int IDM, int OFF>
__global__ void __launch_bounds__(256) k_nbr_decode(GView g, NbrArgs a) {
  const int lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t q = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < a.k; q += warps) {
    const uint32_t vo = a.vertices[q];
    if (vo >= g.n) continue;
    const uint64_t v = g.perm ? (uint64_t)g.perm[vo] : vo;
    uint64_t x0, x1, start;
    uint32_t d, w;
    offset_pair<OFF>(g, v, x0, x1);
    vgeo<IDM>(g, x0, x1, start, d, w);
    const uint64_t o = a.out_offsets[q];
    uint32_t carry = 0;
    for (uint32_t base = 0; base < d; base += 64) {
      uint32_t id[2];
      warp_ids<IDM, 2>(g, start, w, base, d, carry, id);
#pragma unroll
      for (int u = 0; u < 2; u++) {
        const uint32_t idx = base + 32u * u + lane;
        if (idx < d) {
          a.out_ids[o + idx] = g.inv_perm ? g.inv_perm[id[u]] : id[u];
          if (a.out_weights) {
            uint32_t wt = 0;
            if (IDM == ID_GLOBAL && g.omega) wt = weight_at(g, start, idx);
            if (IDM == ID_CSR32 && g.W32) wt = __ldg(g.W32 + (start >> 5) + idx);
            a.out_weights[o + idx] = wt;
          }
        }
      }
    }
  }
}

// ===========================================================================
// Whole-graph decode (lg_decode): every neighborhood (Section 3.7.2's access
// applied to all vertices) written to a CSR in stored order.
//
// Global IDs (and CSR-32) keep their records in arc order, so record j is
// col[j] and the offsets x_v are the row offsets: one launch writes row_ptr
// from the offsets (a tile decode per 512 vertices) and maps records to IDs,
// consecutive threads on consecutive records (coalesced stream reads and
// coalesced writes, no vertex lookup).  Local IDs: one
// kernel, described above k_dec_local.
//
// Local IDs: a degree pass and a scan give the row offsets, then tiles of TV
// vertices decode their offsets once and split the tile's light fields into
// rounds of DEC_C fields.  In a round every thread decodes a contiguous run of
// fields sequentially (bit reader, one shift and mask per field, a running sum
// for gaps), entering its first neighborhood mid-way if need be, into a
// shared-memory stage; the stage is then written out coalesced.  A run that
// starts inside a gap-coded neighborhood sums its gaps from 0; a segmented
// scan over the threads' last values (absolute once the neighborhood's first
// field has been read) supplies the missing prefix.  Heavy vertices come from
// the heavy schedule, a warp per item, a lane per field.
// ===========================================================================
template <int IDM, int U>
__device__ __forceinline__ void dec_fields(const GView& g, const DecArgs& a, uint64_t start, uint32_t w, uint32_t f0,
                                           uint32_t f1, uint32_t carry, uint64_t o) {
  const uint32_t lane = threadIdx.x & 31u;
  for (uint32_t base = f0; base < f1; base += 32u * U) {
    uint32_t id[U];
    warp_ids<IDM, U>(g, start, w, base, f1, carry, id);
#pragma unroll
    for (int u = 0; u < U; u++) {
      const uint32_t idx = base + 32u * u + lane;
      if (idx < f1) __stcs(a.ids + o + idx, id[u]);
    }
  }
}

constexpr uint32_t DEC_FLAT_CH = 512;                      // records per warp chunk (flat decode)
constexpr uint32_t DEC_FLAT_WORDS = DEC_FLAT_CH * 64 / 32 + 4;  // stream words of a chunk of <= 64-bit records

// Flat decode of global-ID records (or CSR-32 IDs), one launch, one block per
// tile of TV vertices: the block writes the tile's row_ptr entries from the
// offsets, then decodes its share of the records (arcs / tiles, rounded up to
// whole chunks) chunk by chunk, a warp per chunk of DEC_FLAT_CH records: the
// chunk's stream words come into shared memory with 16-byte loads (a chunk
// starts on a 16-byte boundary: DEC_FLAT_CH * r bits is a multiple of 128),
// then lane l extracts records l, l + 32, ... with a funnel shift and writes
// them coalesced.
template <int IDM, int OFF>
__global__ void __launch_bounds__(256) k_dec_flat(GView g, DecArgs a, uint64_t per_block) {
  __shared__ __align__(16) uint32_t fw[TNT / 32][DEC_FLAT_WORDS];
  {
    __shared__ uint64_t xs[TV + 1];
    __shared__ TileScratch ts;
    const uint64_t v0 = (uint64_t)blockIdx.x * TV;
    const int cnt = (int)min((uint64_t)TV, g.n - v0);
    tile_offsets<OFF>(g, v0, cnt, xs, ts);
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += TNT) a.row_out[v0 + i] = xs[i];
    if (v0 + (uint64_t)cnt == g.n && threadIdx.x == 0) a.row_out[g.n] = xs[cnt];
  }
  const uint64_t arcs = g.arcs;
  const uint64_t jb = (uint64_t)blockIdx.x * per_block, je = min(arcs, jb + per_block);
  const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
  const bool want_w = a.weights != nullptr;
  if constexpr (IDM == ID_CSR32) {
    for (uint64_t j = jb + threadIdx.x; j < je; j += TNT) {
      __stcs(a.ids + j, __ldcs(g.A32 + j));
      if (want_w) __stcs(a.weights + j, g.W32 ? __ldcs(g.W32 + j) : 0u);
    }
  } else {
    const uint32_t r = g.r, s = g.s;
    const uint32_t ms = mask_lo(s), mw = mask_lo(g.omega);
    uint32_t* sw = fw[wid];
    for (uint64_t c = jb + (uint64_t)wid * DEC_FLAT_CH; c < je; c += (uint64_t)(TNT / 32) * DEC_FLAT_CH) {
      const uint32_t nrec = (uint32_t)min((uint64_t)DEC_FLAT_CH, je - c);
      const uint64_t w0 = c * r / 32;  // a multiple of 4: c is a multiple of DEC_FLAT_CH
      const uint32_t nw = (nrec * r + 31) / 32 + 1;  // the chunk's words and the one after
      const uint4* src = reinterpret_cast<const uint4*>(g.A32 + w0);
      for (uint32_t q = lane; q * 4 < nw; q += 32) reinterpret_cast<uint4*>(sw)[q] = __ldcs(src + q);
      __syncwarp();
      for (uint32_t t = lane; t < nrec; t += 32) {
        const uint32_t p = t * r;
        const uint32_t x0 = sw[p >> 5], x1 = sw[(p >> 5) + 1];
        __stcs(a.ids + c + t, __funnelshift_r(x0, x1, p & 31u) & ms);
        if (want_w) {
          uint32_t wt = 0;
          if (g.omega) {
            const uint32_t q = p + s;
            wt = __funnelshift_r(sw[q >> 5], sw[(q >> 5) + 1], q & 31u) & mw;
          }
          __stcs(a.weights + c + t, wt);
        }
      }
      __syncwarp();
    }
  }
}

// ---------------------------------------------------------------------------
// Local-ID decode: one launch writes row_ptr and every row.
//
// Blocks take a ticket when they start: tickets below the tile count are tile
// CTAs (tiles in start order), the rest are heavy-schedule CTAs.  A tile CTA
// decodes its offsets and geometry, publishes its arc count, and finds the
// arcs of all earlier tiles by a decoupled look-back over their published
// counts (a tile waits only on tiles that started before it).  It writes its
// row offsets, flags them ready (heavy items read their row start there), and
// then decodes its light vertices window by window: a window is up to DEC_C
// light fields of one run of light vertices with no heavy vertex between them,
// so its stream bits are contiguous; they are staged in shared memory with
// 16-byte loads, every thread decodes DEC_C / TNT consecutive fields from
// there (a shift and a mask per field, a running sum for gaps), a segmented
// scan over the threads supplies the prefix of gap runs entered mid-way, and
// the window is written out coalesced.
// ---------------------------------------------------------------------------
constexpr int DEC_P = 9;                   // light fields per lane and window (odd: the lanes' stage
                                           // stores fall in distinct banks)
constexpr int DEC_WF = 32 * DEC_P;         // light fields per warp window
constexpr int DEC_WCAP = 400;              // stream words a warp window may stage (longer windows shrink)
constexpr uint64_t DEC_AGG = 1ull << 62, DEC_INCL = 2ull << 62, DEC_VAL = (1ull << 62) - 1;

struct DecWarp {
  __align__(16) uint32_t words[DEC_WCAP + 8];  // stream words of the warp's current window
  uint32_t stage[DEC_WF];                      // decoded IDs of the warp's current window
};

struct DecSmem {
  TileSmem t;                  // offsets (xs, reused for the all-degree prefix), geometry, light list
  DecWarp w[TNT / 32];
  uint64_t rdelta[TV];         // per run of light vertices: output index - light field index
  uint16_t rfirst[TV + 1];     // per run: its first light index
  uint64_t base;               // arcs of all earlier tiles
  uint64_t scan2[2 * (TNT / 32)];
  uint32_t nruns, ticket, ok;
};

static_assert(sizeof(DecSmem) <= 44 * 1024, "five decode CTAs per SM");

__device__ __forceinline__ uint64_t ld_acquire_u64(const unsigned long long* p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t dec_clock_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// bit of light field k of a vertex starting at bit st with field width w
template <int IDM>
__device__ __forceinline__ uint64_t dec_pos(uint64_t st, uint32_t k, uint32_t w, uint32_t s) {
  if (IDM == ID_LOCAL_GAP) return k == 0 ? st : st + s + (uint64_t)(k - 1) * w;
  return st + (uint64_t)k * w;
}
template <int IDM>
__device__ __forceinline__ uint32_t dec_width(uint32_t k, uint32_t w, uint32_t s) {
  return (IDM == ID_LOCAL_GAP && k == 0) ? s : w;
}

// segmented combine of (absolute?, value) pairs: x = e then x
__device__ __forceinline__ void seg_after(uint32_t& xf, uint32_t& xv, uint32_t ef, uint32_t ev) {
  if (!xf) { xv += ev; xf = ef; }
}

// Arcs of all tiles before tile b (warp 0 of the tile CTA; the result in lane 0).
// Returns false if a wait ran out.
__device__ __forceinline__ bool dec_lookback(const DecArgs& a, uint64_t b, uint64_t& base) {
  const uint32_t lane = threadIdx.x & 31u;
  base = 0;
  int64_t p = (int64_t)b - 1 - (int64_t)lane;  // lane 0 reads the nearest predecessor
  const uint64_t t0 = dec_clock_ns();
  uint64_t spins = 0;
  while (true) {
    const uint64_t v = p >= 0 ? ld_acquire_u64(a.tile_status + p) : DEC_INCL;  // nothing before tile 0
    const uint64_t flag = v >> 62;
    const uint32_t incl = __ballot_sync(LG_FULL_MASK, flag == 2);
    const uint32_t stop = incl ? (uint32_t)(__ffs(incl) - 1) : 31u;  // nearest inclusive prefix
    const uint32_t unready = __ballot_sync(LG_FULL_MASK, flag == 0 && lane <= stop);
    if (unready) {
      if (++spins > (a.wait_ns >> 5) + 1024 || ((spins & 63u) == 0 && dec_clock_ns() - t0 > a.wait_ns)) return false;
      __nanosleep(32);
      continue;
    }
    base += warp_sum<uint64_t>(lane <= stop ? (v & DEC_VAL) : 0ull);
    if (incl) return true;
    p -= 32;
  }
}

template <int IDM, int OFF>
__global__ void __launch_bounds__(TNT, 5) k_dec_local(GView g, DecArgs a) {
  extern __shared__ __align__(16) unsigned char dec_smem_raw[];
  DecSmem& sm = *reinterpret_cast<DecSmem*>(dec_smem_raw);
  TileSmem& ts = sm.t;
  const uint64_t ntiles = (g.n + TV - 1) / TV;
  if (threadIdx.x == 0) sm.ticket = atomicAdd(a.ticket, 1u);
  __syncthreads();
  const uint64_t b = sm.ticket;
  const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
  if (b >= ntiles) {
    // heavy items, a warp each; the row start comes from the tile that owns the vertex
    const uint64_t it = (b - ntiles) * (TNT / 32) + wid;
    if (it >= g.n_items) return;
    const HeavyItem h = g.items[it];
    uint64_t o = 0;
    bool ok = true;
    if (lane == 0) {
      const uint64_t t0 = dec_clock_ns();
      uint64_t spins = 0;
      while (ld_acquire_u32(a.tile_ready + h.v / TV) == 0) {
        if (++spins > (a.wait_ns >> 5) + 1024 || ((spins & 63u) == 0 && dec_clock_ns() - t0 > a.wait_ns)) {
          ok = false;
          break;
        }
        __nanosleep(64);
      }
      if (ok) o = __ldcg(a.row_ptr + h.v);
      else atomicOr(a.err, DERR_INTERNAL);
    }
    if (!__shfl_sync(LG_FULL_MASK, ok ? 1u : 0u, 0)) return;
    o = __shfl_sync(LG_FULL_MASK, o, 0);
    dec_fields<IDM, HEAVY_U>(g, a, h.bit, h.w, h.f0, h.f0 + h.nf, h.carry, o);
    return;
  }
  // ---- tile: offsets and geometry
  const uint64_t v0 = b * TV;
  const int cnt = (int)min((uint64_t)TV, g.n - v0);
  tile_offsets<OFF>(g, v0, cnt, ts.xs, ts.ts);
  __syncthreads();
  uint32_t lc = 0, lf = 0, hc = 0;
  uint64_t all = 0;
  bool light[TV / TNT];
  uint32_t dq[TV / TNT];
#pragma unroll
  for (int q = 0; q < TV / TNT; q++) {
    const int i = threadIdx.x * (TV / TNT) + q;
    light[q] = false;
    dq[q] = 0;
    if (i < cnt) {
      uint64_t start; uint32_t d, w;
      vgeo<IDM>(g, ts.xs[i], ts.xs[i + 1], start, d, w);
      ts.st[i] = start; ts.deg[i] = d; ts.wid[i] = (uint8_t)w;
      dq[q] = d;
      all += d;
      if (d > 0 && d <= g.heavy_min) { light[q] = true; lc++; lf += d; }
      hc += d > g.heavy_min;
    }
  }
  // one pass over the block: (heavy count, light count, light fields) packed
  // into 16 / 16 / 32 bits, and the sum of all degrees
  uint64_t lpre, apre, ltot, atot;
  block_excl_scan2<uint64_t, TNT>(((uint64_t)hc << 48) | ((uint64_t)lc << 32) | lf, all, lpre, apre, ltot, atot,
                                  sm.scan2);  // xs reads are done
  const bool no_heavy = (ltot >> 48) == 0;
  ltot &= (1ull << 48) - 1;
  lpre &= (1ull << 48) - 1;
  uint64_t* pre_all = ts.xs;  // reused: in-tile exclusive prefix of all degrees
  {
    uint32_t ci = (uint32_t)(lpre >> 32), cf = (uint32_t)lpre;
    uint64_t ca = apre;
#pragma unroll
    for (int q = 0; q < TV / TNT; q++) {
      const int i = threadIdx.x * (TV / TNT) + q;
      if (i < cnt) pre_all[i] = ca;
      ca += dq[q];
      if (light[q]) {
        ts.clist[ci] = (uint16_t)i;
        ts.fpre[ci] = cf;
        ci++;
        cf += dq[q];
      }
    }
  }
  if (threadIdx.x == 0) {
    ts.nlight = (uint32_t)(ltot >> 32);
    ts.nfields = (uint32_t)ltot;
    ts.fpre[ts.nlight] = (uint32_t)ltot;
    sm.ok = 1;
  }
  // ---- arcs before this tile (decoupled look-back), then the row offsets
  if (wid == 0) {
    if (lane == 0) {
      if (b == 0) st_release_u64(a.tile_status, DEC_INCL | atot);
      else st_release_u64(a.tile_status + b, DEC_AGG | atot);
    }
    uint64_t base = 0;
    bool ok = true;
    if (b > 0) ok = dec_lookback(a, b, base);
    if (lane == 0) {
      if (!ok) { atomicOr(a.err, DERR_INTERNAL); sm.ok = 0; }
      if (b > 0) st_release_u64(a.tile_status + b, DEC_INCL | (base + atot));
      sm.base = base;
    }
  }
  __syncthreads();
  if (!sm.ok) return;
  const uint64_t base = sm.base;
  for (int i = threadIdx.x; i < cnt; i += TNT) a.row_out[v0 + i] = base + pre_all[i];
  if (v0 + (uint64_t)cnt == g.n && threadIdx.x == 0) a.row_out[g.n] = base + atot;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    st_release_u32(a.tile_ready + b, 1u);
  }
  const uint32_t nl = ts.nlight;
  if (nl == 0) return;
  // ---- runs of light vertices with contiguous output rows (a heavy vertex breaks a run)
  if (no_heavy) {  // one run
    if (threadIdx.x == 0) {
      sm.nruns = 1;
      sm.rfirst[0] = 0;
      sm.rfirst[1] = (uint16_t)nl;
      sm.rdelta[0] = base + pre_all[ts.clist[0]];
    }
  } else {
    uint32_t fl[TV / TNT], c = 0;
    uint64_t dl[TV / TNT];
#pragma unroll
    for (int q = 0; q < TV / TNT; q++) {
      const uint32_t j = threadIdx.x * (TV / TNT) + q;
      fl[q] = 0;
      dl[q] = 0;
      if (j < nl) {
        // output index of light field f is row_ptr[v] + (f - fpre[j]): constant offset
        // along light vertices with only zero-degree vertices between them
        dl[q] = base + pre_all[ts.clist[j]] - (uint64_t)ts.fpre[j];
        fl[q] = j == 0 || dl[q] != base + pre_all[ts.clist[j - 1]] - (uint64_t)ts.fpre[j - 1];
        c += fl[q];
      }
    }
    uint32_t total;
    uint32_t pos = block_excl_scan<uint32_t, TNT>(c, total, ts.ts.red);
#pragma unroll
    for (int q = 0; q < TV / TNT; q++) {
      const uint32_t j = threadIdx.x * (TV / TNT) + q;
      if (fl[q]) { sm.rfirst[pos] = (uint16_t)j; sm.rdelta[pos] = dl[q]; pos++; }
    }
    if (threadIdx.x == 0) { sm.nruns = total; sm.rfirst[total] = (uint16_t)nl; }
  }
  __syncthreads();
  // ---- warps: ranges of whole light vertices balanced by fields, decoded in
  // windows of up to DEC_WF fields that never cross a run (contiguous stream
  // bits, one output offset); lanes decode DEC_P consecutive fields each
  {
    const uint32_t s = g.s, F = ts.nfields;
    const uint32_t* fpre = ts.fpre;
    DecWarp& W = sm.w[wid];
    // warp range: from the first light vertex starting at or after F * wid / 8
    // to the one starting at or after F * (wid + 1) / 8
    auto first_at_or_after = [&](uint32_t target) {
      uint32_t lo = 0, hi = nl;
      while (lo < hi) { const uint32_t m = (lo + hi) >> 1; if (fpre[m] < target) lo = m + 1; else hi = m; }
      return lo;
    };
    const uint32_t jr0 = first_at_or_after((uint32_t)((uint64_t)F * wid / (TNT / 32)));
    const uint32_t jr1 = wid + 1 == TNT / 32 ? nl : first_at_or_after((uint32_t)((uint64_t)F * (wid + 1) / (TNT / 32)));
    const uint32_t Rend = fpre[jr1];
    // the last light vertex holding field f, searched in [lo, hi]
    auto vertex_of = [&](uint32_t f, uint32_t lo, uint32_t hi) {
      while (lo < hi) { const uint32_t m = (lo + hi + 1) >> 1; if (fpre[m] <= f) lo = m; else hi = m - 1; }
      return lo;
    };
    uint32_t q = 0;           // run holding W0
    uint32_t wcarry = 0;      // absolute ID of the field before W0 (gap mode, W0 inside a vertex)
    for (uint32_t W0 = fpre[jr0]; W0 < Rend;) {
      while (q + 1 < sm.nruns && fpre[sm.rfirst[q + 1]] <= W0) q++;
      const uint32_t RE = min(Rend, fpre[sm.rfirst[q + 1]]);
      uint32_t Fw = min((uint32_t)DEC_WF, RE - W0);
      const uint32_t ja = vertex_of(W0, jr0, jr1 - 1);
      const int ia = ts.clist[ja];
      const uint64_t bA = dec_pos<IDM>(ts.st[ia], W0 - fpre[ja], ts.wid[ia], s);
      const uint64_t wA = (bA >> 5) & ~3ull;
      uint32_t jb, nw;
      while (true) {  // shrink the window until its stream words fit
        jb = vertex_of(W0 + Fw - 1, ja, jr1 - 1);
        const int ib = ts.clist[jb];
        const uint32_t kb = W0 + Fw - 1 - fpre[jb];
        const uint64_t bB = dec_pos<IDM>(ts.st[ib], kb, ts.wid[ib], s) + dec_width<IDM>(kb, ts.wid[ib], s);
        nw = (uint32_t)(((bB + 31) >> 5) + 1 - wA);
        if (nw <= DEC_WCAP || Fw == 1) break;
        Fw = (Fw + 1) >> 1;
      }
      const uint4* src = reinterpret_cast<const uint4*>(g.A32 + wA);
      uint4* dst = reinterpret_cast<uint4*>(W.words);
      for (uint32_t x = lane; x * 4 < nw; x += 32) dst[x] = __ldcs(src + x);
      __syncwarp();
      const uint32_t fa = W0 + Fw * lane / 32, fb = W0 + Fw * (lane + 1) / 32;
      uint32_t lastf = 0, lastv = 0, pend = fa;
      if (fa < fb) {
        uint32_t j = vertex_of(fa, ja, jb), f = fa, k = fa - fpre[j];
        pend = k ? min(fb, fpre[j + 1]) : fa;  // fields of a neighborhood entered mid-way
        const uint64_t wbase = wA * 32;
        while (f < fb) {
          const int i = ts.clist[j];
          const uint32_t w = ts.wid[i], mw = mask_lo(w);
          uint32_t m = min(ts.deg[i] - k, fb - f);
          uint32_t* out = W.stage + (f - W0);
          f += m;
          uint32_t p = (uint32_t)(dec_pos<IDM>(ts.st[i], k, w, s) - wbase);
          uint32_t run = 0;
          if (IDM == ID_LOCAL_GAP && k == 0) {
            run = __funnelshift_r(W.words[p >> 5], W.words[(p >> 5) + 1], p & 31u) & mask_lo(s);
            *out++ = run;
            p += s;
            m--;
          }
          for (; m; m--) {
            const uint32_t x = __funnelshift_r(W.words[p >> 5], W.words[(p >> 5) + 1], p & 31u) & mw;
            p += w;
            if (IDM == ID_LOCAL_GAP) { run += x; *out++ = run; }
            else *out++ = x;
          }
          lastf = k == 0;
          lastv = run;
          j++;
          k = 0;
        }
      }
      if (IDM == ID_LOCAL_GAP) {
        // inclusive segmented scan of (lastf, lastv) over the lanes, after the
        // window's carry (the absolute ID of field W0 - 1 when W0 is inside a vertex)
        const uint32_t cf = fpre[ja] < W0 ? 1u : 0u, cv = cf ? wcarry : 0u;
        uint32_t xf = lastf, xv = lastv;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t ef = __shfl_up_sync(LG_FULL_MASK, xf, o), ev = __shfl_up_sync(LG_FULL_MASK, xv, o);
          if (lane >= (uint32_t)o) seg_after(xf, xv, ef, ev);
        }
        uint32_t lf = __shfl_up_sync(LG_FULL_MASK, xf, 1), lv = __shfl_up_sync(LG_FULL_MASK, xv, 1);
        if (lane == 0) { lf = 0; lv = 0; }
        seg_after(lf, lv, cf, cv);
        for (uint32_t f = fa; f < pend; f++) W.stage[f - W0] += lv;
        seg_after(xf, xv, cf, cv);
        wcarry = __shfl_sync(LG_FULL_MASK, xv, 31);  // the absolute ID of the window's last field
      }
      __syncwarp();
      const uint64_t dst0 = sm.rdelta[q] + W0;
      for (uint32_t x = lane; x < Fw; x += 32) __stcs(a.ids + dst0 + x, W.stage[x]);
      __syncwarp();
      W0 += Fw;
    }
  }
}

// ===========================================================================
// heavy-vertex schedule, built once per graph from the encoded arrays
// ===========================================================================
__device__ __forceinline__ uint32_t items_of(const GView& g, uint32_t d) {
  return d > g.heavy_min ? (d + g.heavy_seg - 1) / g.heavy_seg : 0u;
}

template <int IDM, int OFF>
__global__ void __launch_bounds__(TNT) k_plan_count(GView g, PlanArgs p) {
  __shared__ TileSmem sm;
  const uint64_t v0 = (uint64_t)blockIdx.x * TV;
  const int cnt = (int)min((uint64_t)TV, g.n - v0);
  tile_offsets<OFF>(g, v0, cnt, sm.xs, sm.ts);
  __syncthreads();
  uint64_t mine = 0;
  for (int i = threadIdx.x; i < cnt; i += TNT) {
    uint64_t start; uint32_t d, w;
    vgeo<IDM>(g, sm.xs[i], sm.xs[i + 1], start, d, w);
    const uint32_t k = items_of(g, d);
    mine += ((uint64_t)k << 32) | (k > 1 ? 1u : 0u);
  }
  uint64_t total;
  block_excl_scan<uint64_t, TNT>(mine, total, sm.red64);
  if (threadIdx.x == 0) {
    p.tile_count[blockIdx.x] = (uint32_t)(total >> 32);
    p.multi_count[blockIdx.x] = (uint32_t)total;
  }
}

template <int IDM, int OFF>
__global__ void __launch_bounds__(TNT) k_plan_fill(GView g, PlanArgs p) {
  __shared__ TileSmem sm;
  const uint64_t v0 = (uint64_t)blockIdx.x * TV;
  const int cnt = (int)min((uint64_t)TV, g.n - v0);
  tile_offsets<OFF>(g, v0, cnt, sm.xs, sm.ts);
  __syncthreads();
  uint64_t st_[TV / TNT];
  uint32_t d_[TV / TNT], w_[TV / TNT];
  uint64_t mine = 0;
#pragma unroll
  for (int q = 0; q < TV / TNT; q++) {
    const int i = threadIdx.x * (TV / TNT) + q;
    d_[q] = 0;
    if (i < cnt) vgeo<IDM>(g, sm.xs[i], sm.xs[i + 1], st_[q], d_[q], w_[q]);
    const uint32_t k = items_of(g, d_[q]);
    mine += ((uint64_t)k << 32) | (k > 1 ? 1u : 0u);
  }
  uint64_t total;
  const uint64_t pre = block_excl_scan<uint64_t, TNT>(mine, total, sm.red64);
  uint64_t it = p.tile_off[blockIdx.x] + (pre >> 32);
  uint64_t slot = p.multi_off[blockIdx.x] + (uint32_t)pre;
#pragma unroll
  for (int q = 0; q < TV / TNT; q++) {
    const uint32_t k = items_of(g, d_[q]);
    if (k == 0) continue;
    const uint64_t first = it;
    for (uint32_t j = 0; j < k; j++) {
      HeavyItem h;
      h.bit = st_[q];
      h.v = (uint32_t)(v0 + threadIdx.x * (TV / TNT) + q);
      h.f0 = j * g.heavy_seg;
      h.nf = min(g.heavy_seg, d_[q] - h.f0);
      h.carry = 0;
      h.deg = d_[q];
      h.first = (uint32_t)first;
      h.nitems = k;
      h.w = w_[q];
      h.slot = k > 1 ? (uint32_t)slot : 0xffffffffu;
      p.items[it++] = h;
    }
    if (k > 1) p.multi[slot++] = (uint32_t)first;
  }
}

// per item of a split vertex: the sum of its values (for gap-coded IDs the
// first item's sum is its last ID, later items' sums are sums of differences)
template <int IDM, int OFF>
__global__ void __launch_bounds__(256) k_plan_carry(GView g, PlanArgs p) {
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t it = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); it < g.n_items; it += warps) {
    const HeavyItem h = g.items[it];
    if (h.nitems == 1) continue;
    uint32_t carry = 0;
    const uint32_t f1 = h.f0 + h.nf;
    for (uint32_t base = h.f0; base < f1; base += 32 * HEAVY_U) {
      uint32_t id[HEAVY_U];
      warp_ids<IDM, HEAVY_U>(g, h.bit, h.w, base, f1, carry, id);
    }
    if ((threadIdx.x & 31) == 0) p.segsum[it] = carry;
  }
}

// ===========================================================================
// launchers
// ===========================================================================
inline unsigned tiles_of(uint64_t n) { return (unsigned)((n + TV - 1) / TV); }

template <int IDM, int OFF>
cudaError_t launch_pr_init(const GView& g, const PrArgs& a, cudaStream_t st) {
  k_pr_init<IDM, OFF><<<tiles_of(g.n), TNT, 0, st>>>(g, a);
  count_launch();
  return cudaGetLastError();
}
template <int IDM, int OFF>
cudaError_t launch_pr_pull(const GView& g, const PrArgs& a, cudaStream_t st) {
  k_pr_pull<IDM, OFF><<<heavy_blocks(g.n_items) + tiles_of(g.n), TNT, 0, st>>>(g, a);
  count_launch();
  return cudaGetLastError();
}
template <int IDM, int OFF>
cudaError_t launch_bfs_pull(const GView& g, const BfsArgs& a, int mb, cudaStream_t st) {
  const unsigned grid = heavy_blocks(g.n_items) + tiles_of(g.n);
  if (mb == 2) { k_bfs_pull<IDM, OFF, uint16_t><<<grid, TNT, 0, st>>>(g, a); count_launch(); }
  else if (mb == 4) { k_bfs_pull<IDM, OFF, uint32_t><<<grid, TNT, 0, st>>>(g, a); count_launch(); }
  else { k_bfs_pull<IDM, OFF, uint64_t><<<grid, TNT, 0, st>>>(g, a); count_launch(); }
  return cudaGetLastError();
}
template <int IDM, int OFF>
cudaError_t launch_bfs_push(const GView& g, const BfsArgs& a, int mb, cudaStream_t st) {
  if (a.queue_in_len == 0) return cudaSuccess;
  const unsigned hb = heavy_blocks(g.n_items);
  const unsigned grid = hb + grid_for(a.queue_in_len, 8, 152 * 16);
  if (mb == 2) { k_bfs_push<IDM, OFF, uint16_t><<<grid, 256, 0, st>>>(g, a, hb); count_launch(); }
  else if (mb == 4) { k_bfs_push<IDM, OFF, uint32_t><<<grid, 256, 0, st>>>(g, a, hb); count_launch(); }
  else { k_bfs_push<IDM, OFF, uint64_t><<<grid, 256, 0, st>>>(g, a, hb); count_launch(); }
  return cudaGetLastError();
}
template <int IDM, int OFF>
cudaError_t launch_nbr_degrees(const GView& g, const NbrArgs& a, cudaStream_t st) {
  if (a.k == 0) return cudaSuccess;
  k_nbr_degrees<IDM, OFF><<<grid_for(a.k, 8, 152 * 16), 256, 0, st>>>(g, a);
  count_launch();
  return cudaGetLastError();
}
template <int IDM, int OFF>
cudaError_t launch_nbr_decode(const GView& g, const NbrArgs& a, cudaStream_t st) {
  if (a.k == 0) return cudaSuccess;
  k_nbr_decode<IDM, OFF><<<grid_for(a.k, 8, 152 * 16), 256, 0, st>>>(g, a);
  count_launch();
  return cudaGetLastError();
}
template <int IDM, int OFF>
cudaError_t launch_plan_count(const GView& g, const PlanArgs& p, cudaStream_t st) {
  k_plan_count<IDM, OFF><<<tiles_of(g.n), TNT, 0, st>>>(g, p);
  count_launch();
  return cudaGetLastError();
}
template <int IDM, int OFF>
cudaError_t launch_plan_fill(const GView& g, const PlanArgs& p, cudaStream_t st) {
  k_plan_fill<IDM, OFF><<<tiles_of(g.n), TNT, 0, st>>>(g, p);
  count_launch();
  return cudaGetLastError();
}
template <int IDM, int OFF>
cudaError_t launch_plan_carry(const GView& g, const PlanArgs& p, cudaStream_t st) {
  if (g.n_items == 0) return cudaSuccess;
  k_plan_carry<IDM, OFF><<<grid_for(g.n_items, 8, 152 * 16), 256, 0, st>>>(g, p);
  count_launch();
  return cudaGetLastError();
}

template <int IDM, int OFF>
cudaError_t launch_ppr_pull(const GView& g, const PprArgs& a, cudaStream_t st) {
  k_ppr_pull<IDM, OFF><<<heavy_blocks(g.n_items) + tiles_of(g.n), TNT, 0, st>>>(g, a);
  count_launch();
  return cudaGetLastError();
}
template <int IDM, int OFF>
cudaError_t launch_ppr_join(const GView& g, float* cin, uint32_t slot, uint32_t src, cudaStream_t st) {
  k_ppr_join<IDM, OFF><<<1, 32, 0, st>>>(g, cin, slot, src);
  count_launch();
  return cudaGetLastError();
}

template <int IDM, int OFF>
cudaError_t launch_dec_all(const GView& g, const DecArgs& a, cudaStream_t st) {
  if (g.n == 0) return cudaSuccess;
  if constexpr (IDM == ID_GLOBAL || IDM == ID_CSR32) {
    const uint64_t tiles = tiles_of(g.n);
    const uint64_t unit = (uint64_t)(TNT / 32) * DEC_FLAT_CH;
    const uint64_t per_block = (g.arcs + tiles - 1) / tiles;
    k_dec_flat<IDM, OFF><<<(unsigned)tiles, 256, 0, st>>>(g, a, (per_block + unit - 1) / unit * unit);
  } else {
    const cudaError_t e = cudaFuncSetAttribute(k_dec_local<IDM, OFF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)sizeof(DecSmem));
    if (e != cudaSuccess) return e;
    k_dec_local<IDM, OFF><<<tiles_of(g.n) + heavy_blocks(g.n_items), TNT, sizeof(DecSmem), st>>>(g, a);
  }
  count_launch();
  return cudaGetLastError();
}

template <int IDM, int OFF>
const TravOps* make_ops() {
  static const TravOps ops = {
      &launch_pr_init<IDM, OFF>,    &launch_pr_pull<IDM, OFF>,     &launch_bfs_pull<IDM, OFF>,
      &launch_bfs_push<IDM, OFF>,   &launch_nbr_degrees<IDM, OFF>, &launch_nbr_decode<IDM, OFF>,
      &launch_plan_count<IDM, OFF>, &launch_plan_fill<IDM, OFF>,   &launch_plan_carry<IDM, OFF>,
      &launch_ppr_pull<IDM, OFF>,   &launch_ppr_join<IDM, OFF>,   &launch_dec_all<IDM, OFF>,
  };
  return &ops;
}

}  // namespace lg
