// Batches of independent graphs in one persistent launch.
//
// Every graph g of the batch is encoded with its own widths -- vertex IDs at
// s_g = bits(n_g - 1) (Section 3.2.1, 0-based IDs) and offsets packed at
// w_O = bits(arcs_g) (Section 3.4, "ptrLogn") -- then searched breadth-first
// from its vertex 0 and ranked by pull PageRank (Section 7.1.2), reading only
// the stream it just wrote.  The whole batch is ONE kernel launch, captured
// once as a CUDA graph and replayed.
//
// Work queue.  Items are (graph, member) pairs in a size-ordered queue
// (largest per-member work first).  A graph larger than the tile gets a team
// of p members that take p consecutive queue slots; the team splits encode
// words and vertex ranges evenly and meets at team barriers between phases,
// BFS levels and PageRank iterations.  A team waits only for slots that
// running CTAs take next, so the queue makes progress as long as p <= grid;
// each wait also has a time limit after which the CTA records a timeout and
// abandons the graph.  Streams are read with ordinary loads after the encode
// barrier (see sfield); per-vertex data that other CTAs of a team rewrite
// between sweeps or levels (contributions, depths, queues) is read with
// L2-coherent loads (ld.global.cg).
//
// Each graph decodes its neighborhoods with T lanes per vertex (T = 1, 4, 8
// or 32); T per average-degree class and the team tile are chosen by a timing
// autotuner when the batch is created.
#include <cstdio>
#include <cstring>
#include <vector>
#include <algorithm>
#include <mutex>

#include "lg_internal.h"

namespace lg {

struct BatchGraph {
  uint64_t vbase;   // first vertex in the batch vertex space
  uint64_t abase;   // first arc in the input arrays
  uint64_t a_word;  // first u64 word of the graph's A stream
  uint64_t o_word;  // first u64 word of its packed offsets
  uint32_t n, arcs;
  uint32_t s, w_O;
  uint32_t lanes;   // decode lanes per vertex
  uint32_t team;    // CTAs working on the graph
  uint32_t pad[2];
};
static_assert(sizeof(BatchGraph) == 64, "BatchGraph layout");

struct BatchItem {
  uint32_t g, member;
};

constexpr int BNT = 256;  // threads per batch CTA
constexpr uint32_t PH_ENCODE = 1, PH_BFS = 2, PH_PR = 4;
constexpr uint32_t BERR_TIMEOUT = 1;
constexpr uint32_t SYNC_WORDS = 4;  // per graph: barrier count + 3 rotating queue counters
constexpr uint32_t INF32 = 0xffffffffu;

struct BatchArgs {
  const BatchGraph* graphs;
  const BatchItem* items;
  uint32_t n_items;
  unsigned int* next;       // queue head
  uint32_t* sync;           // SYNC_WORDS per graph
  uint32_t* err;
  const uint64_t* row_ptr;  // input CSR (global arc offsets)
  const uint32_t* col;      // input local IDs
  uint64_t* A;
  uint64_t* O;
  uint32_t* depth;          // output, batch vertex space
  float* ranks;             // output
  uint32_t* q0;
  uint32_t* q1;             // BFS queues, batch vertex space
  float* c0;
  float* c1;                // PageRank contributions
  float damp;
  uint32_t iters;
  uint32_t phases;
  int32_t lanes_override;   // > 0: this T for every graph (autotuner)
  uint64_t wait_ns;         // team barrier time limit
};

// field of w <= 32 bits at bit p of a graph's stream.  Every graph's streams
// start on a 128-byte line and are written before the barrier that ends the
// encode phase; a CTA never reads a line of them before it is written (no
// line is shared with another graph, and stores do not allocate in L1), so
// after that barrier ordinary L1-cached loads see the written words.
__device__ __forceinline__ uint32_t sfield(const uint64_t* S, uint64_t p, uint32_t w) {
  const uint64_t wi = p >> 6;
  const uint32_t sh = (uint32_t)p & 63u;
  uint64_t v = S[wi] >> sh;
  if (sh + w > 64) v |= S[wi + 1] << (64u - sh);
  return (uint32_t)(v & ((1ull << w) - 1ull));
}

// per-vertex arrays rewritten by other CTAs of a team between sweeps / levels
// are read through L2 (ld.global.cg); a single-CTA graph reads them plainly
template <bool TEAM>
__device__ __forceinline__ float cget(const float* p) {
  return TEAM ? __ldcg(p) : *p;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Team barrier: every member adds one to the graph's counter and waits until
// it reaches p * round.  Returns false (for the whole CTA) if the wait ran
// out; the error word then holds BERR_TIMEOUT.
__device__ bool team_sync(const BatchArgs& a, uint32_t* bar, uint32_t p, uint32_t round) {
  __shared__ int ok;
  __syncthreads();
  if (p == 1) return true;
  if (threadIdx.x == 0) {
    ok = 1;
    __threadfence();
    atomicAdd(bar, 1u);
    const uint32_t target = p * round;
    const uint64_t t0 = globaltimer_ns();
    // the clock decides; the spin cap (each spin polls L2, well over 16 ns)
    // only bounds the loop should the clock not advance
    const uint64_t max_spins = a.wait_ns / 16 + 1024;
    for (uint64_t spins = 1; *(volatile uint32_t*)bar < target; spins++) {
      __nanosleep(64);
      if (spins >= max_spins || ((spins & 63u) == 0 && globaltimer_ns() - t0 > a.wait_ns)) {
        ok = 0;
        atomicOr(a.err, BERR_TIMEOUT);
        break;
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

template <int T>
__device__ __forceinline__ float group_sum(float x) {
#pragma unroll
  for (int o = T / 2; o > 0; o >>= 1) x += __shfl_xor_sync(LG_FULL_MASK, x, o);
  return x;
}

// Pull PageRank over vertices [v0, v1) of one graph, T lanes per vertex; each
// lane keeps four fields (and their four gathers) in flight.
template <int T, bool TEAM>
__device__ void pr_sweep(const BatchArgs& a, const BatchGraph& G, uint32_t v0, uint32_t v1, const float* cin,
                         float* cout, bool last) {
  const uint64_t* A = a.A + G.a_word;
  const uint64_t* O = a.O + G.o_word;
  constexpr uint32_t groups = BNT / T;
  const uint32_t gid = threadIdx.x / T, lane = threadIdx.x % T;
  const float base = (1.0f - a.damp) / (float)G.n;
  const uint32_t s = G.s;
  // every group runs the same number of rounds so the shuffles stay converged
  for (uint32_t vb = v0; vb < v1; vb += groups) {
    const uint32_t v = vb + gid;
    float sum = 0.f, sum2 = 0.f;
    uint32_t x0 = 0, x1 = 0;
    if (v < v1) {
      x0 = sfield(O, (uint64_t)v * G.w_O, G.w_O);
      x1 = sfield(O, (uint64_t)(v + 1) * G.w_O, G.w_O);
      uint32_t j = x0 + lane;
      for (; j + 3 * T < x1; j += 4 * T) {
        const uint32_t u0 = sfield(A, (uint64_t)j * s, s), u1 = sfield(A, (uint64_t)(j + T) * s, s);
        const uint32_t u2 = sfield(A, (uint64_t)(j + 2 * T) * s, s), u3 = sfield(A, (uint64_t)(j + 3 * T) * s, s);
        const float f0 = cget<TEAM>(cin + u0), f1 = cget<TEAM>(cin + u1);
        const float f2 = cget<TEAM>(cin + u2), f3 = cget<TEAM>(cin + u3);
        sum += f0 + f1;
        sum2 += f2 + f3;
      }
      for (; j < x1; j += T) sum += cget<TEAM>(cin + sfield(A, (uint64_t)j * s, s));
    }
    sum += sum2;
    if (T > 1) sum = group_sum<T>(sum);
    if (v < v1 && lane == 0) {
      const uint32_t d = x1 - x0;
      const float r = base + a.damp * sum;
      cout[v] = d ? r / (float)d : 0.f;
      if (last) a.ranks[G.vbase + v] = r;
    }
  }
}

// One BFS level: this member's share of the frontier, T lanes per vertex.
template <int T>
__device__ void bfs_level(const BatchArgs& a, const BatchGraph& G, uint32_t member, uint32_t p, const uint32_t* qin,
                          uint32_t qlen, uint32_t* qout, uint32_t* qn, uint32_t level) {
  const uint64_t* A = a.A + G.a_word;
  const uint64_t* O = a.O + G.o_word;
  uint32_t* depth = a.depth + G.vbase;
  constexpr uint32_t groups = BNT / T;
  const uint32_t gid = threadIdx.x / T, lane = threadIdx.x % T;
  for (uint32_t q = member * groups + gid; q < qlen; q += p * groups) {
    const uint32_t v = __ldcg(qin + q);
    const uint32_t x0 = sfield(O, (uint64_t)v * G.w_O, G.w_O);
    const uint32_t x1 = sfield(O, (uint64_t)(v + 1) * G.w_O, G.w_O);
    for (uint32_t j = x0 + lane; j < x1; j += T) {
      const uint32_t u = sfield(A, (uint64_t)j * G.s, G.s);
      if (__ldcg(depth + u) == INF32 && atomicCAS(&depth[u], INF32, level + 1) == INF32) qout[atomicAdd(qn, 1u)] = u;
    }
  }
}

// Word-owner packing: word k of a stream of fixed-width records gets every
// record overlapping bits [64k, 64k + 64); rec(j) returns record j.
template <typename Rec>
__device__ __forceinline__ void pack_words(uint64_t* out, uint64_t k0, uint64_t k1, uint64_t nrec, uint32_t w,
                                           Rec rec) {
  for (uint64_t k = k0 + threadIdx.x; k < k1; k += BNT) {
    const uint64_t b0 = k * 64, j0 = b0 / w;
    uint64_t j1 = (b0 + 63) / w;
    if (j1 >= nrec) j1 = nrec - 1;
    uint64_t acc = 0;
    for (uint64_t j = j0; j <= j1; j++) {
      const int64_t off = (int64_t)(j * w) - (int64_t)b0;
      const uint64_t r = rec(j);
      acc |= off >= 0 ? (r << off) : (r >> (-off));
    }
    out[k] = acc;
  }
}

__device__ void process_item(const BatchArgs& a, uint32_t gi, uint32_t m) {
  const BatchGraph G = a.graphs[gi];
  const uint32_t p = G.team;
  uint32_t* bar = a.sync + (uint64_t)gi * SYNC_WORDS;
  uint32_t* cnt = bar + 1;
  uint32_t round = 0;
  const uint32_t T = a.lanes_override > 0 ? (uint32_t)a.lanes_override : G.lanes;
  const uint32_t v0 = (uint32_t)((uint64_t)G.n * m / p), v1 = (uint32_t)((uint64_t)G.n * (m + 1) / p);

  if (a.phases & PH_ENCODE) {
    const uint64_t wa = ((uint64_t)G.arcs * G.s + 63) / 64;
    const uint64_t wo = ((uint64_t)(G.n + 1) * G.w_O + 63) / 64;
    const uint32_t* col = a.col + G.abase;
    const uint64_t* rp = a.row_ptr + G.vbase;
    const uint64_t ab = G.abase;
    if (G.arcs)
      pack_words(a.A + G.a_word, wa * m / p, wa * (m + 1) / p, G.arcs, G.s,
                 [&](uint64_t j) { return (uint64_t)__ldg(col + j); });
    pack_words(a.O + G.o_word, wo * m / p, wo * (m + 1) / p, (uint64_t)G.n + 1, G.w_O,
               [&](uint64_t j) { return __ldg(rp + j) - ab; });
    if (!team_sync(a, bar, p, ++round)) return;
  }

  if (a.phases & PH_BFS) {
    uint32_t* depth = a.depth + G.vbase;
    for (uint32_t v = v0 + threadIdx.x; v < v1; v += BNT) depth[v] = INF32;
    __syncthreads();
    uint32_t* qa = a.q0 + G.vbase;
    uint32_t* qb = a.q1 + G.vbase;
    if (m == 0 && threadIdx.x == 0) {
      depth[0] = 0;
      qa[0] = 0;
    }
    if (!team_sync(a, bar, p, ++round)) return;
    uint32_t qlen = 1;
    for (uint32_t level = 0; qlen > 0 && level < G.n; level++) {
      // level L appends to counter L mod 3; counter (L+1) mod 3 was last read
      // before the previous barrier, so the leader clears it now
      uint32_t* qn = cnt + level % 3;
      if (m == 0 && threadIdx.x == 0) cnt[(level + 1) % 3] = 0;
      if (T == 1) bfs_level<1>(a, G, m, p, qa, qlen, qb, qn, level);
      else if (T == 4) bfs_level<4>(a, G, m, p, qa, qlen, qb, qn, level);
      else if (T == 8) bfs_level<8>(a, G, m, p, qa, qlen, qb, qn, level);
      else bfs_level<32>(a, G, m, p, qa, qlen, qb, qn, level);
      if (!team_sync(a, bar, p, ++round)) return;
      qlen = *(volatile uint32_t*)qn;
      uint32_t* t = qa;
      qa = qb;
      qb = t;
    }
  }

  if ((a.phases & PH_PR) && a.iters > 0) {
    const uint64_t* O = a.O + G.o_word;
    float* ci = a.c0 + G.vbase;
    float* co = a.c1 + G.vbase;
    const float r0 = 1.0f / (float)G.n;
    for (uint32_t v = v0 + threadIdx.x; v < v1; v += BNT) {
      const uint32_t d = sfield(O, (uint64_t)(v + 1) * G.w_O, G.w_O) - sfield(O, (uint64_t)v * G.w_O, G.w_O);
      ci[v] = d ? r0 / (float)d : 0.f;
    }
    if (!team_sync(a, bar, p, ++round)) return;
    for (uint32_t t = 0; t < a.iters; t++) {
      const bool last = t + 1 == a.iters;
      if (p > 1) {
        if (T == 1) pr_sweep<1, true>(a, G, v0, v1, ci, co, last);
        else if (T == 4) pr_sweep<4, true>(a, G, v0, v1, ci, co, last);
        else if (T == 8) pr_sweep<8, true>(a, G, v0, v1, ci, co, last);
        else pr_sweep<32, true>(a, G, v0, v1, ci, co, last);
      } else {
        if (T == 1) pr_sweep<1, false>(a, G, v0, v1, ci, co, last);
        else if (T == 4) pr_sweep<4, false>(a, G, v0, v1, ci, co, last);
        else if (T == 8) pr_sweep<8, false>(a, G, v0, v1, ci, co, last);
        else pr_sweep<32, false>(a, G, v0, v1, ci, co, last);
      }
      if (!team_sync(a, bar, p, ++round)) return;
      float* x = ci;
      ci = co;
      co = x;
    }
  }
}

__global__ void __launch_bounds__(BNT, 8) k_batch(BatchArgs a) {
  __shared__ unsigned int slot_s;
  for (;;) {
    if (threadIdx.x == 0) slot_s = atomicAdd(a.next, 1u);
    __syncthreads();
    const unsigned int slot = slot_s;
    __syncthreads();
    if (slot >= a.n_items) return;
    const BatchItem it = a.items[slot];
    if (a.graphs[it.g].n == 0) continue;
    process_item(a, it.g, it.member);
  }
}

// every graph's rows: bounds monotone inside the graph's arc range, local IDs
// < n_g, rows strictly increasing
__global__ void __launch_bounds__(BNT) k_batch_validate(const BatchGraph* graphs, uint32_t count,
                                                        const uint64_t* row_ptr, const uint32_t* col, int* err) {
  for (uint32_t g = blockIdx.x; g < count; g += gridDim.x) {
    const BatchGraph G = graphs[g];
    int flags = 0;
    for (uint32_t v = threadIdx.x; v < G.n; v += BNT) {
      const uint64_t lo = row_ptr[G.vbase + v], hi = row_ptr[G.vbase + v + 1];
      if (hi < lo || lo < G.abase || hi > G.abase + G.arcs) {
        flags |= DERR_ROWPTR;
        continue;
      }
      for (uint64_t j = lo; j < hi; j++) {
        if (col[j] >= G.n) flags |= DERR_COL_RANGE;
        if (j > lo && col[j] <= col[j - 1]) flags |= DERR_UNSORTED;
      }
    }
    if (flags) atomicOr(err, flags);
  }
}

__global__ void k_gather_abase(const uint64_t* vptr, const uint64_t* row_ptr, uint32_t count, uint64_t* out) {
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g <= count; g += gridDim.x * blockDim.x)
    out[g] = row_ptr[vptr[g]];
}

}  // namespace lg

using namespace lg;

struct lg_batch {
  int device = 0;
  uint32_t count = 0;
  uint64_t V = 0, arcs = 0;
  const uint64_t* row_ptr = nullptr;  // caller's input (kept by reference)
  const uint32_t* col = nullptr;
  lg_batch_opts opts{};
  std::vector<BatchGraph> host;
  std::vector<BatchItem> items_h;
  BatchGraph* graphs = nullptr;  // device descriptors
  BatchItem* items = nullptr;
  uint32_t n_items = 0;
  unsigned int* next = nullptr;  // queue head
  uint32_t* sync = nullptr;      // SYNC_WORDS per graph
  uint32_t* err = nullptr;
  uint64_t* A = nullptr;
  uint64_t* O = nullptr;
  uint64_t words_A = 0, words_O = 0;
  uint32_t* q0 = nullptr;
  uint32_t* q1 = nullptr;
  float* c0 = nullptr;
  float* c1 = nullptr;
  uint64_t tile_arcs = 0;
  int grid = 1;
  uint64_t launches = 0;         // batch kernel launches (each graph replay counts one)
  std::mutex mu;                 // guards the cached executable graph
  cudaStream_t cap = nullptr;    // private stream used for capture
  cudaGraphExec_t exec = nullptr;
  uint32_t exec_iters = 0;
  float exec_damp = 0.f;
  uint32_t* exec_depth = nullptr;
  float* exec_ranks = nullptr;
};

namespace {
lg_status batch_fail(const char* what, cudaError_t e) {
  char msg[256];
  snprintf(msg, sizeof msg, "%s: %s", what, cudaGetErrorString(e));
  set_error_message(msg);
  return e == cudaErrorMemoryAllocation ? LG_ENOMEM : LG_ECUDA;
}
#define BTRY(call)                                       \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return batch_fail(#call, e_); \
  } while (0)

// Team sizes and the queue: by decreasing work per member, a team's members
// on consecutive slots.
void plan_queue(lg_batch* b, uint64_t tile) {
  const uint32_t max_team = (uint32_t)std::max(1, b->grid / 2);
  for (auto& x : b->host) {
    uint64_t p = tile ? (x.arcs + tile - 1) / tile : 1;
    p = std::max<uint64_t>(p, 1);
    p = std::min<uint64_t>(p, max_team);
    p = std::min<uint64_t>(p, std::max<uint32_t>(1, x.n / BNT));
    x.team = (uint32_t)p;
  }
  std::vector<uint32_t> order(b->count);
  for (uint32_t g = 0; g < b->count; g++) order[g] = g;
  auto work = [&](uint32_t g) { return ((uint64_t)b->host[g].arcs * 2 + b->host[g].n) / b->host[g].team; };
  std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) { return work(x) > work(y); });
  b->items_h.clear();
  for (uint32_t g : order)
    for (uint32_t m = 0; m < b->host[g].team; m++) b->items_h.push_back({g, m});
  b->n_items = (uint32_t)b->items_h.size();
}

lg_status upload_plan(lg_batch* b, cudaStream_t st) {
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  BTRY(cudaStreamSynchronize(st));
  cudaFree(b->items);
  b->items = nullptr;
  BTRY(cudaMalloc((void**)&b->items, b->items_h.size() * sizeof(BatchItem) + 16));
  BTRY(cudaMemcpyAsync(b->items, b->items_h.data(), b->items_h.size() * sizeof(BatchItem), cudaMemcpyHostToDevice,
                       st));
  BTRY(cudaMemcpyAsync(b->graphs, b->host.data(), b->count * sizeof(BatchGraph), cudaMemcpyHostToDevice, st));
  BTRY(cudaStreamSynchronize(st));
  return LG_OK;
}

BatchArgs make_args(lg_batch* b, uint32_t* depth, float* ranks, float damp, uint32_t iters, uint32_t phases,
                    const BatchItem* items, uint32_t n_items, int lanes) {
  BatchArgs a;
  memset(&a, 0, sizeof(a));
  a.graphs = b->graphs;
  a.items = items;
  a.n_items = n_items;
  a.next = b->next;
  a.sync = b->sync;
  a.err = b->err;
  a.row_ptr = b->row_ptr;
  a.col = b->col;
  a.A = b->A;
  a.O = b->O;
  a.depth = depth;
  a.ranks = ranks;
  a.q0 = b->q0;
  a.q1 = b->q1;
  a.c0 = b->c0;
  a.c1 = b->c1;
  a.damp = damp;
  a.iters = iters;
  a.phases = phases;
  a.lanes_override = lanes;
  a.wait_ns = (uint64_t)(b->opts.wait_limit_us ? b->opts.wait_limit_us : 2000000u) * 1000ull;
  return a;
}

// one run: reset the queue head, team counters and error word, then the persistent launch
void enqueue_run(lg_batch* b, const BatchArgs& a, cudaStream_t st) {
  cudaMemsetAsync(b->next, 0, sizeof(unsigned int), st);
  cudaMemsetAsync(b->sync, 0, (size_t)b->count * SYNC_WORDS * 4, st);
  cudaMemsetAsync(b->err, 0, 4, st);
  k_batch<<<b->grid, BNT, 0, st>>>(a);
}

lg_status time_run(lg_batch* b, const BatchArgs& a, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, int reps,
                   float* best) {
  *best = 1e30f;
  for (int r = 0; r < reps; r++) {
    BTRY(cudaEventRecord(e0, st));
    enqueue_run(b, a, st);
    b->launches++;
    count_launch();
    BTRY(cudaGetLastError());
    BTRY(cudaEventRecord(e1, st));
    BTRY(cudaEventSynchronize(e1));
    float ms = 0;
    BTRY(cudaEventElapsedTime(&ms, e0, e1));
    *best = std::min(*best, ms);
  }
  return LG_OK;
}

// Timing autotuner.  (1) T per average-degree class: the class's 64 largest
// graphs run alone (encode + 2 PageRank sweeps) with T = 1, 4, 8 and 32.
// (2) The team tile, if not fixed: the whole batch (encode + BFS + 2 sweeps)
// with tiles of 2^18 .. 2^21 arcs.
lg_status autotune(lg_batch* b, uint32_t* depth_tmp, float* ranks_tmp, cudaStream_t st, cudaEvent_t e0,
                   cudaEvent_t e1) {
  const int cand_t[4] = {1, 4, 8, 32};
  std::vector<std::vector<uint32_t>> bins(5);
  for (uint32_t g = 0; g < b->count; g++) {
    const BatchGraph& x = b->host[g];
    const double avg = x.n ? (double)x.arcs / x.n : 0.0;
    bins[avg <= 8 ? 0 : avg <= 16 ? 1 : avg <= 32 ? 2 : avg <= 64 ? 3 : 4].push_back(g);
  }
  const size_t max_items = 64 * (size_t)std::max(1, b->grid / 2);
  BatchItem* dlist = nullptr;
  BTRY(cudaMalloc((void**)&dlist, max_items * sizeof(BatchItem) + 16));
  lg_status s = LG_OK;
  for (auto& bin : bins) {
    if (bin.empty()) continue;
    std::vector<uint32_t> sample(bin);
    std::sort(sample.begin(), sample.end(),
              [&](uint32_t x, uint32_t y) { return b->host[x].arcs > b->host[y].arcs; });
    if (sample.size() > 64) sample.resize(64);
    std::vector<BatchItem> its;
    for (uint32_t g : sample)
      for (uint32_t m = 0; m < b->host[g].team; m++) its.push_back({g, m});
    if (cudaMemcpyAsync(dlist, its.data(), its.size() * sizeof(BatchItem), cudaMemcpyHostToDevice, st) !=
        cudaSuccess) {
      s = batch_fail("lg_batch_create: autotune upload", cudaGetLastError());
      break;
    }
    float best = 1e30f;
    int best_t = 8;
    for (int c = 0; c < 4 && s == LG_OK; c++) {
      BatchArgs a = make_args(b, depth_tmp, ranks_tmp, 0.85f, 2, PH_ENCODE | PH_PR, dlist, (uint32_t)its.size(),
                              cand_t[c]);
      float ms = 0;
      s = time_run(b, a, st, e0, e1, 2, &ms);
      if (ms < best) {
        best = ms;
        best_t = cand_t[c];
      }
    }
    for (uint32_t g : bin) b->host[g].lanes = (uint32_t)best_t;
  }
  cudaFree(dlist);
  if (s != LG_OK) return s;
  if (b->opts.tile_arcs == 0) {
    const uint64_t cand_k[4] = {1ull << 18, 1ull << 19, 1ull << 20, 1ull << 21};
    float best = 1e30f;
    uint64_t best_k = b->tile_arcs;
    for (uint64_t k : cand_k) {
      plan_queue(b, k);
      if ((s = upload_plan(b, st)) != LG_OK) return s;
      BatchArgs a = make_args(b, depth_tmp, ranks_tmp, 0.85f, 2, PH_ENCODE | PH_BFS | PH_PR, b->items, b->n_items, 0);
      float ms = 0;
      if ((s = time_run(b, a, st, e0, e1, 2, &ms)) != LG_OK) return s;
      if (ms < best) {
        best = ms;
        best_k = k;
      }
    }
    b->tile_arcs = best_k;
    plan_queue(b, best_k);
  }
  if ((s = upload_plan(b, st)) != LG_OK) return s;
  uint32_t herr = 0;
  BTRY(cudaMemcpy(&herr, b->err, 4, cudaMemcpyDeviceToHost));
  if (herr) {
    set_error_message("lg_batch_create: a team barrier ran out of time during autotuning");
    return LG_ETIMEOUT;
  }
  return LG_OK;
}

lg_status batch_create_impl(lg_batch* b, const uint64_t* graph_vptr, cudaStream_t st) {
  const uint32_t G = b->count;
  std::vector<uint64_t> vptr(G + 1), abase(G + 1);
  BTRY(cudaMemcpyAsync(vptr.data(), graph_vptr, (G + 1) * 8, cudaMemcpyDeviceToHost, st));
  BTRY(cudaStreamSynchronize(st));
  if (vptr[0] != 0 || vptr[G] != b->V) {
    set_error_message("lg_batch_create: graph_vptr must start at 0 and end at V");
    return LG_EINVAL;
  }
  for (uint32_t g = 0; g < G; g++)
    if (vptr[g + 1] < vptr[g] || vptr[g + 1] - vptr[g] > 0xffffffffull) {
      set_error_message("lg_batch_create: graph_vptr not monotone or a graph has >= 2^32 vertices");
      return LG_EINVAL;
    }
  uint64_t* d_ab = nullptr;
  BTRY(cudaMalloc((void**)&d_ab, (G + 1) * 8));
  k_gather_abase<<<grid_for(G + 1, 256, 1024), 256, 0, st>>>(graph_vptr, b->row_ptr, G, d_ab);
  count_launch();
  cudaError_t ce = cudaMemcpyAsync(abase.data(), d_ab, (G + 1) * 8, cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  cudaFree(d_ab);
  if (ce != cudaSuccess) return batch_fail("lg_batch_create: graph bounds", ce);
  if (abase[0] != 0 || abase[G] != b->arcs) {
    set_error_message("lg_batch_create: row_ptr must span [0, arcs)");
    return LG_EINVAL;
  }
  b->host.assign(G, BatchGraph{});
  uint64_t aw = 0, ow = 0;
  for (uint32_t g = 0; g < G; g++) {
    BatchGraph& x = b->host[g];
    if (abase[g + 1] < abase[g] || abase[g + 1] - abase[g] > 0xffffffffull) {
      set_error_message("lg_batch_create: row_ptr not monotone across graphs or a graph has >= 2^32 arcs");
      return LG_EINVAL;
    }
    x.vbase = vptr[g];
    x.abase = abase[g];
    x.n = (uint32_t)(vptr[g + 1] - vptr[g]);
    x.arcs = (uint32_t)(abase[g + 1] - abase[g]);
    x.s = x.n > 1 ? host_bits(x.n - 1) : 1;  // ceil(log2 n) for 0-based IDs
    x.w_O = x.arcs ? host_bits(x.arcs) : 1;  // offsets 0 .. arcs
    x.lanes = b->opts.lanes ? b->opts.lanes : 8;
    x.team = 1;
    x.a_word = aw;
    x.o_word = ow;
    const uint64_t wa = ((uint64_t)x.arcs * x.s + 63) / 64;
    const uint64_t wo = ((uint64_t)(x.n + 1) * x.w_O + 63) / 64;
    aw += (wa + 15) / 16 * 16;  // each graph's streams start on a 128-byte line
    ow += (wo + 15) / 16 * 16;
  }
  b->words_A = aw + 4;  // + zero guard
  b->words_O = ow + 4;
  int per_sm = 0, sms = 0;
  BTRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, BNT, 0));
  BTRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
  b->grid = std::max(1, per_sm) * std::max(1, sms);
  b->tile_arcs = b->opts.tile_arcs ? b->opts.tile_arcs : (1ull << 19);
  plan_queue(b, b->tile_arcs);
  BTRY(cudaMalloc((void**)&b->graphs, G * sizeof(BatchGraph) + 16));
  BTRY(cudaMalloc((void**)&b->next, 16));
  BTRY(cudaMalloc((void**)&b->sync, (size_t)G * SYNC_WORDS * 4 + 16));
  BTRY(cudaMalloc((void**)&b->err, 16));
  BTRY(cudaMalloc((void**)&b->A, b->words_A * 8));
  BTRY(cudaMalloc((void**)&b->O, b->words_O * 8));
  BTRY(cudaMalloc((void**)&b->q0, b->V * 4 + 16));
  BTRY(cudaMalloc((void**)&b->q1, b->V * 4 + 16));
  BTRY(cudaMalloc((void**)&b->c0, b->V * 4 + 16));
  BTRY(cudaMalloc((void**)&b->c1, b->V * 4 + 16));
  BTRY(cudaMemsetAsync(b->A, 0, b->words_A * 8, st));
  BTRY(cudaMemsetAsync(b->O, 0, b->words_O * 8, st));
  BTRY(cudaMemsetAsync(b->err, 0, 16, st));
  lg_status s = upload_plan(b, st);
  if (s != LG_OK) return s;
  int* d_err = nullptr;
  BTRY(cudaMalloc((void**)&d_err, 4));
  BTRY(cudaMemsetAsync(d_err, 0, 4, st));
  k_batch_validate<<<grid_for(G, 1, 152 * 16), BNT, 0, st>>>(b->graphs, G, b->row_ptr, b->col, d_err);
  count_launch();
  int herr = 0;
  ce = cudaMemcpyAsync(&herr, d_err, 4, cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  cudaFree(d_err);
  if (ce != cudaSuccess) return batch_fail("lg_batch_create: validation", ce);
  if (herr) {
    set_error_message("lg_batch_create: invalid input (row bounds, local ID >= n_g, or unsorted row)");
    return LG_EINVAL;
  }
  BTRY(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
  if (b->opts.autotune) {
    uint32_t* dtmp = nullptr;
    float* rtmp = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BTRY(cudaMalloc((void**)&dtmp, b->V * 4 + 16));
    ce = cudaMalloc((void**)&rtmp, b->V * 4 + 16);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    s = ce == cudaSuccess ? autotune(b, dtmp, rtmp, st, e0, e1) : batch_fail("lg_batch_create: autotune setup", ce);
    cudaStreamSynchronize(st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(dtmp);
    cudaFree(rtmp);
    if (s != LG_OK) return s;
  }
  if (b->opts.flags & LG_BATCH_FLAG_DROP_MEMBER) {
    // failure injection on the host: the last member of the first team is
    // left out of the queue, so that team's first barrier can end only by its
    // time limit
    for (size_t i = 0; i < b->items_h.size(); i++) {
      const uint32_t g = b->items_h[i].g;
      if (b->host[g].team < 2) continue;
      size_t j = i;
      while (j + 1 < b->items_h.size() && b->items_h[j + 1].g == g) j++;
      b->items_h.erase(b->items_h.begin() + (long)j);
      b->n_items--;
      break;
    }
    if ((s = upload_plan(b, st)) != LG_OK) return s;
  }
  return LG_OK;
}
}  // namespace

extern "C" void lg_batch_free(lg_batch* b) {
  if (!b) return;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != b->device) cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->cap) cudaStreamDestroy(b->cap);
  cudaFree(b->graphs);
  cudaFree(b->items);
  cudaFree(b->next);
  cudaFree(b->sync);
  cudaFree(b->err);
  cudaFree(b->A);
  cudaFree(b->O);
  cudaFree(b->q0);
  cudaFree(b->q1);
  cudaFree(b->c0);
  cudaFree(b->c1);
  if (prev != b->device) cudaSetDevice(prev);
  delete b;
}

extern "C" lg_status lg_batch_create(const uint64_t* graph_vptr, const uint64_t* row_ptr, const uint32_t* col,
                                     uint32_t count, uint64_t V, uint64_t arcs, const lg_batch_opts* opts,
                                     void* stream, lg_batch** out) {
  set_error_message("");
  if (!out || !graph_vptr || !row_ptr || (arcs && !col) || count == 0) {
    set_error_message("lg_batch_create: null argument or empty batch");
    return LG_EINVAL;
  }
  *out = nullptr;
  if (opts && opts->lanes && opts->lanes != 1 && opts->lanes != 4 && opts->lanes != 8 && opts->lanes != 32) {
    set_error_message("lg_batch_create: lanes must be 0, 1, 4, 8 or 32");
    return LG_EINVAL;
  }
  lg_batch* b = new lg_batch();
  cudaGetDevice(&b->device);
  b->count = count;
  b->V = V;
  b->arcs = arcs;
  b->row_ptr = row_ptr;
  b->col = col;
  if (opts) b->opts = *opts;
  if (b->opts.lanes) b->opts.autotune = 0;
  lg_status s = batch_create_impl(b, graph_vptr, reinterpret_cast<cudaStream_t>(stream));
  if (s != LG_OK) {
    lg_batch_free(b);
    return s;
  }
  *out = b;
  return LG_OK;
}

extern "C" lg_status lg_batch_run(lg_batch* b, float damping, uint32_t iters, uint32_t* depths, float* ranks,
                                  void* stream) {
  set_error_message("");
  if (!b || !depths || !ranks) {
    set_error_message("lg_batch_run: null argument");
    return LG_EINVAL;
  }
  if (!(damping >= 0.0f && damping <= 1.0f)) {
    set_error_message("lg_batch_run: damping must be in [0, 1]");
    return LG_EINVAL;
  }
  std::lock_guard<std::mutex> lock(b->mu);
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != b->device) cudaSetDevice(b->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  lg_status status = LG_OK;
  if (!b->exec || b->exec_iters != iters || b->exec_damp != damping || b->exec_depth != depths ||
      b->exec_ranks != ranks) {
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    BatchArgs a = make_args(b, depths, ranks, damping, iters, PH_ENCODE | PH_BFS | PH_PR, b->items, b->n_items, 0);
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      enqueue_run(b, a, b->cap);
      e = cudaStreamEndCapture(b->cap, &graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      b->exec = nullptr;
      status = batch_fail("lg_batch_run: graph capture", e);
    } else {
      b->exec_iters = iters;
      b->exec_damp = damping;
      b->exec_depth = depths;
      b->exec_ranks = ranks;
    }
  }
  if (status == LG_OK) {
    cudaError_t e = cudaGraphLaunch(b->exec, st);
    b->launches++;
    count_launch();
    if (e != cudaSuccess) status = batch_fail("lg_batch_run: cudaGraphLaunch", e);
  }
  if (prev != b->device) cudaSetDevice(prev);
  return status;
}

extern "C" lg_status lg_batch_status(lg_batch* b, void* stream) {
  set_error_message("");
  if (!b) {
    set_error_message("lg_batch_status: null argument");
    return LG_EINVAL;
  }
  uint32_t herr = 0;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(&herr, b->err, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return batch_fail("lg_batch_status", e);
  if (herr & BERR_TIMEOUT) {
    set_error_message("lg_batch_run: a team barrier ran out of time; that graph's results are incomplete");
    return LG_ETIMEOUT;
  }
  return LG_OK;
}

extern "C" lg_status lg_batch_info_get(const lg_batch* b, lg_batch_info* out) {
  if (!b || !out) {
    set_error_message("lg_batch_info_get: null argument");
    return LG_EINVAL;
  }
  memset(out, 0, sizeof(*out));
  out->count = b->count;
  out->V = b->V;
  out->arcs = b->arcs;
  out->A = b->A;
  out->words_A = b->words_A;
  out->O = b->O;
  out->words_O = b->words_O;
  out->graphs = reinterpret_cast<const lg_batch_graph*>(b->graphs);
  out->n_items = b->n_items;
  out->grid = (uint32_t)b->grid;
  out->threads = BNT;
  out->tile_arcs = b->tile_arcs;
  uint64_t teams = 0, bits = 0, max_team = 0;
  for (const auto& x : b->host) {
    teams += x.team > 1;
    max_team = std::max<uint64_t>(max_team, x.team);
    bits += (uint64_t)x.arcs * x.s + (uint64_t)(x.n + 1) * x.w_O;
    const int k = x.lanes == 1 ? 0 : x.lanes == 4 ? 1 : x.lanes == 8 ? 2 : 3;
    out->graphs_by_lanes[k]++;
  }
  out->teams = (uint32_t)teams;
  out->max_team = (uint32_t)max_team;
  out->bits_total = bits;
  out->launches = b->launches;
  return LG_OK;
}
