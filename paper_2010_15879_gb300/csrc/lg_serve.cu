// Serving: a request loop over resident compressed graphs with continuous
// batching.  The paper has no serving layer; its operations are the
// neighborhood access of Section 3.7.2 (getNeighbors), BFS and personalized
// PageRank of Section 7.1.2 -- this file keeps graphs resident and runs many
// such queries at once.
//
// Per resident graph there are three engines, each a host thread with its own
// CUDA stream, so work of different engines overlaps on the device:
//   * BFS engine: one multi-source sweep with 64 slots (bit s of the visited
//     and frontier masks is slot s).  Between two levels, waiting sources join
//     free slots of the RUNNING sweep (their source enters the current
//     frontier; the kernels count its depths from its join level); a slot
//     whose frontier bits died out retires: its row is copied out, its
//     visited bits are cleared, and the slot is free again.
//   * PPR engine: PPR_K slots of personalized PageRank iterated together, the
//     contributions of all slots of a vertex in one 32-byte sector; a request
//     joins a free slot between two iterations and retires after its own
//     iteration count.  A freed slot is reused after one sweep in which the
//     kernel writes its column to zero.
//   * neighborhood engine: all waiting lookups merged into one decode launch.
// Admission is by device memory: every request's device state (a BFS depth
// row, a PPR result vector, a lookup's output) comes from a fixed device
// arena, and a request waits until its allocation succeeds.  Results land in
// a pinned host arena owned by the server until the client releases them.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "lg_arena.h"
#include "lg_internal.h"

namespace lg {

constexpr uint32_t INFD = 0xffffffffu;
constexpr int BFS_SLOTS = 64;

// ---------------------------------------------------------------- kernels
// new sources enter the current frontier (one thread: duplicates merge)
struct JoinItem {
  uint32_t src, slot;  // stored label of the source, slot
  uint32_t orig, pad;  // the source's original ID (its index in the depth row)
};
__global__ void k_bfs_join(uint64_t* vis, uint64_t* cur, uint32_t* const* rows, uint32_t* row_base,
                           const JoinItem* joins, uint32_t J, uint32_t level, uint32_t* queue, uint32_t* qlen) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  uint32_t q = *qlen;
  for (uint32_t j = 0; j < J; j++) {
    const uint32_t s = joins[j].src;
    const uint64_t bit = 1ull << joins[j].slot;
    if (cur[s] == 0) queue[q++] = s;
    cur[s] |= bit;
    vis[s] |= bit;
    rows[joins[j].slot][joins[j].orig] = 0;
    row_base[joins[j].slot] = level;  // later depths are written as level + 1 - base
  }
  *qlen = q;
}

// OR of the frontier masks listed in the queue (which slots are still alive)
__global__ void k_frontier_or(const uint64_t* front, const uint32_t* queue, const uint32_t* qlen,
                              unsigned long long* alive) {
  const uint32_t n = *qlen;
  uint64_t acc = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) acc |= front[queue[i]];
  for (int o = 16; o > 0; o >>= 1) acc |= __shfl_xor_sync(LG_FULL_MASK, acc, o);
  if ((threadIdx.x & 31) == 0 && acc) atomicOr(alive, (unsigned long long)acc);
}

__global__ void k_and_mask(uint64_t* m, uint64_t n, uint64_t keep) {
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x)
    m[v] &= keep;
}

__global__ void k_clear_queue64(uint64_t* m, const uint32_t* queue, uint32_t nq) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += gridDim.x * blockDim.x) m[queue[i]] = 0;
}

}  // namespace lg

using namespace lg;

namespace {

uint64_t now_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Req {
  uint64_t ticket = 0, user = 0;
  uint32_t kind = 0, graph = 0, source = 0, iters = 0;
  float damping = 0.85f;
  std::vector<uint32_t> vertices;
  uint64_t t_submit = 0, t_admit = 0, t_done = 0;
  int32_t status = LG_OK;
  void* host = nullptr;  // result (pinned arena)
  uint64_t bytes = 0, count = 0;
};

struct Engine;

}  // namespace

struct lg_server {
  int device = 0;
  std::vector<const lg_graph*> graphs;
  std::vector<std::vector<uint32_t>> perms;  // host copies of relabeled graphs' perm
  lg_server_opts opts{};
  // arenas
  std::mutex mem_mu;
  RangeArena dev_arena, host_arena;
  char* dev_base = nullptr;
  char* host_base = nullptr;
  // completed results
  std::mutex done_mu;
  std::condition_variable done_cv;
  std::deque<Req*> done;
  std::unordered_map<uint64_t, Req*> delivered;
  std::atomic<uint64_t> next_ticket{1};
  std::atomic<bool> stop{false};
  std::vector<std::unique_ptr<Engine>> engines;  // 3 per graph: BFS, PPR, NBR
  // statistics
  std::atomic<uint64_t> submitted{0}, completed{0}, by_kind[3]{}, failed{0};
  std::atomic<uint64_t> bfs_levels{0}, bfs_joins{0}, bfs_joins_running{0}, bfs_max_active{0};
  std::atomic<uint64_t> ppr_iterations{0}, ppr_joins{0}, ppr_joins_running{0}, ppr_max_active{0};
  std::atomic<uint64_t> nbr_batches{0}, nbr_max_batch{0}, admission_waits{0};

  void* dev_alloc(uint64_t bytes) {
    std::lock_guard<std::mutex> l(mem_mu);
    uint64_t off;
    if (!dev_arena.alloc(bytes, &off)) return nullptr;
    return dev_base + off;
  }
  void dev_free(void* p) {
    if (!p) return;
    std::lock_guard<std::mutex> l(mem_mu);
    dev_arena.release((uint64_t)((char*)p - dev_base));
  }
  void* host_alloc(uint64_t bytes) {
    std::lock_guard<std::mutex> l(mem_mu);
    uint64_t off;
    if (!host_arena.alloc(bytes, &off)) return nullptr;
    return host_base + off;
  }
  void* host_alloc_wait(uint64_t bytes) {  // results wait for the client to release older ones
    {
      std::lock_guard<std::mutex> l(mem_mu);
      if (bytes > host_arena.size()) return nullptr;  // can never fit
    }
    for (;;) {
      void* p = host_alloc(bytes);
      if (p || stop.load()) return p;
      std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
  }
  void host_free(void* p) {
    if (!p) return;
    std::lock_guard<std::mutex> l(mem_mu);
    host_arena.release((uint64_t)((char*)p - host_base));
  }
  void post(Req* r) {
    r->t_done = now_ns();
    completed++;
    if (r->status != LG_OK) failed++;
    {
      std::lock_guard<std::mutex> l(done_mu);
      done.push_back(r);
    }
    done_cv.notify_all();
  }
  static void bump_max(std::atomic<uint64_t>& m, uint64_t v) {
    uint64_t c = m.load();
    while (v > c && !m.compare_exchange_weak(c, v)) {
    }
  }
};

namespace {

struct Engine {
  lg_server* srv;
  uint32_t gi;
  const lg_graph* g;
  GView view;
  const TravOps* ops;
  cudaStream_t st = nullptr;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Req*> pending;
  std::thread th;
  bool ok = true;  // false after a CUDA failure: every later request fails at once
  // device time of the engine's kernels, from CUDA events on its stream
  std::atomic<uint64_t> ops_done{0}, gpu_ns{0};
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  void add_elapsed(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) == cudaSuccess) gpu_ns += (uint64_t)((double)ms * 1e6);
    ops_done++;
  }
  lg_status make_timers() {
    if (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess) return LG_ECUDA;
    return LG_OK;
  }
  void destroy_timers() {
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
  }

  const std::vector<uint32_t>* perm_h = nullptr;  // original -> stored label (relabeled graphs)

  Engine(lg_server* s, uint32_t i) : srv(s), gi(i), g(s->graphs[i]) {
    view = make_view(g);
    ops = trav_ops((int)g->id_mode, (int)g->off_mode);
    if (g->perm) perm_h = &s->perms[i];
  }
  uint32_t stored(uint32_t v) const { return perm_h ? (*perm_h)[v] : v; }
  virtual ~Engine() = default;
  virtual lg_status setup() = 0;
  virtual void loop() = 0;
  virtual void teardown() {}

  // Stream priority by latency class: lookups (tiny, latency-bound) first,
  // then BFS levels, then PageRank sweeps (full-graph, throughput-bound), so
  // the block scheduler dispatches a lookup's blocks ahead of the queued
  // blocks of a long sweep.
  cudaError_t make_stream(int rank) {
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    // numerically lower is more urgent: greatest <= mid <= least
    const int prio = rank == 0 ? greatest : rank == 1 ? least + (greatest - least) / 2 : least;
    return cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, prio);
  }
  void start() {
    th = std::thread([this] {
      cudaSetDevice(srv->device);
      loop();
    });
  }
  void push(Req* r) {
    {
      std::lock_guard<std::mutex> l(mu);
      pending.push_back(r);
    }
    cv.notify_one();
  }
  // wait until there is pending work (or stop); returns false on stop
  bool wait_pending(bool have_active) {
    std::unique_lock<std::mutex> l(mu);
    if (have_active) return !srv->stop.load();
    cv.wait_for(l, std::chrono::milliseconds(50), [&] { return srv->stop.load() || !pending.empty(); });
    return !srv->stop.load();
  }
  void fail_all(Req* r) {
    r->status = LG_ECUDA;
    srv->post(r);
  }
  void drain_pending_failed() {
    std::deque<Req*> q;
    {
      std::lock_guard<std::mutex> l(mu);
      q.swap(pending);
    }
    for (Req* r : q) fail_all(r);
  }
};

#define ECHK(call)                 \
  do {                             \
    if ((call) != cudaSuccess) {   \
      ok = false;                  \
      return;                      \
    }                              \
  } while (0)

// ------------------------------------------------------------------ BFS
struct BfsEngine : Engine {
  uint64_t n;
  uint64_t *vis = nullptr, *fa = nullptr, *fb = nullptr, *hacc = nullptr;
  uint32_t *qa = nullptr, *qb = nullptr, *counters = nullptr;
  unsigned long long* alive = nullptr;
  uint32_t** rows_dev = nullptr;
  uint32_t* base_dev = nullptr;  // join level of each slot
  JoinItem* joins_dev = nullptr;
  int* err = nullptr;
  // pinned staging
  uint32_t** rows_h = nullptr;
  JoinItem* joins_h = nullptr;
  uint32_t* small_h = nullptr;  // [0] queue length, [1] pairs, [2] join queue length, [4..5] alive
  struct Slot {
    Req* r = nullptr;
    uint32_t* row = nullptr;
    uint32_t join_level = 0;
  } slots[BFS_SLOTS];
  uint32_t nslots;
  uint64_t active = 0;
  uint32_t level = 0, nq = 0;
  uint64_t* cur = nullptr;
  uint64_t* nxt = nullptr;
  uint32_t *qcur = nullptr, *qnxt = nullptr;

  BfsEngine(lg_server* s, uint32_t i) : Engine(s, i), n(g->n) {
    nslots = std::min<uint32_t>(BFS_SLOTS, s->opts.bfs_slots ? s->opts.bfs_slots : BFS_SLOTS);
  }

  lg_status setup() override {
    cudaError_t e = cudaSuccess;
    auto A = [&](void** p, size_t b) {
      if (e == cudaSuccess) e = cudaMalloc(p, b);
    };
    A((void**)&vis, n * 8 + 16);
    A((void**)&fa, n * 8 + 16);
    A((void**)&fb, n * 8 + 16);
    A((void**)&hacc, g->n_multi * 8 + 16);
    A((void**)&qa, n * 4 + 16);
    A((void**)&qb, n * 4 + 16);
    A((void**)&counters, 64);
    A((void**)&alive, 16);
    A((void**)&rows_dev, BFS_SLOTS * sizeof(void*));
    A((void**)&base_dev, BFS_SLOTS * sizeof(uint32_t));
    A((void**)&joins_dev, BFS_SLOTS * sizeof(JoinItem));
    A((void**)&err, 16);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&rows_h, BFS_SLOTS * sizeof(void*), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&joins_h, BFS_SLOTS * sizeof(JoinItem), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&small_h, 64, cudaHostAllocDefault);
    if (e == cudaSuccess) e = make_stream(1);
    if (e == cudaSuccess) e = cudaMemsetAsync(vis, 0, n * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(fa, 0, n * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(fb, 0, n * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(hacc, 0, g->n_multi * 8 + 16, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, 16, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      set_error_message(cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? LG_ENOMEM : LG_ECUDA;
    }
    if (make_timers() != LG_OK) return LG_ECUDA;
    memset(rows_h, 0, BFS_SLOTS * sizeof(void*));
    cur = fa;
    nxt = fb;
    qcur = qa;
    qnxt = qb;
    return LG_OK;
  }

  void teardown() override {
    cudaFree(vis); cudaFree(fa); cudaFree(fb); cudaFree(hacc); cudaFree(qa); cudaFree(qb);
    cudaFree(counters); cudaFree(alive); cudaFree(rows_dev); cudaFree(base_dev); cudaFree(joins_dev);
    cudaFree(err);
    cudaFreeHost(rows_h); cudaFreeHost(joins_h); cudaFreeHost(small_h);
    destroy_timers();
    if (st) cudaStreamDestroy(st);
  }

  // waiting sources take free slots while device memory for their rows lasts
  bool mem_blocked = false;
  uint32_t admit() {
    uint32_t J = 0;
    mem_blocked = false;
    std::lock_guard<std::mutex> l(mu);
    while (!pending.empty()) {
      int s = -1;
      for (uint32_t k = 0; k < nslots; k++)
        if (!((active >> k) & 1ull) && !slots[k].r) { s = (int)k; break; }
      if (s < 0) break;
      uint32_t* row = (uint32_t*)srv->dev_alloc(n * 4);
      if (!row) {
        srv->admission_waits++;
        mem_blocked = true;
        break;
      }
      Req* r = pending.front();
      pending.pop_front();
      r->t_admit = now_ns();
      slots[s].r = r;
      slots[s].row = row;
      slots[s].join_level = level;
      joins_h[J++] = JoinItem{stored(r->source), (uint32_t)s, r->source, 0};
    }
    return J;
  }

  void step(uint32_t J) {
    if (J) {
      if (active) srv->bfs_joins_running += J;
      srv->bfs_joins += J;
      for (uint32_t j = 0; j < J; j++) {
        const uint32_t s = joins_h[j].slot;
        ECHK(cudaMemsetAsync(slots[s].row, 0xff, n * 4, st));
        rows_h[s] = slots[s].row;
        active |= 1ull << s;
      }
      small_h[2] = nq;
      ECHK(cudaMemcpyAsync(rows_dev, rows_h, BFS_SLOTS * sizeof(void*), cudaMemcpyHostToDevice, st));
      ECHK(cudaMemcpyAsync(joins_dev, joins_h, J * sizeof(JoinItem), cudaMemcpyHostToDevice, st));
      ECHK(cudaMemcpyAsync(counters + 2, small_h + 2, 4, cudaMemcpyHostToDevice, st));
      k_bfs_join<<<1, 32, 0, st>>>(vis, cur, rows_dev, base_dev, joins_dev, J, level, qcur, counters + 2);
      count_launch();
      ECHK(cudaGetLastError());
      ECHK(cudaMemcpyAsync(small_h + 2, counters + 2, 4, cudaMemcpyDeviceToHost, st));
      ECHK(cudaStreamSynchronize(st));
      nq = small_h[2];
      srv->bump_max(srv->bfs_max_active, (uint64_t)__builtin_popcountll(active));
    }
    if (nq == 0) return;
    // one level of the sweep for every active slot
    ECHK(cudaEventRecord(t0, st));
    ECHK(cudaMemsetAsync(counters, 0, 8, st));
    ECHK(cudaMemsetAsync(alive, 0, 8, st));
    BfsArgs a;
    memset(&a, 0, sizeof(a));
    a.vis = vis;
    a.front_in = cur;
    a.front_out = nxt;
    a.rows = rows_dev;
    a.row_base = base_dev;
    a.row_perm = g->inv_perm;  // rows are indexed by original ID
    a.all_mask = active;
    a.S = BFS_SLOTS;
    a.level = level;
    a.queue_in = qcur;
    a.queue_in_len = nq;
    a.queue_out = qnxt;
    a.counters = counters;
    a.hacc = hacc;
    a.err = err;
    a.hot = hot_rows(g, 8);
    if ((uint64_t)nq > n / 64) {
      ECHK(ops->bfs_pull(view, a, 8, st));
      ECHK(bfs_finish_multi(view, a, 8, st));
    } else {
      ECHK(ops->bfs_push(view, a, 8, st));
    }
    k_frontier_or<<<grid_for(std::max<uint64_t>(nq, 1), 256, 1024), 256, 0, st>>>(nxt, qnxt, counters, alive);
    count_launch();
    ECHK(cudaGetLastError());
    // the consumed frontier becomes the next output buffer: clear it
    if ((uint64_t)nq * 16 < n) {
      k_clear_queue64<<<grid_for(nq, 256, 4096), 256, 0, st>>>(cur, qcur, nq);
      count_launch();
      ECHK(cudaGetLastError());
    } else {
      ECHK(cudaMemsetAsync(cur, 0, n * 8, st));
    }
    ECHK(cudaEventRecord(t1, st));
    ECHK(cudaMemcpyAsync(small_h, counters, 8, cudaMemcpyDeviceToHost, st));
    ECHK(cudaMemcpyAsync(small_h + 4, alive, 8, cudaMemcpyDeviceToHost, st));
    ECHK(cudaStreamSynchronize(st));
    add_elapsed(t0, t1);
    srv->bfs_levels++;
    std::swap(cur, nxt);
    std::swap(qcur, qnxt);
    nq = small_h[0];
    level++;
    uint64_t live;
    memcpy(&live, small_h + 4, 8);
    const uint64_t retire = active & ~live;
    if (!retire) return;
    // retire: rebase rows, copy them out, clear the slots' visited bits
    std::vector<int> out;
    for (int s = 0; s < BFS_SLOTS; s++) {
      if (!((retire >> s) & 1ull)) continue;
      Req* r = slots[s].r;
      r->host = srv->host_alloc_wait(n * 4);
      if (r->host) ECHK(cudaMemcpyAsync(r->host, slots[s].row, n * 4, cudaMemcpyDeviceToHost, st));
      out.push_back(s);
    }
    k_and_mask<<<grid_for(n, 256, 152 * 16), 256, 0, st>>>(vis, n, ~retire);
    count_launch();
    ECHK(cudaGetLastError());
    ECHK(cudaStreamSynchronize(st));
    active &= ~retire;
    for (int s : out) {
      Req* r = slots[s].r;
      r->bytes = n * 4;
      r->count = n;
      r->status = r->host ? LG_OK : LG_ENOMEM;
      srv->dev_free(slots[s].row);
      slots[s] = Slot{};
      rows_h[s] = nullptr;
      srv->post(r);
    }
  }

  void loop() override {
    while (!srv->stop.load()) {
      if (!ok) {
        drain_pending_failed();
        if (!wait_pending(false)) break;
        continue;
      }
      const uint32_t J = admit();
      if (J == 0 && active == 0) {
        if (mem_blocked) std::this_thread::sleep_for(std::chrono::microseconds(100));  // others hold the memory
        else if (!wait_pending(false)) break;
        continue;
      }
      step(J);
      if (!ok) {
        for (auto& s : slots)
          if (s.r) {
            srv->dev_free(s.row);
            fail_all(s.r);
            s = Slot{};
          }
        active = 0;
      }
    }
  }
};

// ------------------------------------------------------------------ PPR
struct PprEngine : Engine {
  uint64_t n;
  float *ca = nullptr, *cb = nullptr, *part = nullptr;
  enum { FREE_CLEAN, FREE_DIRTY, ACTIVE };
  struct Slot {
    Req* r = nullptr;
    float* res = nullptr;
    uint32_t t = 0;
    int state = FREE_CLEAN;
  } slots[PPR_K];
  uint32_t nslots;
  struct Inflight {
    cudaEvent_t ev;
    std::vector<std::pair<Req*, float*>> done;
  };
  std::deque<Inflight> inflight;   // retired slots whose result copies are queued
  std::deque<std::pair<cudaEvent_t, cudaEvent_t>> markers;  // (start, end) of each queued sweep
  std::vector<cudaEvent_t> free_events, free_timed;

  uint32_t hot;  // rows below this stored label are gathered with evict-last

  PprEngine(lg_server* s, uint32_t i) : Engine(s, i), n(g->n) {
    nslots = std::min<uint32_t>(PPR_K, s->opts.ppr_slots ? s->opts.ppr_slots : PPR_K);
    // DM relabeling puts the hubs first: keep their rows (up to 64 MB) in L2
    // and stream the others; without relabeling every row is kept
    hot = g->relabel ? (uint32_t)std::min<uint64_t>(n, (64ull << 20) / (PPR_K * 4)) : (uint32_t)n;
  }

  lg_status setup() override {
    cudaError_t e = cudaMalloc((void**)&ca, n * PPR_K * 4 + 64);
    if (e == cudaSuccess) e = cudaMalloc((void**)&cb, n * PPR_K * 4 + 64);
    if (e == cudaSuccess) e = cudaMalloc((void**)&part, (g->n_items + 1) * PPR_K * 4);
    if (e == cudaSuccess) e = make_stream(2);
    if (e == cudaSuccess) e = cudaMemsetAsync(ca, 0, n * PPR_K * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(cb, 0, n * PPR_K * 4, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      set_error_message(cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? LG_ENOMEM : LG_ECUDA;
    }
    return LG_OK;
  }
  void teardown() override {
    for (auto& f : inflight) cudaEventDestroy(f.ev);
    for (auto& m : markers) {
      cudaEventDestroy(m.first);
      cudaEventDestroy(m.second);
    }
    for (auto ev : free_events) cudaEventDestroy(ev);
    for (auto ev : free_timed) cudaEventDestroy(ev);
    cudaFree(ca); cudaFree(cb); cudaFree(part);
    if (st) cudaStreamDestroy(st);
  }
  cudaEvent_t get_timed() {
    if (!free_timed.empty()) {
      cudaEvent_t e = free_timed.back();
      free_timed.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void retire_marker() {
    auto m = markers.front();
    markers.pop_front();
    cudaEventSynchronize(m.second);
    add_elapsed(m.first, m.second);
    free_timed.push_back(m.first);
    free_timed.push_back(m.second);
  }
  cudaEvent_t get_event() {
    if (!free_events.empty()) {
      cudaEvent_t e = free_events.back();
      free_events.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    return e;
  }
  // post the retired slots whose copies have finished; `all` waits for every copy
  void reap(bool all) {
    while (!inflight.empty()) {
      Inflight& f = inflight.front();
      if (all) cudaEventSynchronize(f.ev);
      else if (cudaEventQuery(f.ev) != cudaSuccess) break;
      for (auto& d : f.done) {
        srv->dev_free(d.second);
        srv->post(d.first);
      }
      free_events.push_back(f.ev);
      inflight.pop_front();
    }
  }
  uint32_t active_mask() const {
    uint32_t m = 0;
    for (uint32_t k = 0; k < nslots; k++)
      if (slots[k].state == ACTIVE) m |= 1u << k;
    return m;
  }

  void loop() override {
    while (!srv->stop.load()) {
      if (!ok) {
        drain_pending_failed();
        if (!wait_pending(false)) break;
        continue;
      }
      // admit into clean free slots
      std::vector<uint32_t> joins;
      uint32_t act = active_mask();
      bool mem_blocked = false;
      {
        std::lock_guard<std::mutex> l(mu);
        bool dirty_only = true;
        for (uint32_t k = 0; k < nslots; k++)
          if (slots[k].state == FREE_CLEAN) dirty_only = false;
        if (!pending.empty() && act == 0 && dirty_only) {  // idle: zero both arrays, every slot clean
          if (cudaMemsetAsync(ca, 0, n * PPR_K * 4, st) != cudaSuccess ||
              cudaMemsetAsync(cb, 0, n * PPR_K * 4, st) != cudaSuccess)
            ok = false;
          for (uint32_t k = 0; k < nslots; k++) slots[k].state = FREE_CLEAN;
        }
        for (uint32_t k = 0; k < nslots && !pending.empty(); k++) {
          if (slots[k].state != FREE_CLEAN) continue;
          float* res = (float*)srv->dev_alloc(n * 4);
          if (!res) {
            srv->admission_waits++;
            mem_blocked = true;
            break;
          }
          Req* r = pending.front();
          pending.pop_front();
          r->t_admit = now_ns();
          slots[k].r = r;
          slots[k].res = res;
          slots[k].t = 0;
          slots[k].state = ACTIVE;
          joins.push_back(k);
        }
      }
      if (!ok) continue;
      if (joins.empty() && act == 0) {
        reap(true);
        while (!markers.empty()) retire_marker();
        if (mem_blocked) std::this_thread::sleep_for(std::chrono::microseconds(100));  // others hold the memory
        else if (!wait_pending(false)) break;
        continue;
      }
      if (!joins.empty()) {
        if (act) srv->ppr_joins_running += joins.size();
        srv->ppr_joins += joins.size();
        for (uint32_t k : joins)
          if (ops->ppr_join(view, ca, k, stored(slots[k].r->source), st) != cudaSuccess) ok = false;
      }
      act = active_mask();
      srv->bump_max(srv->ppr_max_active, (uint64_t)__builtin_popcount(act));
      PprArgs a;
      memset(&a, 0, sizeof(a));
      a.cin = ca;
      a.cout = cb;
      a.part = part;
      a.active = act;
      a.result_perm = g->inv_perm;  // results indexed by original ID
      a.hot = hot;
      std::vector<uint32_t> retiring;
      bool was_dirty[PPR_K];
      for (uint32_t k = 0; k < PPR_K; k++) {
        was_dirty[k] = k < nslots && slots[k].state == FREE_DIRTY;
        if (k < nslots && slots[k].state == ACTIVE) {
          a.src[k] = stored(slots[k].r->source);
          a.damp[k] = slots[k].r->damping;
          a.result[k] = slots[k].res;
          if (slots[k].t + 1 == slots[k].r->iters) {
            a.last |= 1u << k;
            retiring.push_back(k);
          }
        }
      }
      cudaEvent_t ts = get_timed(), te = get_timed();
      cudaEventRecord(ts, st);
      if (ops->ppr_pull(view, a, st) != cudaSuccess || ppr_finish_multi(view, a, st) != cudaSuccess) ok = false;
      cudaEventRecord(te, st);
      markers.push_back({ts, te});
      std::swap(ca, cb);
      srv->ppr_iterations++;
      for (uint32_t k = 0; k < nslots; k++) {
        if (slots[k].state == ACTIVE) slots[k].t++;
        else if (was_dirty[k]) slots[k].state = FREE_CLEAN;  // its column was just written as zero
      }
      if (!retiring.empty()) {
        Inflight f;
        for (uint32_t k : retiring) {
          Req* r = slots[k].r;
          r->host = srv->host_alloc_wait(n * 4);
          r->bytes = n * 4;
          r->count = n;
          r->status = r->host ? LG_OK : LG_ENOMEM;
          if (r->host && cudaMemcpyAsync(r->host, slots[k].res, n * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            ok = false;
          f.done.push_back({r, slots[k].res});
          slots[k] = Slot{};
          slots[k].state = FREE_DIRTY;
        }
        f.ev = get_event();
        cudaEventRecord(f.ev, st);
        inflight.push_back(std::move(f));
      }
      // keep at most two sweeps queued ahead of the device, so that a new
      // request joins within about two sweeps of its arrival
      while (markers.size() > 2) retire_marker();
      reap(false);
      if (!ok) {
        reap(true);
        for (auto& s : slots)
          if (s.r) {
            srv->dev_free(s.res);
            fail_all(s.r);
            s = Slot{};
          }
      }
    }
    reap(true);
    while (!markers.empty()) retire_marker();
  }
};

// ------------------------------------------------------------------ neighborhoods
struct NbrEngine : Engine {
  NbrEngine(lg_server* s, uint32_t i) : Engine(s, i) {}
  lg_status setup() override {
    cudaError_t e = make_stream(0);
    if (e != cudaSuccess) {
      set_error_message(cudaGetErrorString(e));
      return LG_ECUDA;
    }
    return make_timers();
  }
  void teardown() override {
    destroy_timers();
    if (st) cudaStreamDestroy(st);
  }

  void run_batch(std::vector<Req*>& batch) {
    uint64_t k = 0;
    for (Req* r : batch) k += r->vertices.size();
    const uint64_t tmpw = scan_tmp_words(k);
    char* d = (char*)srv->dev_alloc(k * 4 + (k + 1) * 8 + tmpw * 8 + 64);
    uint32_t* hv = (uint32_t*)srv->host_alloc_wait(k * 4 + (k + 1) * 8 + 64);
    if (!d || !hv) {
      srv->dev_free(d);
      srv->host_free(hv);
      for (Req* r : batch) {
        r->status = LG_ENOMEM;
        srv->post(r);
      }
      return;
    }
    uint32_t* dv = (uint32_t*)d;
    uint64_t* doff = (uint64_t*)(d + ((k * 4 + 7) / 8) * 8);
    uint64_t* dtmp = doff + k + 1;
    int* derr = (int*)(dtmp + tmpw);
    uint64_t o = 0;
    for (Req* r : batch) {
      memcpy(hv + o, r->vertices.data(), r->vertices.size() * 4);
      o += r->vertices.size();
    }
    uint64_t* hoff = (uint64_t*)((char*)hv + ((k * 4 + 7) / 8) * 8);
    NbrArgs a;
    memset(&a, 0, sizeof(a));
    a.vertices = dv;
    a.k = k;
    a.out_offsets = doff;
    a.err = derr;
    char* dids = nullptr;
    uint32_t* hids = nullptr;
    uint64_t total = 0;
    bool good = cudaMemcpyAsync(dv, hv, k * 4, cudaMemcpyHostToDevice, st) == cudaSuccess &&
                cudaMemsetAsync(derr, 0, 4, st) == cudaSuccess && cudaEventRecord(t0, st) == cudaSuccess &&
                ops->nbr_degrees(view, a, st) == cudaSuccess &&
                scan_excl_u64(doff, k, doff, dtmp, st) == cudaSuccess &&
                cudaMemcpyAsync(hoff, doff, (k + 1) * 8, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
                cudaStreamSynchronize(st) == cudaSuccess;
    if (good) {
      total = hoff[k];
      uint64_t arena_size;
      {
        std::lock_guard<std::mutex> l(srv->mem_mu);
        arena_size = srv->dev_arena.size();
      }
      for (;;) {  // output of the whole batch (admission by memory)
        if (total * 4 + 16 > arena_size) break;  // can never fit: the batch fails with LG_ENOMEM
        dids = (char*)srv->dev_alloc(total * 4 + 16);
        if (dids || srv->stop.load()) break;
        srv->admission_waits++;
        std::this_thread::sleep_for(std::chrono::microseconds(100));
      }
      hids = dids ? (uint32_t*)srv->host_alloc_wait(total * 4 + 16) : nullptr;
      if (!dids || !hids) {
        srv->dev_free(dids);
        srv->dev_free(d);
        srv->host_free(hids);
        srv->host_free(hv);
        for (Req* r : batch) {
          r->status = LG_ENOMEM;
          srv->post(r);
        }
        return;
      }
      good = true;
      if (good) {
        a.out_ids = (uint32_t*)dids;
        good = ops->nbr_decode(view, a, st) == cudaSuccess &&
               (!g->relabel || segmented_sort(a.out_ids, nullptr, doff, k, total, g->max_degree, st) == cudaSuccess) &&
               cudaEventRecord(t1, st) == cudaSuccess &&
               cudaMemcpyAsync(hids, dids, total * 4, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
               cudaStreamSynchronize(st) == cudaSuccess;
        if (good) add_elapsed(t0, t1);  // degrees + scan + offsets copy + decode
      }
    }
    if (!good) ok = false;
    // one result per request: [u64 offsets (count+1), from 0][u32 ids]
    o = 0;
    for (Req* r : batch) {
      const uint64_t c = r->vertices.size();
      if (!good) {
        r->status = LG_ECUDA;
      } else {
        const uint64_t b0 = hoff[o], b1 = hoff[o + c];
        const uint64_t bytes = (c + 1) * 8 + (b1 - b0) * 4;
        r->host = srv->host_alloc_wait(bytes);
        if (r->host) {
          uint64_t* ro = (uint64_t*)r->host;
          for (uint64_t i = 0; i <= c; i++) ro[i] = hoff[o + i] - b0;
          memcpy(ro + c + 1, hids + b0, (b1 - b0) * 4);
          r->bytes = bytes;
          r->count = c;
        } else {
          r->status = LG_ENOMEM;
        }
      }
      o += c;
      srv->post(r);
    }
    srv->dev_free(dids);
    srv->dev_free(d);
    srv->host_free(hids);
    srv->host_free(hv);
  }

  void loop() override {
    const uint64_t cap = srv->opts.nbr_batch_vertices ? srv->opts.nbr_batch_vertices : (1u << 20);
    while (!srv->stop.load()) {
      std::vector<Req*> batch;
      {
        std::unique_lock<std::mutex> l(mu);
        cv.wait_for(l, std::chrono::milliseconds(50), [&] { return srv->stop.load() || !pending.empty(); });
        uint64_t k = 0;
        while (!pending.empty() && (batch.empty() || k + pending.front()->vertices.size() <= cap)) {
          k += pending.front()->vertices.size();
          pending.front()->t_admit = now_ns();
          batch.push_back(pending.front());
          pending.pop_front();
        }
      }
      if (batch.empty()) continue;
      if (!ok) {
        for (Req* r : batch) fail_all(r);
        continue;
      }
      srv->nbr_batches++;
      srv->bump_max(srv->nbr_max_batch, batch.size());
      run_batch(batch);
    }
  }
};

lg_status submit_impl(lg_server* s, const lg_request* q, uint64_t t_submit, uint64_t* ticket) {
  if (q->graph >= s->graphs.size()) {
    set_error_message("lg_server_submit: graph index out of range");
    return LG_EINVAL;
  }
  const lg_graph* g = s->graphs[q->graph];
  Req* r = new Req;
  r->kind = q->kind;
  r->graph = q->graph;
  r->user = q->user;
  r->source = q->source;
  r->iters = q->iters ? q->iters : (s->opts.ppr_iters ? s->opts.ppr_iters : 10);
  r->damping = q->damping > 0.0f ? q->damping : 0.85f;
  if (q->kind == LG_REQ_NEIGHBORS) {
    if (q->count == 0 || q->count > (1u << 20) || !q->vertices) {
      delete r;
      set_error_message("lg_server_submit: a lookup needs 1 .. 2^20 vertices");
      return LG_EINVAL;
    }
    r->vertices.assign(q->vertices, q->vertices + q->count);
    for (uint32_t v : r->vertices)
      if (v >= g->n) {
        delete r;
        set_error_message("lg_server_submit: lookup vertex >= n");
        return LG_EINVAL;
      }
  } else if (q->kind == LG_REQ_BFS || q->kind == LG_REQ_PPR) {
    if (q->source >= g->n) {
      delete r;
      set_error_message("lg_server_submit: source >= n");
      return LG_EINVAL;
    }
    if (!(r->damping > 0.0f && r->damping <= 1.0f)) {
      delete r;
      set_error_message("lg_server_submit: damping must be in (0, 1]");
      return LG_EINVAL;
    }
  } else {
    delete r;
    set_error_message("lg_server_submit: unknown request kind");
    return LG_EINVAL;
  }
  {
    // device state of one request must fit the arena, else it could never be admitted
    const uint64_t need = q->kind == LG_REQ_NEIGHBORS ? (uint64_t)q->count * 12 + 64 : g->n * 4;
    std::lock_guard<std::mutex> l(s->mem_mu);
    if (need > s->dev_arena.size() || (q->kind != LG_REQ_NEIGHBORS && g->n * 4 > s->host_arena.size())) {
      delete r;
      set_error_message("lg_server_submit: the request's memory exceeds the server's arenas");
      return LG_ENOMEM;
    }
  }
  r->ticket = s->next_ticket++;
  r->t_submit = t_submit;
  if (ticket) *ticket = r->ticket;
  s->submitted++;
  s->by_kind[q->kind]++;
  const uint32_t e = q->graph * 3 + (q->kind == LG_REQ_BFS ? 0 : q->kind == LG_REQ_PPR ? 1 : 2);
  s->engines[e]->push(r);
  return LG_OK;
}

void fill_result(const Req* r, lg_result* o) {
  o->ticket = r->ticket;
  o->user = r->user;
  o->kind = r->kind;
  o->graph = r->graph;
  o->status = r->status;
  o->data = r->host;
  o->bytes = r->bytes;
  o->count = r->count;
  o->t_submit_ns = r->t_submit;
  o->t_admit_ns = r->t_admit;
  o->t_done_ns = r->t_done;
}

}  // namespace

extern "C" void lg_server_destroy(lg_server* s) {
  if (!s) return;
  s->stop = true;
  for (auto& e : s->engines) e->cv.notify_all();
  for (auto& e : s->engines)
    if (e->th.joinable()) e->th.join();
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != s->device) cudaSetDevice(s->device);
  for (auto& e : s->engines) {
    for (Req* r : e->pending) delete r;
    e->teardown();
  }
  s->engines.clear();
  for (Req* r : s->done) delete r;
  for (auto& kv : s->delivered) delete kv.second;
  cudaFree(s->dev_base);
  cudaFreeHost(s->host_base);
  if (prev != s->device) cudaSetDevice(prev);
  delete s;
}

extern "C" lg_status lg_server_create(const lg_graph* const* graphs, uint32_t count, const lg_server_opts* opts,
                                      lg_server** out) {
  set_error_message("");
  if (!out || !graphs || count == 0) {
    set_error_message("lg_server_create: null argument or no graphs");
    return LG_EINVAL;
  }
  *out = nullptr;
  lg_server* s = new lg_server;
  cudaGetDevice(&s->device);
  if (opts) s->opts = *opts;
  for (uint32_t i = 0; i < count; i++) {
    if (!graphs[i] || graphs[i]->device != s->device) {
      delete s;
      set_error_message("lg_server_create: every graph must live on the current device");
      return LG_EINVAL;
    }
    s->graphs.push_back(graphs[i]);
  }
  s->perms.resize(count);
  for (uint32_t i = 0; i < count; i++) {
    if (!graphs[i]->perm) continue;
    s->perms[i].resize(graphs[i]->n);
    if (cudaMemcpy(s->perms[i].data(), graphs[i]->perm, graphs[i]->n * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
      delete s;
      set_error_message("lg_server_create: reading a permutation failed");
      return LG_ECUDA;
    }
  }
  const uint64_t dev_bytes = s->opts.device_bytes ? s->opts.device_bytes : (16ull << 30);
  const uint64_t host_bytes = s->opts.host_bytes ? s->opts.host_bytes : (4ull << 30);
  cudaError_t e = cudaMalloc((void**)&s->dev_base, dev_bytes);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&s->host_base, host_bytes, cudaHostAllocDefault);
  if (e != cudaSuccess) {
    set_error_message("lg_server_create: arena allocation failed");
    cudaFree(s->dev_base);
    delete s;
    return LG_ENOMEM;
  }
  s->dev_arena.init(dev_bytes, 256);
  s->host_arena.init(host_bytes, 256);
  for (uint32_t i = 0; i < count; i++) {
    s->engines.emplace_back(new BfsEngine(s, i));
    s->engines.emplace_back(new PprEngine(s, i));
    s->engines.emplace_back(new NbrEngine(s, i));
  }
  for (auto& eng : s->engines) {
    const lg_status st = eng->setup();
    if (st != LG_OK) {
      lg_server_destroy(s);
      return st;
    }
  }
  for (auto& eng : s->engines) eng->start();
  *out = s;
  return LG_OK;
}

extern "C" lg_status lg_server_submit(lg_server* s, const lg_request* req, uint64_t* ticket) {
  set_error_message("");
  if (!s || !req) {
    set_error_message("lg_server_submit: null argument");
    return LG_EINVAL;
  }
  return submit_impl(s, req, now_ns(), ticket);
}

extern "C" lg_status lg_server_wait(lg_server* s, lg_result* out, uint32_t max, uint32_t* got, uint32_t timeout_us) {
  set_error_message("");
  if (!s || !got || (max && !out)) {
    set_error_message("lg_server_wait: null argument");
    return LG_EINVAL;
  }
  *got = 0;
  std::unique_lock<std::mutex> l(s->done_mu);
  s->done_cv.wait_for(l, std::chrono::microseconds(timeout_us), [&] { return !s->done.empty(); });
  while (*got < max && !s->done.empty()) {
    Req* r = s->done.front();
    s->done.pop_front();
    s->delivered[r->ticket] = r;
    fill_result(r, out + *got);
    (*got)++;
  }
  return LG_OK;
}

extern "C" lg_status lg_server_release(lg_server* s, uint64_t ticket) {
  set_error_message("");
  if (!s) {
    set_error_message("lg_server_release: null argument");
    return LG_EINVAL;
  }
  Req* r = nullptr;
  {
    std::lock_guard<std::mutex> l(s->done_mu);
    auto it = s->delivered.find(ticket);
    if (it == s->delivered.end()) {
      set_error_message("lg_server_release: unknown or already released ticket");
      return LG_EINVAL;
    }
    r = it->second;
    s->delivered.erase(it);
  }
  s->host_free(r->host);
  delete r;
  return LG_OK;
}

extern "C" lg_status lg_server_stats_get(lg_server* s, lg_server_stats* o) {
  if (!s || !o) {
    set_error_message("lg_server_stats_get: null argument");
    return LG_EINVAL;
  }
  memset(o, 0, sizeof(*o));
  o->submitted = s->submitted;
  o->completed = s->completed;
  o->failed = s->failed;
  for (int k = 0; k < 3; k++) o->by_kind[k] = s->by_kind[k];
  o->bfs_levels = s->bfs_levels;
  o->bfs_joins = s->bfs_joins;
  o->bfs_joins_running = s->bfs_joins_running;
  o->bfs_max_active = s->bfs_max_active;
  o->ppr_iterations = s->ppr_iterations;
  o->ppr_joins = s->ppr_joins;
  o->ppr_joins_running = s->ppr_joins_running;
  o->ppr_max_active = s->ppr_max_active;
  o->nbr_batches = s->nbr_batches;
  o->nbr_max_batch = s->nbr_max_batch;
  o->admission_waits = s->admission_waits;
  std::lock_guard<std::mutex> l(s->mem_mu);
  o->device_bytes = s->dev_arena.size();
  o->device_used = s->dev_arena.used();
  o->device_peak = s->dev_arena.peak();
  o->host_bytes = s->host_arena.size();
  o->host_used = s->host_arena.used();
  o->host_peak = s->host_arena.peak();
  return LG_OK;
}

extern "C" lg_status lg_server_replay(lg_server* s, uint64_t n, const uint32_t* kind, const uint32_t* graph,
                                      const uint32_t* source, const uint64_t* nbr_off, const uint32_t* nbr_vertices,
                                      const uint64_t* arrival_ns, void* const* keep, uint64_t* latency_ns,
                                      lg_replay_stats* out) {
  set_error_message("");
  if (!s || !kind || !graph || !source || !nbr_off || !arrival_ns || !latency_ns || (n && !nbr_vertices && nbr_off[n])) {
    set_error_message("lg_server_replay: null argument");
    return LG_EINVAL;
  }
  // validate everything before the clock starts
  for (uint64_t i = 0; i < n; i++) {
    if (graph[i] >= s->graphs.size() || kind[i] > 2 || nbr_off[i + 1] < nbr_off[i]) {
      set_error_message("lg_server_replay: bad request");
      return LG_EINVAL;
    }
    const uint64_t nv = s->graphs[graph[i]]->n;
    if (kind[i] == LG_REQ_NEIGHBORS) {
      if (nbr_off[i + 1] == nbr_off[i] || nbr_off[i + 1] - nbr_off[i] > (1u << 20)) {
        set_error_message("lg_server_replay: a lookup needs 1 .. 2^20 vertices");
        return LG_EINVAL;
      }
      for (uint64_t j = nbr_off[i]; j < nbr_off[i + 1]; j++)
        if (nbr_vertices[j] >= nv) {
          set_error_message("lg_server_replay: lookup vertex >= n");
          return LG_EINVAL;
        }
    } else if (source[i] >= nv) {
      set_error_message("lg_server_replay: source >= n");
      return LG_EINVAL;
    }
  }
  const uint64_t t0 = now_ns() + 1000000;  // first arrival 1 ms from now
  std::atomic<uint64_t> submitted{0};
  std::atomic<int> sub_err{0};
  std::thread submitter([&] {
    for (uint64_t i = 0; i < n; i++) {
      const uint64_t at = t0 + arrival_ns[i];
      for (;;) {
        const uint64_t t = now_ns();
        if (t >= at) break;
        if (at - t > 200000) std::this_thread::sleep_for(std::chrono::nanoseconds(at - t - 100000));
        else std::this_thread::yield();
      }
      lg_request q;
      memset(&q, 0, sizeof(q));
      q.kind = kind[i];
      q.graph = graph[i];
      q.source = source[i];
      q.count = (uint32_t)(nbr_off[i + 1] - nbr_off[i]);
      q.vertices = nbr_vertices ? nbr_vertices + nbr_off[i] : nullptr;
      q.user = i;
      if (submit_impl(s, &q, now_ns(), nullptr) != LG_OK) sub_err = 1;
      submitted++;
    }
  });
  uint64_t got_all = 0, failed = 0, t_last = t0;
  std::vector<lg_result> buf(256);
  while (got_all < n) {
    uint32_t got = 0;
    lg_server_wait(s, buf.data(), (uint32_t)buf.size(), &got, 20000);
    if (got == 0 && sub_err.load() && submitted.load() == n) break;
    for (uint32_t j = 0; j < got; j++) {
      const lg_result& r = buf[j];
      const uint64_t i = r.user;
      if (i < n) {
        latency_ns[i] = r.t_done_ns - (t0 + arrival_ns[i]);
        if (keep && keep[i] && r.data) memcpy(keep[i], r.data, r.bytes);
      }
      if (r.status != LG_OK) failed++;
      t_last = std::max(t_last, r.t_done_ns);
      lg_server_release(s, r.ticket);
      got_all++;
    }
  }
  submitter.join();
  if (out) {
    memset(out, 0, sizeof(*out));
    out->completed = got_all;
    out->failed = failed;
    out->makespan_ns = t_last - t0;
  }
  if (sub_err.load()) {
    set_error_message("lg_server_replay: a submit failed");
    return LG_EINVAL;
  }
  return failed ? LG_ECUDA : LG_OK;
}

extern "C" lg_status lg_server_engine_time(lg_server* s, uint32_t graph, uint32_t kind, uint64_t* ops,
                                           uint64_t* gpu_ns) {
  set_error_message("");
  if (!s || !ops || !gpu_ns || graph >= s->graphs.size() || kind > 2) {
    set_error_message("lg_server_engine_time: bad argument");
    return LG_EINVAL;
  }
  const uint32_t e = graph * 3 + (kind == LG_REQ_BFS ? 0 : kind == LG_REQ_PPR ? 1 : 2);
  *ops = s->engines[e]->ops_done.load();
  *gpu_ns = s->engines[e]->gpu_ns.load();
  return LG_OK;
}
