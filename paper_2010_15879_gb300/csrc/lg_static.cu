// lg_pagerank_noalloc: PageRank that allocates no device memory.
//
// Some callers cannot call cudaMalloc / cudaFree: a process whose device memory
// is owned by another allocator or pre-reserved under a fixed budget (extra
// allocations fail or fragment it), or a latency-sensitive loop that must not
// hit cudaFree's implicit device synchronization.  For them this entry point
// runs the same PageRank kernels as lg_pagerank with its scratch (two FP32
// contribution arrays and the partial sums of split vertices) in the
// file-scope array below.  The array is part of the module image, so every
// GPU that loads the library holds it until the process exits.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "lg_internal.h"

namespace {

constexpr uint64_t kMaxVertices = 1ull << 20;  // graphs up to 1,048,576 vertices
constexpr uint64_t kMaxItems = 1ull << 18;     // heavy-schedule items with partial sums
constexpr uint64_t kScratchFloats = 2 * kMaxVertices + kMaxItems;  // 9 MiB

__device__ __align__(256) float g_pr_scratch[kScratchFloats];

// Host code must not use g_pr_scratch's name as an address: its device address
// is looked up once per device (with that device current) and cached here.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
float* g_dev_ptr[kMaxDevices] = {};

}  // namespace

// The first call on each device looks up the scratch array's device address
// (cudaGetSymbolAddress, with that device current) and caches it; make that
// first call before any stream capture.
static cudaError_t scratch_on_device(int dev, float** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_pr_scratch);
    if (e != cudaSuccess) return e;
    g_dev_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_dev_ptr[dev];
  return cudaSuccess;
}

extern "C" lg_status lg_pagerank_noalloc(const lg_graph* g, float damping, uint32_t iters,
                                         const uint32_t* personalize_source, float* ranks, void* stream) {
  using namespace lg;
  char g_msg[512];
  set_error_message("");
  if (!g || !ranks) {
    set_error_message("lg_pagerank_noalloc: null argument");
    return LG_EINVAL;
  }
  if (!(damping >= 0.0f && damping <= 1.0f)) {
    set_error_message("lg_pagerank_noalloc: damping must be in [0, 1]");
    return LG_EINVAL;
  }
  if (g->n > kMaxVertices || (g->n_multi && g->n_items > kMaxItems)) {
    snprintf(g_msg, sizeof g_msg,
             "lg_pagerank_noalloc: graph has %llu vertices and %llu split schedule items; the fixed scratch "
             "holds at most %llu vertices and %llu items (use lg_pagerank)",
             (unsigned long long)g->n, (unsigned long long)(g->n_multi ? g->n_items : 0),
             (unsigned long long)kMaxVertices, (unsigned long long)kMaxItems);
    set_error_message(g_msg);
    return LG_ERANGE;
  }
  int64_t personal = -1;
  if (personalize_source) {
    if (*personalize_source >= g->n) {
      set_error_message("lg_pagerank_noalloc: personalize_source >= n");
      return LG_EINVAL;
    }
    personal = *personalize_source;
  }
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) {
    set_error_message("lg_pagerank_noalloc: no CUDA device");
    return LG_ECUDA;
  }
  if (prev != g->device) cudaSetDevice(g->device);
  lg_status status = LG_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  float* scratch = nullptr;
  cudaError_t e = cudaSuccess;
  if (iters == 0) {
    // PageRank after zero iterations is r_0 itself: no scratch is needed
    e = pr_fill0(ranks, g->n, personal, st);
    if (e != cudaSuccess) {
      snprintf(g_msg, sizeof g_msg, "lg_pagerank_noalloc: %s", cudaGetErrorString(e));
      set_error_message(g_msg);
      status = LG_ECUDA;
    }
    if (prev != g->device) cudaSetDevice(prev);
    return status;
  }
  e = scratch_on_device(g->device, &scratch);
  if (e != cudaSuccess) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const bool capturing = cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
    snprintf(g_msg, sizeof g_msg,
             "lg_pagerank_noalloc: looking up the scratch array on device %d failed (%s)%s", g->device,
             cudaGetErrorString(e),
             capturing ? "; the first call on a device must come before any stream capture" : "");
    set_error_message(g_msg);
    if (prev != g->device) cudaSetDevice(prev);
    return LG_ECUDA;
  }
  if (personal >= 0 && g->perm) {
    uint32_t ps = 0;
    e = cudaMemcpyAsync(&ps, g->perm + personal, sizeof(ps), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    personal = ps;
  }
  if (e == cudaSuccess) {
    // scratch layout: contributions A [n], contributions B [n], item partial sums;
    // every element is written before it is read, so nothing needs clearing
    float* ca = scratch;
    float* cb = scratch + kMaxVertices;
    float* part = scratch + 2 * kMaxVertices;
    const GView v = make_view(g);
    const TravOps* ops = trav_ops((int)g->id_mode, (int)g->off_mode);
    PrArgs a;
    memset(&a, 0, sizeof(a));
    a.damp = damping;
    a.personal = personal;
    a.base_all = personal < 0 ? (1.0f - damping) / (float)g->n : (1.0f - damping);
    a.r0_all = 1.0f / (float)g->n;
    a.part = part;
    a.hot = hot_rows(g, sizeof(float));
    a.ranks_out = ranks;
    a.contrib_out = ca;
    e = ops->pr_init(v, a, st);
    float* cur = ca;
    float* nxt = cb;
    for (uint32_t t = 0; t < iters && e == cudaSuccess; t++) {
      a.contrib_in = cur;
      a.contrib_out = nxt;
      a.last = (t + 1 == iters);
      e = ops->pr_pull(v, a, st);
      if (e == cudaSuccess) e = pr_finish_multi(v, a, st);
      float* tt = cur; cur = nxt; nxt = tt;
    }
  }
  if (e != cudaSuccess) {
    snprintf(g_msg, sizeof g_msg, "lg_pagerank_noalloc: %s", cudaGetErrorString(e));
    set_error_message(g_msg);
    status = LG_ECUDA;
  }
  if (prev != g->device) cudaSetDevice(prev);
  return status;
}
