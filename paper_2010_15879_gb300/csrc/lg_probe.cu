// lg_probe_gather: the access pattern of a pull sweep's contribution gathers
// without the decode, so that a pull kernel's speed can be read against the
// rate at which this GPU serves scattered 4-byte reads (Section 7.1.2's
// PageRank reads r[u] / d_u once per arc, at random u).
//
// Thread i reads idx[i] (a coalesced stream, as the compressed neighborhoods
// are) and gathers table[idx[i]] with the same load instruction and L2 policy
// as the pull kernels (evict-last), four gathers in flight per thread; each
// thread writes its sum so the loads are not dead.
#include <cstdio>

#include "lg_internal.h"

namespace {

__global__ void __launch_bounds__(256) k_probe_gather(const uint32_t* __restrict__ idx, uint64_t count,
                                                      const float* __restrict__ table, float* out) {
  const uint64_t pkeep = lg::policy_keep();
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  float s0 = 0.f, s1 = 0.f;
  uint64_t i = t;
  for (; i + 3 * stride < count; i += 4 * stride) {
    const uint32_t u0 = __ldcs(idx + i), u1 = __ldcs(idx + i + stride);
    const uint32_t u2 = __ldcs(idx + i + 2 * stride), u3 = __ldcs(idx + i + 3 * stride);
    const float f0 = lg::ldg_gather(table + u0, pkeep), f1 = lg::ldg_gather(table + u1, pkeep);
    const float f2 = lg::ldg_gather(table + u2, pkeep), f3 = lg::ldg_gather(table + u3, pkeep);
    s0 += f0 + f1;
    s1 += f2 + f3;
  }
  for (; i < count; i += stride) s0 += lg::ldg_gather(table + __ldcs(idx + i), pkeep);
  if (t < count) out[t] = s0 + s1;
}

}  // namespace

extern "C" lg_status lg_probe_gather(const uint32_t* idx, uint64_t count, const float* table, uint64_t table_len,
                                     float* out, void* stream) {
  lg::set_error_message("");
  if (count && (!idx || !table || !out || table_len == 0)) {
    lg::set_error_message("lg_probe_gather: null argument or empty table");
    return LG_EINVAL;
  }
  if (count == 0) return LG_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const unsigned grid = lg::grid_for(count, 256 * 4, 152 * 8);
  k_probe_gather<<<grid, 256, 0, st>>>(idx, count, table, out);
  lg::count_launch();
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    char msg[160];
    snprintf(msg, sizeof msg, "lg_probe_gather: %s", cudaGetErrorString(e));
    lg::set_error_message(msg);
    return LG_ECUDA;
  }
  return LG_OK;
}
