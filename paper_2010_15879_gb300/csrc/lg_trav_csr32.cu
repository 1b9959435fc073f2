// Kernel instantiations for the uncompressed baseline: 32-bit IDs and 64-bit
// row offsets, run by the same kernels as the compressed modes.
#include "lg_traverse.cuh"

namespace lg {
const TravOps* trav_ops_csr32() { return make_ops<ID_CSR32, OFF_ROWPTR>(); }
}  // namespace lg
