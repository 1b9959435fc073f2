// Kernel instantiations for ID_LOCAL (packed and Elias-Fano offsets).
#include "lg_traverse.cuh"

namespace lg {
const TravOps* trav_ops_local_packed() { return make_ops<ID_LOCAL, OFF_PACKED>(); }
const TravOps* trav_ops_local_ef() { return make_ops<ID_LOCAL, OFF_EF>(); }
}  // namespace lg
