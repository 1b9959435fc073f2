// Kernel instantiations for ID_GLOBAL (packed and Elias-Fano offsets).
#include "lg_traverse.cuh"

namespace lg {
const TravOps* trav_ops_global_packed() { return make_ops<ID_GLOBAL, OFF_PACKED>(); }
const TravOps* trav_ops_global_ef() { return make_ops<ID_GLOBAL, OFF_EF>(); }
}  // namespace lg
