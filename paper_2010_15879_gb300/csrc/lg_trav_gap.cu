// Kernel instantiations for ID_LOCAL_GAP (packed and Elias-Fano offsets).
#include "lg_traverse.cuh"

namespace lg {
const TravOps* trav_ops_gap_packed() { return make_ops<ID_LOCAL_GAP, OFF_PACKED>(); }
const TravOps* trav_ops_gap_ef() { return make_ops<ID_LOCAL_GAP, OFF_EF>(); }
}  // namespace lg
