// Instantiations: pressure mass, 2D and 3D.
#include "op_launch.cuh"
namespace mfns {
MFNS_INSTANTIATE_OP(2, 1, OP_PMASS)
MFNS_INSTANTIATE_OP(2, 2, OP_PMASS)
MFNS_INSTANTIATE_OP(2, 3, OP_PMASS)
MFNS_INSTANTIATE_OP(3, 1, OP_PMASS)
MFNS_INSTANTIATE_OP(3, 2, OP_PMASS)
MFNS_INSTANTIATE_OP(3, 3, OP_PMASS)
}  // namespace mfns
