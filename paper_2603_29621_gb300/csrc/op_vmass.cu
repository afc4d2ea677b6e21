// Instantiations: velocity mass of the Taylor--Hood velocity space, 2D and 3D.
#include "op_launch.cuh"
namespace mfns {
MFNS_INSTANTIATE_OP(2, 2, OP_VMASS)
MFNS_INSTANTIATE_OP(2, 3, OP_VMASS)
MFNS_INSTANTIATE_OP(2, 4, OP_VMASS)
MFNS_INSTANTIATE_OP(3, 2, OP_VMASS)
MFNS_INSTANTIATE_OP(3, 3, OP_VMASS)
MFNS_INSTANTIATE_OP(3, 4, OP_VMASS)
}  // namespace mfns
