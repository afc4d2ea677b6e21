// Instantiations: Taylor--Hood Stokes, 3D.
#include "op_launch.cuh"
namespace mfns {
MFNS_INSTANTIATE_OP(3, 2, OP_STOKES)
MFNS_INSTANTIATE_OP(3, 3, OP_STOKES)
MFNS_INSTANTIATE_OP(3, 4, OP_STOKES)
}  // namespace mfns
