// Instantiations: vector Laplacian (A block), 2D.
#include "op_launch.cuh"
namespace mfns {
MFNS_INSTANTIATE_OP(2, 1, OP_STOKES_A)
MFNS_INSTANTIATE_OP(2, 2, OP_STOKES_A)
MFNS_INSTANTIATE_OP(2, 3, OP_STOKES_A)
MFNS_INSTANTIATE_OP(2, 4, OP_STOKES_A)
}  // namespace mfns
