// Instantiations: stabilised Navier--Stokes, 3D.
#include "op_launch.cuh"
namespace mfns {
MFNS_INSTANTIATE_OP(3, 1, OP_STAB_NS)
MFNS_INSTANTIATE_OP(3, 2, OP_STAB_NS)
MFNS_INSTANTIATE_OP(3, 3, OP_STAB_NS)
}  // namespace mfns
