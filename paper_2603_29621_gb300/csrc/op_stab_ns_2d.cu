// Instantiations: stabilised Navier--Stokes, 2D.
#include "op_launch.cuh"
namespace mfns {
MFNS_INSTANTIATE_OP(2, 1, OP_STAB_NS)
MFNS_INSTANTIATE_OP(2, 2, OP_STAB_NS)
MFNS_INSTANTIATE_OP(2, 3, OP_STAB_NS)
MFNS_INSTANTIATE_OP(2, 4, OP_STAB_NS)
}  // namespace mfns
