// Instantiation of the fused stencil for (links/clover, input, output) = (P16, P16, P16).
#include "dd_hop.cuh"
namespace dd {
DD_INSTANTIATE_HOP(P16, P16, P16)
DD_INSTANTIATE_HOP_NORM(P16, P16, P16)
}  // namespace dd
