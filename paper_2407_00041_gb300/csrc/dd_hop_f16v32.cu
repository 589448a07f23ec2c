// Instantiation of the fused stencil for (links/clover, input, output) = (P16, P32, P32).
#include "dd_hop.cuh"
namespace dd {
DD_INSTANTIATE_HOP(P16, P32, P32)
DD_INSTANTIATE_HOP_NORM(P16, P32, P32)
}  // namespace dd
