// Instantiation of the fused stencil for (links/clover, input, output) = (P32, P32, P32).
#include "dd_hop.cuh"
namespace dd {
DD_INSTANTIATE_HOP(P32, P32, P32)
DD_INSTANTIATE_HOP_NORM(P32, P32, P32)
}  // namespace dd
