// Instantiation of the fused stencil for (links/clover, input, output) = (P64, P64, P64).
#include "dd_hop.cuh"
namespace dd {
DD_INSTANTIATE_HOP(P64, P64, P64)
}  // namespace dd
