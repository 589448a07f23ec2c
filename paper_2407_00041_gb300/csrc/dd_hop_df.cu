// Instantiation of the fused stencil for (links/clover, input, output) = (PDF, PDF, PDF):
// FP64-accurate arithmetic in FP32 pairs.
#include "dd_hop.cuh"
namespace dd {
DD_INSTANTIATE_HOP(PDF, PDF, PDF)
}  // namespace dd
