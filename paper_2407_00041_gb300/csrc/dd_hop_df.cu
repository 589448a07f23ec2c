// Instantiation of the fused stencil for (links/clover, input, output) = (PDF, PDF, PDF)
// and (PDF, P64, P64): FP64-accurate arithmetic in FP32 pairs, on fields of
// FP32 pairs or of FP64 values (the solver's vectors, split on load).
#include "dd_hop.cuh"
namespace dd {
DD_INSTANTIATE_HOP(PDF, PDF, PDF)
DD_INSTANTIATE_HOP(PDF, P64, P64)
}  // namespace dd
