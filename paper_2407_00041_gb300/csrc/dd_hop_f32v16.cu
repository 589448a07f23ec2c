// Instantiation of the fused stencil for (links/clover, input, output) = (P32, P16, P16):
// FP32 links and self coupling on FP16 vectors (the CG vectors of DD_PRECOND_CGNR16
// inside an FP32-inner solve).
#include "dd_hop.cuh"
namespace dd {
DD_INSTANTIATE_HOP(P32, P16, P16)
DD_INSTANTIATE_HOP_NORM(P32, P16, P16)
}  // namespace dd
