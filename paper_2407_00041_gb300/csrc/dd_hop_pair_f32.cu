// Instantiation of the paired-RHS stencil for FP32 vectors with FP32 or FP16 links and blocks.
#include "dd_hop_pair.cuh"
namespace dd {
DD_INSTANTIATE_HOP_PAIR(P32, P32)
DD_INSTANTIATE_HOP_PAIR(P16, P32)
}  // namespace dd
