// Instantiation of the paired-RHS stencil for FP16-stored vectors, links and blocks.
#include "dd_hop_pair.cuh"
namespace dd {
DD_INSTANTIATE_HOP_PAIR(P16, P16)
}  // namespace dd
