// Domain-decomposed stencil kernels, F16 links and fields.
#include "dd_decomp.cuh"

namespace dd {
DD_INSTANTIATE_DECOMP(P16, P16, P16)
}  // namespace dd
