// Domain-decomposed stencil kernels, F64 links and fields.
#include "dd_decomp.cuh"

namespace dd {
DD_INSTANTIATE_DECOMP(P64, P64, P64)
}  // namespace dd
