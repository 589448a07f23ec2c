// Domain-decomposed stencil kernels, F32 links and fields.
#include "dd_decomp.cuh"

namespace dd {
DD_INSTANTIATE_DECOMP(P32, P32, P32)
}  // namespace dd
