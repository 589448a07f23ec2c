// Two-level AMG preconditioner (dd_amg.cu): the parts the solver uses.
#pragma once

#include "dd_internal.h"

namespace dd {

// z = M^{-1} v (coarse-grid correction, then SAP post-smoothing): full
// native fields of the handle's fine precision with the same RHS count.
int amg_apply(dd_amg* A, const Field& v, const Field& z, cudaStream_t st);
int amg_fine_precision(const dd_amg* A);
int amg_operator_precision(const dd_amg* A);
const dd_clover* amg_operator(const dd_amg* A);

}  // namespace dd
