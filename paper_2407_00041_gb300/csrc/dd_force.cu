// Link derivative of L = Re <phi, D psi> (placeholder until the kernel lands).
#include "dd_internal.h"

namespace dd {
int force(dd_clover*, int, const double*, const double*, int, int, double*, double*, cudaStream_t) {
  return fail(DD_ERR_UNSUPPORTED, "dd_force is not built yet");
}
}  // namespace dd
