// Batched uneven-lattice apply (placeholder until the persistent kernel lands).
#include "dd_internal.h"

extern "C" {
int dd_batch_create(dd_clover* const*, int, int, const int*, dd_batch**) {
  return dd::fail(DD_ERR_UNSUPPORTED, "batched apply is not built yet");
}
int dd_batch_destroy(dd_batch*) { return DD_OK; }
int dd_apply_batched(dd_batch*, const void* const*, void* const*, void*) {
  return dd::fail(DD_ERR_UNSUPPORTED, "batched apply is not built yet");
}
int dd_batch_tune(dd_batch*, const void* const*, void* const*, void*, int*) {
  return dd::fail(DD_ERR_UNSUPPORTED, "batched apply is not built yet");
}
int dd_apply_batched_graph(dd_batch*, const void* const*, void* const*, void*) {
  return dd::fail(DD_ERR_UNSUPPORTED, "batched apply is not built yet");
}
}
