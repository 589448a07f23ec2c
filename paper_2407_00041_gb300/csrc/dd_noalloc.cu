// Allocation-free variant of dd_dot.
//
// Some callers cannot allocate device memory at the time they need an inner
// product: code running inside a memory pool that owns all free device
// memory, callers with a hard cap on allocations, or code in a phase where
// cudaMalloc/cudaFree would synchronise the device and break overlap.
// dd_dot_noalloc serves them: its scratch (the per-block partial sums of the
// two-stage reduction and the per-RHS results) lives in a fixed device array
// defined in this file, so the call allocates nothing.
//
// The array is a file-scope __device__ variable: every GPU that loads this
// library holds it (about 20 KB) until the process exits.  In host code its
// name is only a host-side stand-in, not a device address, so its device
// address is looked up with cudaGetSymbolAddress once per device, with that
// device current, on the first call made on that device.
#include <mutex>

#include "dd_blas.h"
#include "dd_internal.h"

namespace {

// Right-hand sides one call may reduce (the size of the result slots).
constexpr int kMaxRhs = 64;
// Partial sums of one reduction: the vector kernels cap their grid at
// 152 * 8 blocks, one FP64 complex partial per block.
constexpr int kMaxPartials = 152 * 8;

struct NoAllocScratch {
  double2 partials[kMaxPartials];
  double2 results[kMaxRhs];
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_mu;
NoAllocScratch* g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch on the current device (looked up once).
int scratch_address(NoAllocScratch** out) {
  int dev = 0;
  DD_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return dd::fail(DD_ERR_UNSUPPORTED, "device index above 63");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return dd::cuda_fail(e, "cudaGetSymbolAddress of the dd_dot_noalloc scratch");
    g_addr[dev] = reinterpret_cast<NoAllocScratch*>(p);
  }
  *out = g_addr[dev];
  return DD_OK;
}

}  // namespace

extern "C" int dd_dot_noalloc(const double* a, const double* b, int64_t nsites, int nrhs, double* dots_host,
                              void* stream) {
  if (!a || !b || !dots_host || nsites < 1 || nrhs < 1) return dd::fail(DD_ERR_ARG, "null argument or empty field");
  if (nrhs > kMaxRhs)
    return dd::fail(DD_ERR_ARG, "dd_dot_noalloc takes at most 64 right-hand sides per call (fixed scratch size)");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  NoAllocScratch* s = nullptr;
  DD_TRY(scratch_address(&s));
  const int64_t L = nsites * 12;
  for (int r = 0; r < nrhs; ++r) {
    dd::VecList vs;
    vs.p[0] = a + 2 * r * L;
    // every partial the reduction reads is written by the same launch, so
    // nothing in the scratch has to start at zero
    DD_TRY(dd::blas_multidot<dd::P64>(vs, 1, b + 2 * r * L, L, 1, s->results + r, 0, s->partials, st));
  }
  DD_CUDA(cudaMemcpyAsync(dots_host, s->results, (size_t)nrhs * sizeof(double2), cudaMemcpyDeviceToHost, st));
  DD_CUDA(cudaStreamSynchronize(st));
  return DD_OK;
}
