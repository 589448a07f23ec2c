// Arithmetic-throughput probe after Section 3.1 / Table 3.1 of the thesis:
// many threads each run long chains of floating-point operations on
// registers only; operations / time estimates the peak rate.  Eight
// independent fused multiply-add chains per thread keep the pipelines full.
#include "dd_internal.h"

namespace {

template <typename T>
__global__ void k_fma_probe(T* sink, int iters, T b, T c) {
  T a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = (T)(threadIdx.x * 1e-7) + (T)i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = fma(a[i], b, c);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += a[i];
  if (s == (T)-12345.678) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains alive
}

template <typename T>
int probe(int iters, double* out, cudaStream_t st) {
  int dev = 0, sms = 0;
  DD_CUDA(cudaGetDevice(&dev));
  DD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int threads = 256, blocks = sms * 8;
  dd::DevBuf sink;
  DD_TRY(sink.alloc((size_t)threads * blocks * sizeof(T)));
  cudaEvent_t e0, e1;
  DD_CUDA(cudaEventCreate(&e0));
  DD_CUDA(cudaEventCreate(&e1));
  k_fma_probe<T><<<blocks, threads, 0, st>>>((T*)sink.ptr, iters / 4, (T)0.999999, (T)1e-7);  // warm-up
  DD_CUDA(cudaEventRecord(e0, st));
  k_fma_probe<T><<<blocks, threads, 0, st>>>((T*)sink.ptr, iters, (T)0.999999, (T)1e-7);
  DD_CUDA(cudaEventRecord(e1, st));
  DD_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  DD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *out = 2.0 * 8.0 * (double)iters * threads * (double)blocks / (ms * 1e-3);
  return DD_OK;
}

}  // namespace

extern "C" int dd_probe_flops(int prec, double* flops_per_second, void* stream) {
  if (!flops_per_second) return dd::fail(DD_ERR_ARG, "null argument");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (prec == DD_PREC_F64) return probe<double>(1 << 13, flops_per_second, st);
  if (prec == DD_PREC_F32) return probe<float>(1 << 16, flops_per_second, st);
  return dd::fail(DD_ERR_ARG, "probe precision must be F64 or F32");
}
