// Vector kernels of the Krylov solver (see dd_blas.cu for the conventions).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dd {

struct VecList {
  const void* p[32];
};

int blas_grid(int64_t L, int block);
// dots[j][r] (+)= <V_j, w>_r for j < J; partials: scratch of
// blas_grid(L, block) * min(J, 8) * N complex doubles.
template <int PV>
int blas_multidot(const VecList& vs, int J, const void* w, int64_t L, int N, double2* dots_dev, int add,
                  double2* partials, cudaStream_t st);
// w += csign * sum_j c[j][r] V_j (J <= 32); with norm_out, also
// norm_out[r].x = |w_r|^2 of the result (partials: scratch as for multidot)
template <int PV>
int blas_multiaxpy(const VecList& vs, int J, const double2* c_dev, double csign, void* w, int64_t L, int N,
                   cudaStream_t st, double2* norm_out = nullptr, double2* partials = nullptr);
// out = c[r] * in
template <int PV>
int blas_scale(const double2* c_dev, const void* in, void* out, int64_t L, int N, cudaStream_t st);
// CG updates with step sizes from device scalars (squared norms in .x), the
// x update deferred into the direction update: r -= (g/n) w;  x += (g/n) p;
// x += (g/n) p and p = z + (gn/g) p in one pass over p.
template <int PV>
int blas_cg_r(void* r, const void* w, const double2* g, const double2* n, int64_t L, int N, cudaStream_t st);
template <int PV>
int blas_cg_x(void* x, const void* p, const double2* g, const double2* n, int64_t L, int N, cudaStream_t st);
template <int PV>
int blas_cg_xp(void* x, void* p, const void* z, const double2* g, const double2* n, const double2* gn, int64_t L,
               int N, cudaStream_t st);
// out[i] (+)= sum over b < nblocks of partials[b * JN + i], i < JN, summed in
// a fixed order (warp shuffles, then the warps in turn).  From 4096 partials
// on, the sum runs in two stages (64 CTAs over contiguous chunks, then one)
// through `scratch`, blas_reduce_scratch(nblocks, JN) complex doubles.
int blas_reduce_partials(const double2* partials, int nblocks, int JN, double2* out, int add, cudaStream_t st,
                         double2* scratch = nullptr);
inline int blas_reduce_scratch(int nblocks, int JN) { return nblocks >= 4096 ? 64 * JN : 0; }
// FP64 native field -> FP32 native field (nhalf half fields, VN = Vh * N)
int blas_demote(const void* in64, void* out32, int64_t nhalf, int64_t VN, cudaStream_t st);
// FP64 native field += FP32 native field
int blas_promote_add(const void* in32, void* out64, int64_t nhalf, int64_t VN, cudaStream_t st);
// out += in over n complex doubles
int blas_add64(const void* in, void* out, int64_t n, cudaStream_t st);

// Largest number of partial sums blas_multidot needs per RHS and vector chunk.
inline int64_t blas_partials_len(int N) { return (int64_t)152 * 8 * 8 * N; }

}  // namespace dd
