// Vector kernels of the CG preconditioner with FP16-stored vectors
// (DD_PRECOND_CGNR16): the residual r, the direction p, w = A p and
// z' = A^H r are native FP16 fields (8 halves per 16-byte word plus one FP32
// scale per site and RHS), the iterate x stays FP32.  One thread per site
// and RHS: it reads the stored halves with their scale, computes in FP32 and
// writes the halves with a new scale (the site's largest modulus), so every
// update is one pass over its vectors.  Step sizes come from device scalars
// as in the FP32 CG kernels (alpha = g / |w|^2, beta = g' / g; a zero
// denominator gives a zero step).
#include <initializer_list>

#include "dd_blas.h"
#include "dd_internal.h"

namespace dd {

namespace {

struct Two {
  HalfField h[2];
};

// npar = 2: both halves of a full field; npar = 1: the one half a subset
// view holds (the odd half of a subset-1 view sits in h[1])
Two halves(const Field& f, int npar) {
  Two t;
  const HalfField one = f.h[0].base ? f.h[0] : f.h[1];
  t.h[0] = npar == 2 ? f.h[0] : one;
  t.h[1] = npar == 2 ? f.h[1] : one;
  return t;
}

// half-field index of slot i of npar half fields of vn = Vh * N slots
__device__ __forceinline__ int half_of(int64_t& i, int64_t vn) {
  if (i >= vn) {
    i -= vn;
    return 1;
  }
  return 0;
}

__global__ void __launch_bounds__(256) k_to16(Two in32, Two out16, int64_t vn, int npar) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < vn * npar; t += stride) {
    int64_t i = t;
    const int p = half_of(i, vn);
    cx<float> v[12];
    load_spinor<P32, float>(in32.h[p], vn, i, v);
    store_spinor<P16, float>(out16.h[p], vn, i, v);
  }
}

// partials[b * N + r] = sum over the slots of block b with RHS r of |x|^2;
// blockDim and the grid stride are multiples of N, so a thread keeps one RHS
__global__ void __launch_bounds__(256) k_norm16(Two x, int64_t vn, int npar, int N, double2* partials) {
  __shared__ double s[256];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  double acc = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < vn * npar; t += stride) {
    int64_t i = t;
    const int p = half_of(i, vn);
    cx<float> v[12];
    load_spinor<P16, float>(x.h[p], vn, i, v);
    float n2 = 0.f;
#pragma unroll
    for (int c = 0; c < 12; ++c) n2 = __fmaf_rn(v[c].re, v[c].re, __fmaf_rn(v[c].im, v[c].im, n2));
    acc += (double)n2;
  }
  s[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < N) {
    double sum = 0.0;
    for (int j = threadIdx.x; j < (int)blockDim.x; j += N) sum += s[j];  // fixed order
    partials[(int64_t)blockIdx.x * N + threadIdx.x] = make_double2(sum, 0.0);
  }
}

__device__ __forceinline__ float step(const double2* num, const double2* den, int r) {
  const double d = den[r].x;
  return d > 0.0 ? (float)(num[r].x / d) : 0.f;
}

// r -= (g / n) w
__global__ void __launch_bounds__(256) k_cg_r16(Two r16, Two w16, int64_t vn, int npar, int N,
                                                const double2* __restrict__ g, const double2* __restrict__ n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < vn * npar; t += stride) {
    int64_t i = t;
    const int p = half_of(i, vn);
    const float a = step(g, n, (int)(i % N));
    cx<float> rv[12], wv[12];
    load_spinor<P16, float>(r16.h[p], vn, i, rv);
    load_spinor<P16, float>(w16.h[p], vn, i, wv);
#pragma unroll
    for (int c = 0; c < 12; ++c) rv[c] = caxpy(-a, wv[c], rv[c]);
    store_spinor<P16, float>(r16.h[p], vn, i, rv);
  }
}

// x += (g / n) p, and with z: p = z + (gn / g) p
template <bool DIR>
__global__ void __launch_bounds__(256) k_cg_xp16(Two x32, Two p16, Two z16, int64_t vn, int npar, int N,
                                                 const double2* __restrict__ g, const double2* __restrict__ n,
                                                 const double2* __restrict__ gn) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < vn * npar; t += stride) {
    int64_t i = t;
    const int p = half_of(i, vn);
    const int r = (int)(i % N);
    const float a = step(g, n, r);
    cx<float> xv[12], pv[12];
    load_spinor<P32, float>(x32.h[p], vn, i, xv);
    load_spinor<P16, float>(p16.h[p], vn, i, pv);
#pragma unroll
    for (int c = 0; c < 12; ++c) xv[c] = caxpy(a, pv[c], xv[c]);
    store_spinor<P32, float>(x32.h[p], vn, i, xv);
    if constexpr (DIR) {
      const float b = step(gn, g, r);
      cx<float> zv[12];
      load_spinor<P16, float>(z16.h[p], vn, i, zv);
#pragma unroll
      for (int c = 0; c < 12; ++c) zv[c] = caxpy(b, pv[c], zv[c]);
      store_spinor<P16, float>(p16.h[p], vn, i, zv);
    }
  }
}

int grid_for(int64_t slots, int block) {
  const int64_t want = (slots + block - 1) / block;
  const int64_t cap = 152 * 8;
  return (int)(want < 1 ? 1 : want < cap ? want : cap);
}

int block_of(int N) { return N <= 256 ? (256 / N) * N : -1; }

}  // namespace

// npar (1: the odd half, 2: a full field) half fields of Vh * N slots
static bool views_ok(std::initializer_list<const Field*> fs, int npar) {
  for (const Field* f : fs) {
    const Two t = halves(*f, npar);
    if (!t.h[0].base || !t.h[1].base) return false;
  }
  return true;
}

int cg16_convert(const Field& in32, const Field& out16, int64_t Vh, int npar, cudaStream_t st) {
  if (!views_ok({&in32, &out16}, npar)) return fail(DD_ERR_ARG, "CG16: missing half field");
  const int N = in32.nrhs, block = block_of(N);
  if (block <= 0) return fail(DD_ERR_ARG, "too many right-hand sides for the vector kernels");
  const int64_t vn = Vh * N;
  k_to16<<<grid_for(vn * npar, block), block, 0, st>>>(halves(in32, npar), halves(out16, npar), vn, npar);
  DD_CUDA(cudaGetLastError());
  return DD_OK;
}

// out[r].x = |x_r|^2 (partials: at least 152 * 8 * N complex doubles)
int cg16_norm(const Field& x16, int64_t Vh, int npar, double2* partials, double2* out, cudaStream_t st) {
  if (!views_ok({&x16}, npar)) return fail(DD_ERR_ARG, "CG16: missing half field");
  const int N = x16.nrhs, block = block_of(N);
  if (block <= 0) return fail(DD_ERR_ARG, "too many right-hand sides for the vector kernels");
  const int64_t vn = Vh * N;
  const int grid = grid_for(vn * npar, block);
  k_norm16<<<grid, block, 0, st>>>(halves(x16, npar), vn, npar, N, partials);
  DD_CUDA(cudaGetLastError());
  return blas_reduce_partials(partials, grid, N, out, 0, st);
}

int cg16_r(const Field& r16, const Field& w16, int64_t Vh, int npar, const double2* g, const double2* n,
           cudaStream_t st) {
  if (!views_ok({&r16, &w16}, npar)) return fail(DD_ERR_ARG, "CG16: missing half field");
  const int N = r16.nrhs, block = block_of(N);
  if (block <= 0) return fail(DD_ERR_ARG, "too many right-hand sides for the vector kernels");
  const int64_t vn = Vh * N;
  k_cg_r16<<<grid_for(vn * npar, block), block, 0, st>>>(halves(r16, npar), halves(w16, npar), vn, npar, N, g, n);
  DD_CUDA(cudaGetLastError());
  return DD_OK;
}

// x += (g / n) p and, with z non-null, p = z + (gn / g) p
int cg16_xp(const Field& x32, const Field& p16, const Field* z16, int64_t Vh, int npar, const double2* g,
            const double2* n, const double2* gn, cudaStream_t st) {
  if (!views_ok({&x32, &p16}, npar) || (z16 && !views_ok({z16}, npar)))
    return fail(DD_ERR_ARG, "CG16: missing half field");
  const int N = x32.nrhs, block = block_of(N);
  if (block <= 0) return fail(DD_ERR_ARG, "too many right-hand sides for the vector kernels");
  const int64_t vn = Vh * N;
  const int grid = grid_for(vn * npar, block);
  if (z16)
    k_cg_xp16<true><<<grid, block, 0, st>>>(halves(x32, npar), halves(p16, npar), halves(*z16, npar), vn, npar, N,
                                            g, n, gn);
  else
    k_cg_xp16<false><<<grid, block, 0, st>>>(halves(x32, npar), halves(p16, npar), halves(p16, npar), vn, npar, N,
                                             g, n, gn);
  DD_CUDA(cudaGetLastError());
  return DD_OK;
}

}  // namespace dd
