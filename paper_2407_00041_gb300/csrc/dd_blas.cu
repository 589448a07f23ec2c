// Vector kernels for the Krylov solver on native fields.
//
// A native FP64 or FP32 field of N right-hand sides is a flat array of
// 16-byte groups whose RHS index is (group index mod N) (see the layout in
// dd_wilson.h): FP64 groups hold one complex number, FP32 groups two.
// Every kernel runs with a block size that is a multiple of N and a
// grid-stride loop, so a thread always sees the same right-hand side.
//
// Inner products accumulate in FP64 (warp shuffles inside a block, then a
// fixed-order pass over per-block partials, so results are reproducible).
// FP32 data is summed in FP32 over short runs of 16 groups per thread
// before entering the FP64 accumulator.
#include <algorithm>

#include "dd_blas.h"
#include "dd_internal.h"

namespace dd {

namespace {

template <int PV>
struct G;
template <>
struct G<P64> {
  using group = double2;
  using real = double;
};
template <>
struct G<P32> {
  using group = float4;
  using real = float;
};

__device__ __forceinline__ void acc_dot(double2 v, double2 w, double& re, double& im) {
  re = fma(v.x, w.x, re);
  re = fma(v.y, w.y, re);
  im = fma(v.x, w.y, im);
  im = fma(-v.y, w.x, im);
}
__device__ __forceinline__ void acc_dot(float4 v, float4 w, float& re, float& im) {
  re = fmaf(v.x, w.x, re);
  re = fmaf(v.y, w.y, re);
  re = fmaf(v.z, w.z, re);
  re = fmaf(v.w, w.w, re);
  im = fmaf(v.x, w.y, im);
  im = fmaf(-v.y, w.x, im);
  im = fmaf(v.z, w.w, im);
  im = fmaf(-v.w, w.z, im);
}

// w += c * v with complex c
__device__ __forceinline__ void caxpy(double cr, double ci, double2 v, double2& w) {
  w.x = fma(cr, v.x, fma(-ci, v.y, w.x));
  w.y = fma(cr, v.y, fma(ci, v.x, w.y));
}
__device__ __forceinline__ void caxpy(float cr, float ci, float4 v, float4& w) {
  w.x = fmaf(cr, v.x, fmaf(-ci, v.y, w.x));
  w.y = fmaf(cr, v.y, fmaf(ci, v.x, w.y));
  w.z = fmaf(cr, v.z, fmaf(-ci, v.w, w.z));
  w.w = fmaf(cr, v.w, fmaf(ci, v.z, w.w));
}

constexpr int MAXJ = 8;
constexpr int kMaxCoef = 1024;

// Sum of v over the threads of the block with the same t % N, delivered to
// threads t < N; N divides 32 and the block is a multiple of 32 threads.  An
// xor-shuffle tree inside each warp (lanes with equal lane % N), then the
// warps' sums in a fixed order through `sm` (at least blockDim / 32 * N
// doubles): deterministic.
__device__ __forceinline__ double block_sum_by_rhs(double v, int N, double* sm) {
  for (int off = 16; off >= N; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane < N) sm[warp * N + lane] = v;
  __syncthreads();
  double tot = 0.0;
  if ((int)threadIdx.x < N)
    for (int w = 0; w < nw; ++w) tot += sm[w * N + threadIdx.x];
  __syncthreads();
  return tot;
}

// partials[block][j][r] = sum over this block's groups of <V_j, w> for RHS r.
template <int PV, int MAXJ>
__global__ void __launch_bounds__(256) k_multidot(VecList vs, int J, const void* __restrict__ wp, int64_t L, int N,
                                                  double2* partials) {
  using T = typename G<PV>::group;
  using R = typename G<PV>::real;
  __shared__ double sre[256], sim[256];
  const T* w = reinterpret_cast<const T*>(wp);
  double are[MAXJ], aim[MAXJ];
  R fre[MAXJ], fim[MAXJ];
#pragma unroll
  for (int j = 0; j < MAXJ; ++j) are[j] = aim[j] = 0.0, fre[j] = fim[j] = R(0);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // four elements per pass (independent loads in flight); a vector equal to w
  // (a norm) is not read twice
  bool self[MAXJ];
#pragma unroll
  for (int j = 0; j < MAXJ; ++j) self[j] = j < J && vs.p[j] == wp;
  int run = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < L; e += 4 * stride) {
    T we[4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (e + u * stride < L) we[u] = w[e + u * stride];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (e + u * stride >= L) break;
#pragma unroll
      for (int j = 0; j < MAXJ; ++j)
        if (j < J) acc_dot(self[j] ? we[u] : reinterpret_cast<const T*>(vs.p[j])[e + u * stride], we[u], fre[j], fim[j]);
    }
    run += 4;
    if (PV == P32 && run >= 16) {
      run = 0;
#pragma unroll
      for (int j = 0; j < MAXJ; ++j) are[j] += (double)fre[j], aim[j] += (double)fim[j], fre[j] = fim[j] = R(0);
    }
  }
#pragma unroll
  for (int j = 0; j < MAXJ; ++j) are[j] += (double)fre[j], aim[j] += (double)fim[j];
  const int t = threadIdx.x;
  const int per = blockDim.x / N;  // threads per RHS in this block
  // unrolled over MAXJ so that are[] / aim[] stay in registers
#pragma unroll
  for (int j = 0; j < MAXJ; ++j) {
    if (j >= J) break;
    if (32 % N == 0) {  // warp shuffles
      const double re = block_sum_by_rhs(are[j], N, sre);
      const double im = block_sum_by_rhs(aim[j], N, sim);
      if (t < N) partials[((int64_t)blockIdx.x * J + j) * N + t] = make_double2(re, im);
    } else {
      sre[t] = are[j];
      sim[t] = aim[j];
      __syncthreads();
      if (t < N) {
        double re = 0.0, im = 0.0;
        for (int k = 0; k < per; ++k) re += sre[t + k * N], im += sim[t + k * N];
        partials[((int64_t)blockIdx.x * J + j) * N + t] = make_double2(re, im);
      }
      __syncthreads();
    }
  }
}

// out[j][r] (+)= sum over blocks of partials[block][j][r]: one CTA per
// output, a strided pass over the blocks and a fixed-shape tree, so the
// result does not depend on scheduling.
// out[y * JN + i] (+)= sum of entry i over the partials of chunk y (blocks
// y * chunk .. (y + 1) * chunk - 1); grid (JN, chunks).  Eight independent
// loads in flight per thread on long chunks; fixed summation order.
__global__ void __launch_bounds__(1024) k_reduce_partials(const double2* __restrict__ partials, int nblocks, int JN,
                                                          double2* out, int add, int chunk) {
  __shared__ double sre[32], sim[32];
  const int i = blockIdx.x;
  const int nt = blockDim.x;
  const int b0 = blockIdx.y * chunk;
  const int b1 = min(nblocks, b0 + chunk);
  double re = 0.0, im = 0.0;
  int b = b0 + threadIdx.x;
  for (; b + 7 * nt < b1; b += 8 * nt) {
    double2 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = partials[(int64_t)(b + u * nt) * JN + i];
#pragma unroll
    for (int u = 0; u < 8; ++u) re += v[u].x, im += v[u].y;
  }
  for (; b < b1; b += nt) {
    const double2 v = partials[(int64_t)b * JN + i];
    re += v.x;
    im += v.y;
  }
  re = block_sum_by_rhs(re, 1, sre);
  im = block_sum_by_rhs(im, 1, sim);
  if (threadIdx.x == 0) {
    double2* o = out + (int64_t)blockIdx.y * JN + i;
    if (add) {
      re += o->x;
      im += o->y;
    }
    *o = make_double2(re, im);
  }
}

// w += csign * sum_j c[j][r] * V_j; with `partials` set, also the per-RHS
// |w|^2 of the result (per-block partials, as k_multidot writes them).
template <int PV>
__global__ void __launch_bounds__(256) k_multiaxpy(VecList vs, int J, const double2* __restrict__ c, double csign,
                                                   void* wp, int64_t L, int N, double2* partials) {
  using T = typename G<PV>::group;
  using R = typename G<PV>::real;
  __shared__ R scr[kMaxCoef], sci[kMaxCoef];  // [J][N] coefficients, J * N <= kMaxCoef
  __shared__ double sn[256];
  T* w = reinterpret_cast<T*>(wp);
  for (int k = threadIdx.x; k < J * N; k += blockDim.x) {
    const double2 cc = c[k];
    scr[k] = (R)(csign * cc.x);
    sci[k] = (R)(csign * cc.y);
  }
  __syncthreads();
  const int r = threadIdx.x % N;
  double nrm = 0.0;
  R fn = R(0);
  int run = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < L; e += stride) {
    T we = w[e];
    for (int j = 0; j < J; ++j) caxpy(scr[j * N + r], sci[j * N + r], reinterpret_cast<const T*>(vs.p[j])[e], we);
    w[e] = we;
    if (partials) {
      if constexpr (PV == P64) {
        nrm += we.x * we.x + we.y * we.y;
      } else {
        fn += we.x * we.x + we.y * we.y + we.z * we.z + we.w * we.w;
        if (++run == 16) {
          run = 0;
          nrm += (double)fn;
          fn = R(0);
        }
      }
    }
  }
  if (!partials) return;
  nrm += (double)fn;
  if (32 % N == 0) {  // warp shuffles
    const double acc = block_sum_by_rhs(nrm, N, sn);
    if ((int)threadIdx.x < N) partials[(int64_t)blockIdx.x * N + threadIdx.x] = make_double2(acc, 0.0);
    return;
  }
  sn[threadIdx.x] = nrm;
  __syncthreads();
  if (threadIdx.x < N) {
    double acc = 0.0;
    for (int k = 0; k < (int)blockDim.x / N; ++k) acc += sn[threadIdx.x + k * N];
    partials[(int64_t)blockIdx.x * N + threadIdx.x] = make_double2(acc, 0.0);
  }
}

// out = c[r] * in  (complex c [N])
template <int PV>
__global__ void __launch_bounds__(256) k_scale(const double2* __restrict__ c, const void* inp, void* outp, int64_t L,
                                               int N) {
  using T = typename G<PV>::group;
  using R = typename G<PV>::real;
  const T* in = reinterpret_cast<const T*>(inp);
  T* out = reinterpret_cast<T*>(outp);
  const int r = threadIdx.x % N;
  const R cr = (R)c[r].x, ci = (R)c[r].y;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < L; e += stride) {
    T v = in[e], o;
    if constexpr (PV == P64) {
      o.x = cr * v.x - ci * v.y;
      o.y = cr * v.y + ci * v.x;
    } else {
      o.x = cr * v.x - ci * v.y;
      o.y = cr * v.y + ci * v.x;
      o.z = cr * v.z - ci * v.w;
      o.w = cr * v.w + ci * v.z;
    }
    out[e] = o;
  }
}

// FP64 field (L64 double2 groups) -> FP32 field (L64 / 2 float4 groups).
// Group g of an FP32 half field holds components 2g, 2g+1; group c of an FP64
// half field holds component c.  Index maps: FP32 group (h, g, i) with
// i = site * N + r <- FP64 groups (h, 2g, i) and (h, 2g + 1, i).
__global__ void k_demote(const double2* __restrict__ in, float4* out, int64_t nhalf, int64_t VN) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // over nhalf * 6 * VN
  if (t >= nhalf * 6 * VN) return;
  const int64_t i = t % VN;
  const int64_t hg = t / VN;
  const int64_t h = hg / 6, g = hg % 6;
  const double2 a = in[(h * 12 + 2 * g) * VN + i];
  const double2 b = in[(h * 12 + 2 * g + 1) * VN + i];
  out[t] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
}

// x64 += e32 with the same index map
__global__ void k_promote_add(const float4* __restrict__ in, double2* out, int64_t nhalf, int64_t VN) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nhalf * 6 * VN) return;
  const int64_t i = t % VN;
  const int64_t hg = t / VN;
  const int64_t h = hg / 6, g = hg % 6;
  const float4 v = in[t];
  double2* a = out + (h * 12 + 2 * g) * VN + i;
  double2* b = out + (h * 12 + 2 * g + 1) * VN + i;
  a->x += (double)v.x;
  a->y += (double)v.y;
  b->x += (double)v.z;
  b->y += (double)v.w;
}

__global__ void k_add64(const double2* __restrict__ in, double2* out, int64_t n) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  out[t].x += in[t].x;
  out[t].y += in[t].y;
}

// Conjugate-gradient updates with per-RHS step sizes read from device
// scalars (no host round trip):
// g, n, gn: complex double [N] holding squared norms in .x (a zero
// denominator gives a zero step).
//   k_cg_r:   alpha = g / n;  r -= alpha w
//   k_cg_x:   alpha = g / n;  x += alpha p
//   k_cg_xp:  alpha = g / n, beta = gn / g;  x += alpha p;  p = z + beta p
// (the CG step with the x update deferred into the direction update: the
// same arithmetic in one pass over p)
template <int PV>
__global__ void __launch_bounds__(256) k_cg_r(void* rp, const void* wp, const double2* __restrict__ g,
                                              const double2* __restrict__ n, int64_t L, int N) {
  using T = typename G<PV>::group;
  using R = typename G<PV>::real;
  const int r = threadIdx.x % N;
  const double nn = n[r].x;
  const R alpha = nn > 0.0 ? (R)(g[r].x / nn) : R(0);
  T* res = reinterpret_cast<T*>(rp);
  const T* w = reinterpret_cast<const T*>(wp);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < L; e += stride) caxpy(-alpha, R(0), w[e], res[e]);
}

template <int PV>
__global__ void __launch_bounds__(256) k_cg_x(void* xp, const void* pp, const double2* __restrict__ g,
                                              const double2* __restrict__ n, int64_t L, int N) {
  using T = typename G<PV>::group;
  using R = typename G<PV>::real;
  const int r = threadIdx.x % N;
  const double nn = n[r].x;
  const R alpha = nn > 0.0 ? (R)(g[r].x / nn) : R(0);
  T* x = reinterpret_cast<T*>(xp);
  const T* p = reinterpret_cast<const T*>(pp);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < L; e += stride) caxpy(alpha, R(0), p[e], x[e]);
}

template <int PV>
__global__ void __launch_bounds__(256) k_cg_xp(void* xp, void* pp, const void* zp, const double2* __restrict__ g,
                                               const double2* __restrict__ n, const double2* __restrict__ gn,
                                               int64_t L, int N) {
  using T = typename G<PV>::group;
  using R = typename G<PV>::real;
  const int r = threadIdx.x % N;
  const double nn = n[r].x, go = g[r].x;
  const R alpha = nn > 0.0 ? (R)(go / nn) : R(0);
  const R beta = go > 0.0 ? (R)(gn[r].x / go) : R(0);
  T* x = reinterpret_cast<T*>(xp);
  T* p = reinterpret_cast<T*>(pp);
  const T* z = reinterpret_cast<const T*>(zp);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < L; e += stride) {
    const T pe = p[e];
    caxpy(alpha, R(0), pe, x[e]);
    T v = z[e];
    caxpy(beta, R(0), pe, v);
    p[e] = v;
  }
}

// threads of the partial reduce: about four partials per thread, 32..1024
int reduce_threads(int nblocks) {
  const int t = ((nblocks + 3) / 4 + 31) / 32 * 32;
  return t < 32 ? 32 : t > 1024 ? 1024 : t;
}

int block_for(int N) {
  if (N > 256) return -1;
  return (256 / N) * N;
}

}  // namespace

int blas_grid(int64_t L, int block) {
  const int64_t want = (L + block - 1) / block;
  const int64_t cap = 152 * 8;
  return (int)(want < cap ? (want < 1 ? 1 : want) : cap);
}

template <int PV>
int blas_multidot(const VecList& vs, int J, const void* w, int64_t L, int N, double2* dots_dev, int add,
                  double2* partials, cudaStream_t st) {
  const int block = block_for(N);
  if (block <= 0) return fail(DD_ERR_ARG, "too many right-hand sides for the vector kernels");
  const int grid = blas_grid(L, block);
  for (int j0 = 0; j0 < J; j0 += MAXJ) {
    const int Jc = J - j0 < MAXJ ? J - j0 : MAXJ;
    VecList sub;
    for (int j = 0; j < Jc; ++j) sub.p[j] = vs.p[j0 + j];
    if (Jc == 1)  // one vector (a norm or a single product): fewer registers
      k_multidot<PV, 1><<<grid, block, 0, st>>>(sub, Jc, w, L, N, partials);
    else
      k_multidot<PV, MAXJ><<<grid, block, 0, st>>>(sub, Jc, w, L, N, partials);
    const int JN = Jc * N;
    k_reduce_partials<<<JN, reduce_threads(grid), 0, st>>>(partials, grid, JN, dots_dev + (int64_t)j0 * N, add,
                                                           grid);
  }
  DD_CUDA(cudaGetLastError());
  return DD_OK;
}

template <int PV>
int blas_multiaxpy(const VecList& vs, int J, const double2* c_dev, double csign, void* w, int64_t L, int N,
                   cudaStream_t st, double2* norm_out, double2* partials) {
  const int block = block_for(N);
  if (block <= 0) return fail(DD_ERR_ARG, "too many right-hand sides for the vector kernels");
  const int grid = blas_grid(L, block);
  const int jc = std::max(1, std::min(32, kMaxCoef / N));
  for (int j0 = 0; j0 < J || (J == 0 && j0 == 0); j0 += jc) {
    const int Jc = std::min(jc, J - j0);
    const bool last = j0 + jc >= J;
    VecList sub;
    for (int j = 0; j < Jc; ++j) sub.p[j] = vs.p[j0 + j];
    k_multiaxpy<PV><<<grid, block, 0, st>>>(sub, Jc, c_dev + (int64_t)j0 * N, csign, w, L, N,
                                            last && norm_out ? partials : nullptr);
    if (J == 0) break;
  }
  if (norm_out) k_reduce_partials<<<N, reduce_threads(grid), 0, st>>>(partials, grid, N, norm_out, 0, grid);
  DD_CUDA(cudaGetLastError());
  return DD_OK;
}

int blas_reduce_partials(const double2* partials, int nblocks, int JN, double2* out, int add, cudaStream_t st,
                         double2* scratch) {
  if (nblocks < 1 || JN < 1) return fail(DD_ERR_ARG, "empty reduction");
  if (blas_reduce_scratch(nblocks, JN) > 0 && scratch) {
    // FP64 adds are slow on one SM: spread the first stage over 64 CTAs
    const int G = 64, chunk = (nblocks + G - 1) / G;
    k_reduce_partials<<<dim3(JN, G), reduce_threads(chunk), 0, st>>>(partials, nblocks, JN, scratch, 0, chunk);
    k_reduce_partials<<<JN, reduce_threads(G), 0, st>>>(scratch, G, JN, out, add, G);
  } else {
    k_reduce_partials<<<JN, reduce_threads(nblocks), 0, st>>>(partials, nblocks, JN, out, add, nblocks);
  }
  DD_CUDA(cudaGetLastError());
  return DD_OK;
}

template <int PV>
int blas_scale(const double2* c_dev, const void* in, void* out, int64_t L, int N, cudaStream_t st) {
  const int block = block_for(N);
  if (block <= 0) return fail(DD_ERR_ARG, "too many right-hand sides for the vector kernels");
  k_scale<PV><<<blas_grid(L, block), block, 0, st>>>(c_dev, in, out, L, N);
  DD_CUDA(cudaGetLastError());
  return DD_OK;
}

int blas_demote(const void* in64, void* out32, int64_t nhalf, int64_t VN, cudaStream_t st) {
  const int64_t n = nhalf * 6 * VN;
  k_demote<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(reinterpret_cast<const double2*>(in64),
                                                       reinterpret_cast<float4*>(out32), nhalf, VN);
  DD_CUDA(cudaGetLastError());
  return DD_OK;
}

int blas_promote_add(const void* in32, void* out64, int64_t nhalf, int64_t VN, cudaStream_t st) {
  const int64_t n = nhalf * 6 * VN;
  k_promote_add<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(reinterpret_cast<const float4*>(in32),
                                                            reinterpret_cast<double2*>(out64), nhalf, VN);
  DD_CUDA(cudaGetLastError());
  return DD_OK;
}

int blas_add64(const void* in, void* out, int64_t n, cudaStream_t st) {
  k_add64<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(reinterpret_cast<const double2*>(in),
                                                      reinterpret_cast<double2*>(out), n);
  DD_CUDA(cudaGetLastError());
  return DD_OK;
}

template <int PV>
int blas_cg_r(void* r, const void* w, const double2* g, const double2* n, int64_t L, int N, cudaStream_t st) {
  const int block = block_for(N);
  if (block <= 0) return fail(DD_ERR_ARG, "too many right-hand sides for the vector kernels");
  k_cg_r<PV><<<blas_grid(L, block), block, 0, st>>>(r, w, g, n, L, N);
  DD_CUDA(cudaGetLastError());
  return DD_OK;
}

template <int PV>
int blas_cg_x(void* x, const void* p, const double2* g, const double2* n, int64_t L, int N, cudaStream_t st) {
  const int block = block_for(N);
  if (block <= 0) return fail(DD_ERR_ARG, "too many right-hand sides for the vector kernels");
  k_cg_x<PV><<<blas_grid(L, block), block, 0, st>>>(x, p, g, n, L, N);
  DD_CUDA(cudaGetLastError());
  return DD_OK;
}

template <int PV>
int blas_cg_xp(void* x, void* p, const void* z, const double2* g, const double2* n, const double2* gn, int64_t L,
               int N, cudaStream_t st) {
  const int block = block_for(N);
  if (block <= 0) return fail(DD_ERR_ARG, "too many right-hand sides for the vector kernels");
  k_cg_xp<PV><<<blas_grid(L, block), block, 0, st>>>(x, p, z, g, n, gn, L, N);
  DD_CUDA(cudaGetLastError());
  return DD_OK;
}

template int blas_cg_r<P64>(void*, const void*, const double2*, const double2*, int64_t, int, cudaStream_t);
template int blas_cg_r<P32>(void*, const void*, const double2*, const double2*, int64_t, int, cudaStream_t);
template int blas_cg_x<P64>(void*, const void*, const double2*, const double2*, int64_t, int, cudaStream_t);
template int blas_cg_x<P32>(void*, const void*, const double2*, const double2*, int64_t, int, cudaStream_t);
template int blas_cg_xp<P64>(void*, void*, const void*, const double2*, const double2*, const double2*, int64_t, int,
                             cudaStream_t);
template int blas_cg_xp<P32>(void*, void*, const void*, const double2*, const double2*, const double2*, int64_t, int,
                             cudaStream_t);
template int blas_multidot<P64>(const VecList&, int, const void*, int64_t, int, double2*, int, double2*, cudaStream_t);
template int blas_multidot<P32>(const VecList&, int, const void*, int64_t, int, double2*, int, double2*, cudaStream_t);
template int blas_multiaxpy<P64>(const VecList&, int, const double2*, double, void*, int64_t, int, cudaStream_t,
                                 double2*, double2*);
template int blas_multiaxpy<P32>(const VecList&, int, const double2*, double, void*, int64_t, int, cudaStream_t,
                                 double2*, double2*);
template int blas_scale<P64>(const double2*, const void*, void*, int64_t, int, cudaStream_t);
template int blas_scale<P32>(const double2*, const void*, void*, int64_t, int, cudaStream_t);

}  // namespace dd
