// Two-level algebraic multigrid preconditioner of Section 1.3 on the GPU: the
// coarse-grid correction z = P D_c^{-1} R v with the SAP smoother (dd_sap.cu)
// as post-smoother, and the setup that builds P, R = P^H and D_c = R D P.
//
// Construction (the reading stated in include/dd_wilson.h):
//   * aggregates: blocks of a_T x a_Z x a_Y x a_X sites aligned with the
//     origin, numbered lexicographically on the coarse lattice (X fastest);
//     each carries 2 N coarse degrees of freedom, N per chirality (spin
//     components 0, 1 and 2, 3: gamma5 = +1, -1);
//   * P: the N test vectors restricted to (aggregate, chirality) and
//     orthonormalised by modified Gram-Schmidt in order; P is kept as a native
//     fine field of N right-hand sides whose column i, restricted to
//     (A, c), is the fine vector of coarse degree of freedom (A, c, i);
//   * D_c[A][d] (d = 0: A itself; 1 + 2 mu / 2 + 2 mu: the aggregate at
//     +mu / -mu) is the 2N x 2N block of P^H D P: the self part applies the
//     self coupling and the hops inside A, the face parts the hops from the
//     +-mu face of A into the neighbour (with the time-boundary sign);
//   * coarse vectors and D_c are FP64 ([aggregate][2N][nrhs], RHS innermost;
//     D_c[A][d] stored column-major); the coarse system is solved by GMRES
//     (dd_krylov.h) to a relative tolerance.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "dd_hop.cuh"
#include "dd_internal.h"
#include "dd_krylov.h"
#include "dd_ops.h"
#include "dd_blas.h"
#include "dd_sap.h"
#include "dd_amg.h"

namespace dd {

namespace {

constexpr int kAmgThreads = 256;

struct AmgGeom {
  Geom g;      // fine lattice
  int a[4];    // aggregate extents
  int nc[4];   // coarse lattice extents
  int asites;  // sites per aggregate
};

// site k (0 .. asites-1, X fastest) of aggregate `agg`: coordinates, parity, compact index
__device__ __forceinline__ void agg_site(const AmgGeom& G, int agg, int k, int c[4], int& p, int& s, int& lex) {
  int B[4];
  int u = agg;
  B[3] = u % G.nc[3];
  u /= G.nc[3];
  B[2] = u % G.nc[2];
  u /= G.nc[2];
  B[1] = u % G.nc[1];
  B[0] = u / G.nc[1];
  int l[4];
  u = k;
  l[3] = u % G.a[3];
  u /= G.a[3];
  l[2] = u % G.a[2];
  u /= G.a[2];
  l[1] = u % G.a[1];
  l[0] = u / G.a[1];
  lex = 0;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    c[mu] = B[mu] * G.a[mu] + l[mu];
    lex += c[mu] * G.g.stride[mu];
  }
  p = (c[0] + c[1] + c[2] + c[3]) & 1;
  s = lex >> 1;
}

// complex component `comp` of RHS `col` at compact site s of a native half field
template <int PV, typename R>
__device__ __forceinline__ cx<R> ld_comp(const HalfField& f, int64_t Vh, int N, int s, int comp, int col) {
  if constexpr (PV == P64) {
    const double2 v = reinterpret_cast<const double2*>(f.base)[((int64_t)comp * Vh + s) * N + col];
    return mk<R>((R)v.x, (R)v.y);
  } else {
    const float4 v = reinterpret_cast<const float4*>(f.base)[((int64_t)(comp >> 1) * Vh + s) * N + col];
    return (comp & 1) ? mk<R>((R)v.z, (R)v.w) : mk<R>((R)v.x, (R)v.y);
  }
}

template <int PV, typename R>
__device__ __forceinline__ void st_comp(const HalfField& f, int64_t Vh, int N, int s, int comp, int col, cx<R> v) {
  if constexpr (PV == P64) {
    reinterpret_cast<double2*>(f.base)[((int64_t)comp * Vh + s) * N + col] = make_double2((double)v.re, (double)v.im);
  } else {
    float* b = reinterpret_cast<float*>(reinterpret_cast<float4*>(f.base) + ((int64_t)(comp >> 1) * Vh + s) * N + col);
    b[2 * (comp & 1)] = (float)v.re;
    b[2 * (comp & 1) + 1] = (float)v.im;
  }
}

// Sum of K complex doubles over the CTA, written to out[0 .. K) by threads
// t < K (fixed order: warp shuffles, then the warps in turn).  sm: at least
// (blockDim / 32) * 2 K doubles.
template <int K>
__device__ __forceinline__ void block_sum_write(cx<double> v[K], double* sm, double2* out, int64_t out_stride) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      v[k].re += __shfl_xor_sync(0xffffffffu, v[k].re, off);
      v[k].im += __shfl_xor_sync(0xffffffffu, v[k].im, off);
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      sm[(warp * K + k) * 2] = v[k].re;
      sm[(warp * K + k) * 2 + 1] = v[k].im;
    }
  }
  __syncthreads();
  if ((int)threadIdx.x < K) {
    double re = 0.0, im = 0.0;
    for (int w = 0; w < nw; ++w) re += sm[(w * K + threadIdx.x) * 2], im += sm[(w * K + threadIdx.x) * 2 + 1];
    out[(int64_t)threadIdx.x * out_stride] = make_double2(re, im);
  }
  __syncthreads();
}

// ---- P: modified Gram-Schmidt of the N columns on (aggregate, chirality) ----
// grid (n_agg, 2); the field P (N RHS, both parities) is updated in place.
template <int PV, int NT>
__global__ void __launch_bounds__(kAmgThreads) k_amg_orthonormalize(AmgGeom G, HalfField P0, HalfField P1,
                                                                    int* bad) {
  using R = typename Store<PV>::real;
  __shared__ double sm[(kAmgThreads / 32) * 2 + 4];
  const int agg = blockIdx.x, ch = blockIdx.y;
  const int64_t Vh = G.g.Vh;
  const HalfField P[2] = {P0, P1};
  for (int i = 0; i < NT; ++i) {
    for (int k = 0; k <= i; ++k) {
      // k < i: dot = <P_k, P_i>; k == i: the squared norm of P_i
      cx<double> acc[1] = {zero<double>()};
      for (int t = threadIdx.x; t < G.asites; t += blockDim.x) {
        int c[4], p, s, lex;
        agg_site(G, agg, t, c, p, s, lex);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          const int comp = 6 * ch + q;
          const cx<R> a = ld_comp<PV, R>(P[p], Vh, NT, s, comp, k);
          const cx<R> b = ld_comp<PV, R>(P[p], Vh, NT, s, comp, i);
          acc[0] = cfmac(mk<double>(a.re, a.im), mk<double>(b.re, b.im), acc[0]);
        }
      }
      double2* dst = reinterpret_cast<double2*>(sm + (kAmgThreads / 32) * 2);
      block_sum_write<1>(acc, sm, dst, 1);
      const double2 d = dst[0];
      if (k < i) {
        for (int t = threadIdx.x; t < G.asites; t += blockDim.x) {
          int c[4], p, s, lex;
          agg_site(G, agg, t, c, p, s, lex);
#pragma unroll
          for (int q = 0; q < 6; ++q) {
            const int comp = 6 * ch + q;
            const cx<R> a = ld_comp<PV, R>(P[p], Vh, NT, s, comp, k);
            cx<R> b = ld_comp<PV, R>(P[p], Vh, NT, s, comp, i);
            b = cfma(mk<R>((R)-d.x, (R)-d.y), a, b);
            st_comp<PV, R>(P[p], Vh, NT, s, comp, i, b);
          }
        }
      } else {
        const double nrm = sqrt(d.x);
        if (!(nrm > 0.0)) {
          if (threadIdx.x == 0) atomicExch(bad, 1);
          return;  // uniform across the CTA
        }
        const R inv = (R)(1.0 / nrm);
        for (int t = threadIdx.x; t < G.asites; t += blockDim.x) {
          int c[4], p, s, lex;
          agg_site(G, agg, t, c, p, s, lex);
#pragma unroll
          for (int q = 0; q < 6; ++q) {
            const int comp = 6 * ch + q;
            const cx<R> b = ld_comp<PV, R>(P[p], Vh, NT, s, comp, i);
            st_comp<PV, R>(P[p], Vh, NT, s, comp, i, inv * b);
          }
        }
      }
      __syncthreads();
    }
  }
}

// ---- R v: coarse[(agg * 2N + c N + i) * nrhs + r] = <P_i|_(A,c), v_r|_(A,c)> ----
// grid (n_agg, nrhs)
template <int PV, int NT>
__global__ void __launch_bounds__(kAmgThreads) k_amg_restrict(AmgGeom G, HalfField P0, HalfField P1, HalfField V0,
                                                              HalfField V1, int nrhs, double2* coarse) {
  using R = typename Store<PV>::real;
  __shared__ double sm[(kAmgThreads / 32) * 2 * 2 * NT];
  const int agg = blockIdx.x, r = blockIdx.y;
  const int64_t Vh = G.g.Vh;
  const HalfField P[2] = {P0, P1}, Vf[2] = {V0, V1};
  cx<double> acc[2 * NT];
#pragma unroll
  for (int k = 0; k < 2 * NT; ++k) acc[k] = zero<double>();
  for (int t = threadIdx.x; t < G.asites; t += blockDim.x) {
    int c[4], p, s, lex;
    agg_site(G, agg, t, c, p, s, lex);
    cx<R> v[12];
    load_spinor<PV, R>(Vf[p], Vh * nrhs, (int64_t)s * nrhs + r, v);
#pragma unroll
    for (int i = 0; i < NT; ++i) {
      cx<R> w[12];
      load_spinor<PV, R>(P[p], Vh * NT, (int64_t)s * NT + i, w);
#pragma unroll
      for (int q = 0; q < 12; ++q)
        acc[(q / 6) * NT + i] = cfmac(mk<double>(w[q].re, w[q].im), mk<double>(v[q].re, v[q].im), acc[(q / 6) * NT + i]);
    }
  }
  block_sum_write<2 * NT>(acc, sm, coarse + (int64_t)agg * 2 * NT * nrhs + r, nrhs);
}

// ---- P e: v_r(x)[comp] = sum_i P_i(x)[comp] e[(agg(x) * 2N + c(comp) N + i) * nrhs + r] ----
// one thread per (site of an aggregate, r); grid covers n_agg * asites * nrhs
template <int PV, int NT>
__global__ void __launch_bounds__(kAmgThreads) k_amg_prolong(AmgGeom G, HalfField P0, HalfField P1, int nrhs,
                                                             const double2* __restrict__ coarse, HalfField O0,
                                                             HalfField O1, int64_t total) {
  using R = typename Store<PV>::real;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= total) return;
  const int r = (int)(tid % nrhs);
  const int64_t u = tid / nrhs;
  const int agg = (int)(u / G.asites), k = (int)(u % G.asites);
  const int64_t Vh = G.g.Vh;
  const HalfField P[2] = {P0, P1}, O[2] = {O0, O1};
  int c[4], p, s, lex;
  agg_site(G, agg, k, c, p, s, lex);
  cx<R> out[12];
#pragma unroll
  for (int q = 0; q < 12; ++q) out[q] = zero<R>();
#pragma unroll
  for (int i = 0; i < NT; ++i) {
    cx<R> w[12];
    load_spinor<PV, R>(P[p], Vh * NT, (int64_t)s * NT + i, w);
    const double2 e0 = coarse[((int64_t)agg * 2 * NT + i) * nrhs + r];
    const double2 e1 = coarse[((int64_t)agg * 2 * NT + NT + i) * nrhs + r];
    const cx<R> c0 = mk<R>((R)e0.x, (R)e0.y), c1 = mk<R>((R)e1.x, (R)e1.y);
#pragma unroll
    for (int q = 0; q < 12; ++q) out[q] = cfma(w[q], q < 6 ? c0 : c1, out[q]);
  }
  store_spinor<PV, R>(O[p], Vh * nrhs, (int64_t)s * nrhs + r, out);
}

// ---- D_c: one CTA per (aggregate, coarse column j' = c' N + j) ----
struct AmgBuildArgs {
  AmgGeom G;
  HalfField P[2];       // P (N RHS)
  const void* U[2];     // links by parity (three rows)
  const void* M[2];     // self-coupling blocks by parity
  double2* Dc;          // [agg][9][2N col][2N row]
};

// X(y) = column j of P at site y, masked to chirality cp
template <int PV, int NT, typename R>
__device__ __forceinline__ void masked_col(const AmgBuildArgs& a, int p, int s, int j, int cp, cx<R> X[12]) {
  load_spinor<PV, R>(a.P[p], a.G.g.Vh * NT, (int64_t)s * NT + j, X);
#pragma unroll
  for (int q = 0; q < 12; ++q)
    if ((q / 6) != cp) X[q] = zero<R>();
}

template <int PG, int PV, int NT>
__global__ void __launch_bounds__(kAmgThreads) k_amg_build(const AmgBuildArgs a) {
  using R = typename Store<PG>::real;
  constexpr int K = 2 * NT;
  __shared__ double sm[(kAmgThreads / 32) * 2 * K];
  const int agg = blockIdx.x, jcol = blockIdx.y;
  const int cp = jcol / NT, j = jcol % NT;
  const AmgGeom& G = a.G;
  const int64_t Vh = G.g.Vh;
  for (int d = 0; d < 9; ++d) {
    const int mu = (d - 1) >> 1;
    const bool fwd = d > 0 && ((d - 1) & 1) == 0;
    cx<double> acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = zero<double>();
    for (int t = threadIdx.x; t < G.asites; t += blockDim.x) {
      int c[4], p, s, lex;
      agg_site(G, agg, t, c, p, s, lex);
      const int q = p ^ 1;
      int l[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) l[m] = c[m] % G.a[m];
      cx<R> y[12];
      bool any = false;
      if (d == 0) {
        cx<R> X[12];
        masked_col<PV, NT, R>(a, p, s, j, cp, X);
        block_apply_g<PG, false, R>(a.M[p], s, Vh, X, y, false);
        any = true;
#define DD_AMG_INNER(MU)                                                                       \
        if (l[MU] < G.a[MU] - 1) {                                                             \
          cx<R> nb[12], u[9];                                                                  \
          masked_col<PV, NT, R>(a, q, (lex + G.g.stride[MU]) >> 1, j, cp, nb);                 \
          load_link<PG, R>(a.U[p], s, Vh, MU, u);                                              \
          hop_regs<MU, -1, false, R>(y, nb, u, (R)-0.5);                                       \
        }                                                                                      \
        if (l[MU] > 0) {                                                                       \
          cx<R> nb[12], u[9];                                                                  \
          const int ln = lex - G.g.stride[MU];                                                 \
          masked_col<PV, NT, R>(a, q, ln >> 1, j, cp, nb);                                     \
          load_link<PG, R>(a.U[q], ln >> 1, Vh, MU, u);                                        \
          hop_regs<MU, +1, true, R>(y, nb, u, (R)-0.5);                                        \
        }
        DD_AMG_INNER(0)
        DD_AMG_INNER(1)
        DD_AMG_INNER(2)
        DD_AMG_INNER(3)
#undef DD_AMG_INNER
      } else if (fwd ? l[mu] == G.a[mu] - 1 : l[mu] == 0) {
        // the hop from this face site into the neighbouring aggregate
#pragma unroll
        for (int k = 0; k < 12; ++k) y[k] = zero<R>();
        any = true;
        const int n = G.g.n[mu];
        int ln;
        R sg = (R)-0.5;
        if (fwd) {
          ln = c[mu] == n - 1 ? lex - (n - 1) * G.g.stride[mu] : lex + G.g.stride[mu];
          if (mu == 0 && c[0] == n - 1) sg *= (R)G.g.t_bc;
        } else {
          ln = c[mu] == 0 ? lex + (n - 1) * G.g.stride[mu] : lex - G.g.stride[mu];
          if (mu == 0 && c[0] == 0) sg *= (R)G.g.t_bc;
        }
        cx<R> nb[12], u[9];
        masked_col<PV, NT, R>(a, q, ln >> 1, j, cp, nb);
        switch (mu * 2 + (fwd ? 0 : 1)) {
          case 0: load_link<PG, R>(a.U[p], s, Vh, 0, u); hop_regs<0, -1, false, R>(y, nb, u, sg); break;
          case 1: load_link<PG, R>(a.U[q], ln >> 1, Vh, 0, u); hop_regs<0, +1, true, R>(y, nb, u, sg); break;
          case 2: load_link<PG, R>(a.U[p], s, Vh, 1, u); hop_regs<1, -1, false, R>(y, nb, u, sg); break;
          case 3: load_link<PG, R>(a.U[q], ln >> 1, Vh, 1, u); hop_regs<1, +1, true, R>(y, nb, u, sg); break;
          case 4: load_link<PG, R>(a.U[p], s, Vh, 2, u); hop_regs<2, -1, false, R>(y, nb, u, sg); break;
          case 5: load_link<PG, R>(a.U[q], ln >> 1, Vh, 2, u); hop_regs<2, +1, true, R>(y, nb, u, sg); break;
          case 6: load_link<PG, R>(a.U[p], s, Vh, 3, u); hop_regs<3, -1, false, R>(y, nb, u, sg); break;
          default: load_link<PG, R>(a.U[q], ln >> 1, Vh, 3, u); hop_regs<3, +1, true, R>(y, nb, u, sg); break;
        }
      }
      if (any) {
#pragma unroll
        for (int i = 0; i < NT; ++i) {
          cx<R> w[12];
          load_spinor<PV, R>(a.P[p], Vh * NT, (int64_t)s * NT + i, w);
#pragma unroll
          for (int qq = 0; qq < 12; ++qq)
            acc[(qq / 6) * NT + i] =
                cfmac(mk<double>(w[qq].re, w[qq].im), mk<double>(y[qq].re, y[qq].im), acc[(qq / 6) * NT + i]);
        }
      }
    }
    block_sum_write<K>(acc, sm, a.Dc + (((int64_t)agg * 9 + d) * K + jcol) * K, 1);
  }
}

// ---- y = D_c x on the coarse lattice: one warp per (aggregate, r), lane = row ----
template <int NT>
__global__ void __launch_bounds__(32) k_amg_coarse_apply(AmgGeom G, int nrhs, const double2* __restrict__ Dc,
                                                         const double2* __restrict__ x, double2* y) {
  constexpr int K = 2 * NT;
  const int agg = blockIdx.x, r = blockIdx.y, row = threadIdx.x;
  int B[4];
  int u = agg;
  B[3] = u % G.nc[3];
  u /= G.nc[3];
  B[2] = u % G.nc[2];
  u /= G.nc[2];
  B[1] = u % G.nc[1];
  B[0] = u / G.nc[1];
  cx<double> acc = zero<double>();
  for (int d = 0; d < 9; ++d) {
    int nbB[4] = {B[0], B[1], B[2], B[3]};
    if (d > 0) {
      const int mu = (d - 1) >> 1;
      const int step = ((d - 1) & 1) ? -1 : 1;
      nbB[mu] = (nbB[mu] + step + G.nc[mu]) % G.nc[mu];
    }
    const int nb = ((nbB[0] * G.nc[1] + nbB[1]) * G.nc[2] + nbB[2]) * G.nc[3] + nbB[3];
    const double2* Dd = Dc + ((int64_t)agg * 9 + d) * K * K;
    const double2* xn = x + (int64_t)nb * K * nrhs + r;
    for (int col = 0; col < K; ++col) {
      const double2 xv = __ldg(xn + (int64_t)col * nrhs);
      if (row < K) {
        const double2 m = __ldg(Dd + (int64_t)col * K + row);
        acc = cfma(mk(m.x, m.y), mk(xv.x, xv.y), acc);
      }
    }
  }
  if (row < K) y[((int64_t)agg * K + row) * nrhs + r] = make_double2(acc.re, acc.im);
}

}  // namespace

}  // namespace dd

// ---------------------------------------------------------------- the handle
struct dd_amg {
  dd_clover* op = nullptr;
  int pv = 0;  // fine vector precision of P (P64 or P32)
  int pg = 0;  // precision of the operator data of the build and smoothing
  dd_amg_params prm{};
  dd::AmgGeom G{};
  int nagg = 0, K = 0;
  dd::DevBuf P, Vw, Dc, flag;
  // workspace of the two-level apply (grown to the RHS count in use)
  int ws_nrhs = 0;
  dd::DevBuf cf, ce, r, e, sr;
  dd::CoarseKrylov* kry = nullptr;
  int kry_nrhs = 0;
  int last_coarse_steps = 0;
  double setup_seconds = 0.0;
  ~dd_amg() {
    if (kry) dd::coarse_krylov_destroy(kry);
  }
};

namespace dd {

namespace {

template <int NT>
int launch_orth(dd_amg* A, cudaStream_t st) {
  Field f = field_view(A->op->lat, A->pv, 0, A->P.ptr, A->prm.n_tv);
  DD_CUDA(cudaMemsetAsync(A->flag.ptr, 0, sizeof(int), st));
  const dim3 grid((unsigned)A->nagg, 2);
  if (A->pv == P64)
    k_amg_orthonormalize<P64, NT><<<grid, kAmgThreads, 0, st>>>(A->G, f.h[0], f.h[1], (int*)A->flag.ptr);
  else
    k_amg_orthonormalize<P32, NT><<<grid, kAmgThreads, 0, st>>>(A->G, f.h[0], f.h[1], (int*)A->flag.ptr);
  DD_CUDA(cudaGetLastError());
  int bad = 0;
  DD_CUDA(cudaMemcpyAsync(&bad, A->flag.ptr, sizeof(int), cudaMemcpyDeviceToHost, st));
  DD_CUDA(cudaStreamSynchronize(st));
  if (bad) return fail(DD_ERR_SINGULAR, "AMG: test vectors are linearly dependent on an aggregate");
  return DD_OK;
}

template <int NT>
int launch_build(dd_amg* A, cudaStream_t st) {
  AmgBuildArgs b;
  b.G = A->G;
  Field f = field_view(A->op->lat, A->pv, 0, A->P.ptr, NT);
  b.P[0] = f.h[0];
  b.P[1] = f.h[1];
  const int pi = prec_index(A->pg);
  for (int p = 0; p < 2; ++p) {
    b.U[p] = A->op->gauge->U(pi, p);
    b.M[p] = A->op->M(pi, p);
  }
  b.Dc = reinterpret_cast<double2*>(A->Dc.ptr);
  const dim3 grid((unsigned)A->nagg, (unsigned)(2 * NT));
  if (A->pv == P64)
    k_amg_build<P64, P64, NT><<<grid, kAmgThreads, 0, st>>>(b);
  else if (A->pg == P32)
    k_amg_build<P32, P32, NT><<<grid, kAmgThreads, 0, st>>>(b);
  else
    k_amg_build<P16, P32, NT><<<grid, kAmgThreads, 0, st>>>(b);
  DD_CUDA(cudaGetLastError());
  return DD_OK;
}

template <int NT>
int launch_restrict(dd_amg* A, const Field& v, double2* coarse, cudaStream_t st) {
  Field f = field_view(A->op->lat, A->pv, 0, A->P.ptr, NT);
  const dim3 grid((unsigned)A->nagg, (unsigned)v.nrhs);
  if (A->pv == P64)
    k_amg_restrict<P64, NT><<<grid, kAmgThreads, 0, st>>>(A->G, f.h[0], f.h[1], v.h[0], v.h[1], v.nrhs, coarse);
  else
    k_amg_restrict<P32, NT><<<grid, kAmgThreads, 0, st>>>(A->G, f.h[0], f.h[1], v.h[0], v.h[1], v.nrhs, coarse);
  DD_CUDA(cudaGetLastError());
  return DD_OK;
}

template <int NT>
int launch_prolong(dd_amg* A, const double2* coarse, const Field& out, cudaStream_t st) {
  Field f = field_view(A->op->lat, A->pv, 0, A->P.ptr, NT);
  const int64_t total = (int64_t)A->nagg * A->G.asites * out.nrhs;
  const unsigned blocks = (unsigned)((total + kAmgThreads - 1) / kAmgThreads);
  if (A->pv == P64)
    k_amg_prolong<P64, NT><<<blocks, kAmgThreads, 0, st>>>(A->G, f.h[0], f.h[1], out.nrhs, coarse, out.h[0], out.h[1],
                                                          total);
  else
    k_amg_prolong<P32, NT><<<blocks, kAmgThreads, 0, st>>>(A->G, f.h[0], f.h[1], out.nrhs, coarse, out.h[0], out.h[1],
                                                          total);
  DD_CUDA(cudaGetLastError());
  return DD_OK;
}

template <int NT>
int launch_coarse(dd_amg* A, int nrhs, const double2* x, double2* y, cudaStream_t st) {
  k_amg_coarse_apply<NT><<<dim3((unsigned)A->nagg, (unsigned)nrhs), 32, 0, st>>>(
      A->G, nrhs, reinterpret_cast<const double2*>(A->Dc.ptr), x, y);
  DD_CUDA(cudaGetLastError());
  return DD_OK;
}

int amg_orthonormalize(dd_amg* A, cudaStream_t st) {
  const int n = A->prm.n_tv;
  return n == 4 ? launch_orth<4>(A, st) : n == 8 ? launch_orth<8>(A, st) : launch_orth<16>(A, st);
}
int amg_build(dd_amg* A, cudaStream_t st) {
  const int n = A->prm.n_tv;
  return n == 4 ? launch_build<4>(A, st) : n == 8 ? launch_build<8>(A, st) : launch_build<16>(A, st);
}
int amg_restrict(dd_amg* A, const Field& v, double2* c, cudaStream_t st) {
  const int n = A->prm.n_tv;
  return n == 4 ? launch_restrict<4>(A, v, c, st) : n == 8 ? launch_restrict<8>(A, v, c, st)
                                                           : launch_restrict<16>(A, v, c, st);
}
int amg_prolong(dd_amg* A, const double2* c, const Field& out, cudaStream_t st) {
  const int n = A->prm.n_tv;
  return n == 4 ? launch_prolong<4>(A, c, out, st) : n == 8 ? launch_prolong<8>(A, c, out, st)
                                                            : launch_prolong<16>(A, c, out, st);
}
int amg_coarse(dd_amg* A, int nrhs, const double2* x, double2* y, cudaStream_t st) {
  const int n = A->prm.n_tv;
  return n == 4 ? launch_coarse<4>(A, nrhs, x, y, st) : n == 8 ? launch_coarse<8>(A, nrhs, x, y, st)
                                                               : launch_coarse<16>(A, nrhs, x, y, st);
}

int ensure_ws(dd_amg* A, int nrhs) {
  if (A->ws_nrhs >= nrhs && A->kry && A->kry_nrhs == nrhs) return DD_OK;
  const dd_lattice* lat = A->op->lat;
  const size_t cb = (size_t)A->nagg * A->K * nrhs * sizeof(double2);
  const size_t fb = field_bytes(lat, A->pv, 0, nrhs);
  DD_TRY(A->cf.ensure(cb));
  DD_TRY(A->ce.ensure(cb));
  DD_TRY(A->r.ensure(fb));
  DD_TRY(A->e.ensure(fb));
  DD_TRY(A->sr.ensure(fb));
  A->ws_nrhs = std::max(A->ws_nrhs, nrhs);
  if (A->kry) coarse_krylov_destroy(A->kry);
  A->kry = coarse_krylov_create((int64_t)A->nagg * A->K * nrhs, nrhs, A->prm.coarse_restart,
                                [A, nrhs](const void* x, void* y, cudaStream_t s) {
                                  return amg_coarse(A, nrhs, reinterpret_cast<const double2*>(x),
                                                    reinterpret_cast<double2*>(y), s);
                                });
  if (!A->kry) return fail(DD_ERR_OOM, "AMG: coarse solver workspace");
  A->kry_nrhs = nrhs;
  return DD_OK;
}

// z_r = 1 * e_r + z_r over a native field of N RHS (precision pv)
int add_field(int pv, const dd_lattice* lat, const void* e, void* z, int N, double2* ones, cudaStream_t st) {
  VecList vs;
  vs.p[0] = e;
  const int64_t L = (int64_t)(field_bytes(lat, pv, 0, N) / 16);
  if (pv == P64) return blas_multiaxpy<P64>(vs, 1, ones, 1.0, z, L, N, st);
  return blas_multiaxpy<P32>(vs, 1, ones, 1.0, z, L, N, st);
}

}  // namespace

// z = M^{-1} v (full native fields of precision A->pv, N RHS)
int amg_apply(dd_amg* A, const Field& v, const Field& z, cudaStream_t st) {
  const int N = v.nrhs;
  const dd_lattice* lat = A->op->lat;
  DD_TRY(ensure_ws(A, N));
  double2* cf = reinterpret_cast<double2*>(A->cf.ptr);
  double2* ce = reinterpret_cast<double2*>(A->ce.ptr);
  DD_TRY(amg_restrict(A, v, cf, st));
  int steps = 0;
  DD_TRY(coarse_krylov_solve(A->kry, cf, ce, A->prm.coarse_tol, A->prm.coarse_max_restarts, st, &steps));
  A->last_coarse_steps = steps;
  DD_TRY(amg_prolong(A, ce, z, st));
  if (A->prm.sap_cycles > 0) {
    Field Rf = field_view(lat, A->pv, 0, A->r.ptr, N), Ef = field_view(lat, A->pv, 0, A->e.ptr, N),
          Sf = field_view(lat, A->pv, 0, A->sr.ptr, N);
    DD_TRY(op_residual(A->op, A->pg, A->pv, v, z, Rf, st));  // r = v - D z
    DD_TRY(sap_apply(A->op, A->pg, A->pv, A->prm.sap_block, A->prm.sap_cycles, A->prm.sap_mr_steps, Rf, Ef, Sf, st));
    std::vector<double2> one((size_t)N, make_double2(1.0, 0.0));
    DD_CUDA(cudaMemcpyAsync(ce, one.data(), N * sizeof(double2), cudaMemcpyHostToDevice, st));
    DD_TRY(add_field(A->pv, lat, A->e.ptr, z.h[0].base, N, ce, st));
    DD_CUDA(cudaStreamSynchronize(st));  // `one` is a host temporary
  }
  return DD_OK;
}

int amg_fine_precision(const dd_amg* A) { return A->pv; }
int amg_operator_precision(const dd_amg* A) { return A->pg; }
const dd_clover* amg_operator(const dd_amg* A) { return A->op; }

}  // namespace dd

using namespace dd;

extern "C" {

void dd_amg_params_default(dd_amg_params* p) {
  if (!p) return;
  for (int mu = 0; mu < 4; ++mu) p->aggregate[mu] = 4, p->sap_block[mu] = 4;
  p->n_tv = 8;
  p->setup_iters = 2;
  p->init_sap_iters = 2;
  p->sap_cycles = 1;
  p->sap_mr_steps = 4;
  p->coarse_tol = 5e-2;
  p->coarse_restart = 16;
  p->coarse_max_restarts = 4;
}

int dd_amg_create(dd_clover* op, int prec, const dd_amg_params* prm, const double* w0, dd_amg** out) {
  if (!op || !prm || !w0 || !out) return fail(DD_ERR_ARG, "null argument");
  if (prec != DD_PREC_F64 && prec != DD_PREC_F32 && prec != DD_PREC_F16)
    return fail(DD_ERR_ARG, "AMG precision: F64, F32 or F16 (FP16 links / blocks, FP32 vectors)");
  if (prm->n_tv != 4 && prm->n_tv != 8 && prm->n_tv != 16) return fail(DD_ERR_ARG, "AMG: n_tv must be 4, 8 or 16");
  if (prm->setup_iters < 0 || prm->init_sap_iters < 0 || prm->sap_cycles < 0 || prm->sap_mr_steps < 1 ||
      !(prm->coarse_tol > 0) || prm->coarse_restart < 1 || prm->coarse_restart > 32 || prm->coarse_max_restarts < 1)
    return fail(DD_ERR_ARG, "AMG: bad parameters");
  const dd_lattice* lat = op->lat;
  int asites = 1;
  for (int mu = 0; mu < 4; ++mu) {
    const int a = prm->aggregate[mu];
    if (a < 1 || lat->dims[mu] % a != 0) return fail(DD_ERR_ARG, "AMG: aggregate extents must divide the lattice");
    asites *= a;
  }
  if (6 * asites < prm->n_tv) return fail(DD_ERR_ARG, "AMG: an aggregate holds fewer components than test vectors");
  const int pv = prec == DD_PREC_F64 ? P64 : P32;
  const int pg = prec;
  const int pi = prec_index(pg);
  if (!op->gauge->links[pi].ptr || !op->clov[pi].ptr)
    return fail(DD_ERR_UNSUPPORTED, "precision not created in the gauge/operator handles");
  if (prm->sap_cycles > 0 || prm->init_sap_iters > 0) DD_TRY(sap_check_blocks(lat, prm->sap_block, pv));
  dd_amg* A = new (std::nothrow) dd_amg();
  if (!A) return fail(DD_ERR_OOM, "AMG handle");
  const auto t0 = std::chrono::steady_clock::now();
  A->op = op;
  A->pv = pv;
  A->pg = pg;
  A->prm = *prm;
  A->G.g = lat->geom();
  A->G.asites = asites;
  A->nagg = 1;
  for (int mu = 0; mu < 4; ++mu) {
    A->G.a[mu] = prm->aggregate[mu];
    A->G.nc[mu] = lat->dims[mu] / prm->aggregate[mu];
    A->nagg *= A->G.nc[mu];
  }
  A->K = 2 * prm->n_tv;
  const int NT = prm->n_tv;
  cudaStream_t st = 0;
  auto fin = [&](int s) {
    if (s != DD_OK) delete A;
    return s;
  };
  const size_t fb = field_bytes(lat, pv, 0, NT);
  int s = A->P.alloc(fb);
  if (s == DD_OK) s = A->Vw.alloc(fb);
  if (s == DD_OK) s = A->Dc.alloc((size_t)A->nagg * 9 * A->K * A->K * sizeof(double2));
  if (s == DD_OK) s = A->flag.alloc(sizeof(int));
  if (s != DD_OK) return fin(s);
  Field W = field_view(lat, pv, 0, A->Vw.ptr, NT);
  s = pack(lat, pv, 0, w0, W, st);
  if (s != DD_OK) return fin(s);
  // norms and scaling of the N test vectors
  DevBuf red, partials, coef, tmpf;
  s = red.alloc((size_t)NT * sizeof(double2));
  if (s == DD_OK) s = partials.alloc((size_t)blas_partials_len(NT) * sizeof(double2));
  if (s == DD_OK) s = coef.alloc((size_t)NT * sizeof(double2));
  if (s == DD_OK) s = tmpf.alloc(fb);
  if (s != DD_OK) return fin(s);
  const int64_t L = (int64_t)(fb / 16);
  auto normalise = [&](void* f) -> int {
    VecList vs;
    vs.p[0] = f;
    std::vector<double2> h((size_t)NT);
    int e = pv == P64 ? blas_multidot<P64>(vs, 1, f, L, NT, (double2*)red.ptr, 0, (double2*)partials.ptr, st)
                      : blas_multidot<P32>(vs, 1, f, L, NT, (double2*)red.ptr, 0, (double2*)partials.ptr, st);
    if (e != DD_OK) return e;
    DD_CUDA(cudaMemcpy(h.data(), red.ptr, NT * sizeof(double2), cudaMemcpyDeviceToHost));
    for (int i = 0; i < NT; ++i) {
      if (!(h[i].x > 0.0) || !std::isfinite(h[i].x)) return fail(DD_ERR_SINGULAR, "AMG: a test vector vanished");
      h[i] = make_double2(1.0 / std::sqrt(h[i].x), 0.0);
    }
    DD_CUDA(cudaMemcpy(coef.ptr, h.data(), NT * sizeof(double2), cudaMemcpyHostToDevice));
    return pv == P64 ? blas_scale<P64>((double2*)coef.ptr, f, f, L, NT, st)
                     : blas_scale<P32>((double2*)coef.ptr, f, f, L, NT, st);
  };
  Field Tf = field_view(lat, pv, 0, tmpf.ptr, NT);
  // initial smoothing: w_i <- SAP(w_i)
  if (prm->init_sap_iters > 0) s = A->r.ensure(fb);
  for (int k = 0; k < prm->init_sap_iters && s == DD_OK; ++k) {
    Field Rf = field_view(lat, pv, 0, A->r.ptr, NT);
    s = sap_apply(op, pg, pv, prm->sap_block, std::max(prm->sap_cycles, 1), prm->sap_mr_steps, W, Tf, Rf, st);
    if (s == DD_OK) s = cudaMemcpyAsync(A->Vw.ptr, tmpf.ptr, fb, cudaMemcpyDeviceToDevice, st) == cudaSuccess
                            ? DD_OK : cuda_fail(cudaGetLastError(), "copy");
    if (s == DD_OK) s = normalise(A->Vw.ptr);
  }
  if (s == DD_OK) s = normalise(A->Vw.ptr);
  // setup iterations: P, D_c from w; w_i <- M^{-1} w_i
  for (int it = 0; it <= prm->setup_iters && s == DD_OK; ++it) {
    s = cudaMemcpyAsync(A->P.ptr, A->Vw.ptr, fb, cudaMemcpyDeviceToDevice, st) == cudaSuccess
            ? DD_OK : cuda_fail(cudaGetLastError(), "copy");
    if (s == DD_OK) s = amg_orthonormalize(A, st);
    if (s == DD_OK) s = amg_build(A, st);
    if (s != DD_OK || it == prm->setup_iters) break;
    s = amg_apply(A, W, Tf, st);
    if (s == DD_OK) s = cudaMemcpyAsync(A->Vw.ptr, tmpf.ptr, fb, cudaMemcpyDeviceToDevice, st) == cudaSuccess
                            ? DD_OK : cuda_fail(cudaGetLastError(), "copy");
    if (s == DD_OK) s = normalise(A->Vw.ptr);
  }
  if (s == DD_OK && cudaStreamSynchronize(st) != cudaSuccess) s = cuda_fail(cudaGetLastError(), "AMG setup");
  if (s != DD_OK) return fin(s);
  A->setup_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  *out = A;
  return DD_OK;
}

int dd_amg_destroy(dd_amg* A) {
  delete A;
  return DD_OK;
}

int dd_amg_info(const dd_amg* A, int* coarse_dims4, int* dof_per_aggregate, double* setup_seconds,
                int* last_coarse_steps) {
  if (!A) return fail(DD_ERR_ARG, "null handle");
  if (coarse_dims4)
    for (int mu = 0; mu < 4; ++mu) coarse_dims4[mu] = A->G.nc[mu];
  if (dof_per_aggregate) *dof_per_aggregate = A->K;
  if (setup_seconds) *setup_seconds = A->setup_seconds;
  if (last_coarse_steps) *last_coarse_steps = A->last_coarse_steps;
  return DD_OK;
}

int dd_amg_coarse_download(const dd_amg* A, double* Dc_host) {
  if (!A || !Dc_host) return fail(DD_ERR_ARG, "null argument");
  DD_CUDA(cudaDeviceSynchronize());
  DD_CUDA(cudaMemcpy(Dc_host, A->Dc.ptr, A->Dc.bytes, cudaMemcpyDeviceToHost));
  return DD_OK;
}

int dd_amg_apply(dd_amg* A, const void* v, void* z, int nrhs, int layout, void* stream) {
  if (!A || !v || !z || nrhs < 1) return fail(DD_ERR_ARG, "null argument or nrhs < 1");
  if (layout != DD_LAYOUT_CANONICAL && layout != DD_LAYOUT_NATIVE) return fail(DD_ERR_ARG, "AMG: canonical or native");
  const dd_lattice* lat = A->op->lat;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (layout == DD_LAYOUT_NATIVE) {
    Field Vf = field_view(lat, A->pv, 0, const_cast<void*>(v), nrhs), Zf = field_view(lat, A->pv, 0, z, nrhs);
    return amg_apply(A, Vf, Zf, st);
  }
  const size_t nb = field_bytes(lat, A->pv, 0, nrhs);
  DD_TRY(A->op->ws_in.ensure(nb));
  DD_TRY(A->op->ws_out.ensure(nb));
  Field Vf = field_view(lat, A->pv, 0, A->op->ws_in.ptr, nrhs), Zf = field_view(lat, A->pv, 0, A->op->ws_out.ptr, nrhs);
  DD_TRY(pack(lat, A->pv, 0, reinterpret_cast<const double*>(v), Vf, st));
  DD_TRY(amg_apply(A, Vf, Zf, st));
  DD_TRY(unpack(lat, A->pv, 0, Zf, reinterpret_cast<double*>(z), st));
  return DD_OK;
}

}  // extern "C"
