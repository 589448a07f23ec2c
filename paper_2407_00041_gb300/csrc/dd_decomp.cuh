// Domain-decomposed stencil: the neighbour coupling of Algorithm 3 of the
// thesis (Section 2.2) on a lattice split into hyper-rectangular local
// lattices P_i (Section 2.1), one per virtual rank.
//
// For every split direction mu a rank sends two face messages per apply:
//   lambda_mu(x) = (I + T_f gamma_mu) psi(x), projected to its two
//     independent spin components (6 complex), for the sites x of its lowest
//     mu slice (the inner boundary d_mu P_i), in the negative mu direction;
//   chi_mu(x + mu) = U_mu(x)^H (I + T_b gamma_mu) psi(x), again 6 complex,
//     for the sites x of its highest mu slice (whose x + mu lie on the outer
//     boundary), in the positive mu direction.
// The receiving rank multiplies lambda by its own link U_mu(x) and adds it
// for the sites of its highest slice, and adds chi for the sites of its
// lowest slice.  (The thesis folds the factor 1/2 into lambda and chi; here it
// stays in the epilogue's beta, as in the single-domain kernel.)  Sites with
// no hop across a split seam ("interior") need no message and run while the
// messages travel; the others run after them.  Each boundary site performs
// its eight hops in the same order and with the same arithmetic as the
// single-domain kernel (the projection and link product of a received
// message are the ones the sender computed in registers, stored at full
// precision), so the decomposed apply equals the single-domain one bit for
// bit where both use the one-thread-per-(site, RHS) kernel.
#pragma once

#include "dd_decomp.h"
#include "dd_hop.cuh"

namespace dd {

template <typename R>
__device__ __forceinline__ void face_store(void* buf, int64_t n, int64_t i, const cx<R> a[3], const cx<R> b[3],
                                           float scale, bool with_scale) {
  if constexpr (sizeof(R) == 4) {
    float4* q = reinterpret_cast<float4*>(buf) + i;
    q[0] = make_float4(a[0].re, a[0].im, a[1].re, a[1].im);
    q[n] = make_float4(a[2].re, a[2].im, b[0].re, b[0].im);
    q[2 * n] = make_float4(b[1].re, b[1].im, b[2].re, b[2].im);
    if (with_scale) reinterpret_cast<float*>(reinterpret_cast<float4*>(buf) + 3 * n)[i] = scale;
  } else {
    double2* q = reinterpret_cast<double2*>(buf) + i;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      q[c * n] = make_double2(a[c].re, a[c].im);
      q[(3 + c) * n] = make_double2(b[c].re, b[c].im);
    }
  }
}

// Returns the sender's scale (1 without one).
template <typename R>
__device__ __forceinline__ R face_load(const void* buf, int64_t n, int64_t i, cx<R> a[3], cx<R> b[3],
                                       bool with_scale) {
  if constexpr (sizeof(R) == 4) {
    const float4* q = reinterpret_cast<const float4*>(buf) + i;
    const float4 v0 = __ldg(q), v1 = __ldg(q + n), v2 = __ldg(q + 2 * n);
    a[0] = mk<R>(v0.x, v0.y);
    a[1] = mk<R>(v0.z, v0.w);
    a[2] = mk<R>(v1.x, v1.y);
    b[0] = mk<R>(v1.z, v1.w);
    b[1] = mk<R>(v2.x, v2.y);
    b[2] = mk<R>(v2.z, v2.w);
    return with_scale ? (R)__ldg(reinterpret_cast<const float*>(reinterpret_cast<const float4*>(buf) + 3 * n) + i)
                      : (R)1;
  } else {
    const double2* q = reinterpret_cast<const double2*>(buf) + i;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double2 u = __ldg(q + c * n), w = __ldg(q + (3 + c) * n);
      a[c] = mk<R>(u.x, u.y);
      b[c] = mk<R>(w.x, w.y);
    }
    return (R)1;
  }
}

// Index of a site on a face of direction MU: the other three local
// coordinates, lexicographic in the order T, Z, Y, X.
template <int MU>
__device__ __forceinline__ int64_t face_index(const Geom& g, const int c[4]) {
  int64_t f = 0;
#pragma unroll
  for (int d = 0; d < 4; ++d)
    if (d != MU) f = f * g.n[d] + c[d];
  return f;
}

// Pack the two outgoing messages of direction MU: thread slots
// [0, nface * N) build lambda from the lowest mu slice, [nface * N, 2 nface N)
// build chi from the highest.  Only sites of the launch's input parities are
// packed (the others' slots are left untouched and never read).
template <int PG, int PIN, bool DAG, int MU>
__global__ void __launch_bounds__(128) k_face_pack(const DomHopArgs A) {
  using R = typename Store<PG>::real;
  const HopArgs& a = A.h;
  const int64_t nf = A.d.nface[MU] * a.nrhs;
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * nf) return;
  const int kind = t >= nf ? 1 : 0;
  if (kind) t -= nf;
  const int64_t f = t / a.nrhs;
  const int r = (int)(t - f * a.nrhs);
  int c[4];
  int64_t rem = f;
#pragma unroll
  for (int d = 3; d >= 0; --d) {
    if (d == MU) continue;
    c[d] = (int)(rem % a.g.n[d]);
    rem /= a.g.n[d];
  }
  c[MU] = kind ? a.g.n[MU] - 1 : 0;
  const int p = (c[0] + c[1] + c[2] + c[3]) & 1;
  // input parities of the launch: both, or the one opposite to the output parity
  if (a.npar == 1 && p == a.p0) return;
  const int lex = ((c[0] * a.g.n[1] + c[1]) * a.g.n[2] + c[2]) * a.g.n[3] + c[3];
  const int s = lex >> 1;
  constexpr int TF = DAG ? +1 : -1;
  constexpr int TB = -TF;
  if constexpr (PG == P16 && PIN == P16) {
    // the FP16 hop of dd_hop.cuh: half2 projection, mixed-FMA link product
    __half2 psi[12], h0[3], h1[3];
    const float scale = load_spinor_h(a.in[p], a.gstride, (int64_t)s * a.nrhs + r, psi);
    cx<float> f0[3], f1[3];
    if (!kind) {
      hop_project_h<MU, TF>(psi, h0, h1);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float2 x0 = __half22float2(h0[c]), x1 = __half22float2(h1[c]);
        f0[c] = mk(x0.x, x0.y);
        f1[c] = mk(x1.x, x1.y);
      }
      face_store<float>(A.f.lam_send[MU], nf, t, f0, f1, scale, true);
    } else {
      hop_project_h<MU, TB>(psi, h0, h1);
      __half2 u[9];
      load_link_h(a.U[p], s, a.g.Vh, MU, u, a.recon ? 12 : 0);
      hop_mul_h<true>(u, h0, h1, f0, f1);
      face_store<float>(A.f.chi_send[MU], nf, t, f0, f1, scale, true);
    }
    return;
  }
  cx<R> psi[12];
  const R scale = load_spinor_unscaled<PIN, R>(a.in[p], a.gstride, (int64_t)s * a.nrhs + r, psi);
  cx<R> h0[3], h1[3];
  if (!kind) {
    hop_project<MU, TF, R>(psi, h0, h1);
    face_store<R>(A.f.lam_send[MU], nf, t, h0, h1, (float)scale, PIN == P16);
  } else {
    hop_project<MU, TB, R>(psi, h0, h1);
    cx<R> u[9], g0[3], g1[3];
    load_link<PG, R>(a.U[p], s, a.g.Vh, MU, u, (PG != P64 && a.recon) ? 12 : 0);
    hop_mul<true, R>(u, h0, h1, g0, g1);
    face_store<R>(A.f.chi_send[MU], nf, t, g0, g1, (float)scale, PIN == P16);
  }
}

// The decomposed stencil: BOUNDARY = false runs the interior sites of the
// launch (sites with a hop across a split seam return at once), BOUNDARY =
// true the rank's boundary sites from its list, taking the hops across the
// seams from the received messages.
template <int PG, int PIN, int POUT, bool DAG, int EPI, bool BOUNDARY>
__global__ void __launch_bounds__(128, (HopMinBlocks<PG, PIN>::value)) k_hop_dd(const DomHopArgs A) {
  using R = typename Store<PG>::real;
  const HopArgs& a = A.h;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t Vh = a.g.Vh;
  int p, s, r;
  if constexpr (BOUNDARY) {
    const int64_t nsites = a.npar == 2 ? A.nb[0] + A.nb[1] : A.nb[a.p0];
    if (tid >= nsites * a.nrhs) return;
    int k = fdiv((int)tid, a.fblk);
    r = (int)tid - k * a.nrhs;
    if (a.npar == 1 && a.p0 == 1) k += (int)A.nb[0];
    const int e = A.bsites[k];
    p = e >= Vh ? 1 : 0;
    s = e - p * (int)Vh;
  } else {
    const int64_t per = Vh * a.nrhs;
    if (tid >= per * a.npar) return;
    int64_t t = tid;
    p = a.p0;
    if (t >= per) {
      t -= per;
      p ^= 1;
    }
    s = fdiv((int)t, a.fblk);
    r = (int)t - s * a.nrhs;
  }
  const SiteCoord sc = site_coords(a.g, s, p);
  if constexpr (!BOUNDARY) {
#pragma unroll
    for (int mu = 0; mu < 4; ++mu)
      if (A.d.xch[mu] && (sc.c[mu] == 0 || sc.c[mu] == a.g.n[mu] - 1)) return;
  }
  const int q = p ^ 1;
  constexpr int TF = DAG ? +1 : -1;
  constexpr int TB = -TF;
  cx<R> acc[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) acc[c] = zero<R>();

#define DD_DHOP(MU)                                                                                      \
  {                                                                                                      \
    if (BOUNDARY && A.d.xch[MU] && sc.c[MU] == a.g.n[MU] - 1) {                                          \
      const int64_t nf = A.d.nface[MU] * a.nrhs;                                                         \
      cx<R> h0[3], h1[3], g0[3], g1[3], u[9];                                                            \
      const R scl = face_load<R>(A.f.lam_recv[MU], nf, face_index<MU>(a.g, sc.c) * a.nrhs + r, h0, h1,    \
                                 PIN == P16);                                                            \
      R sg = (MU == 0 && sc.c[0] + A.d.off[0] == A.d.N[0] - 1) ? (R)a.g.t_bc : (R)1;                     \
      sg *= scl;                                                                                         \
      if constexpr (PG == P16 && PIN == P16) {                                                          \
        __half2 uh[9], x0[3], x1[3];                                                                     \
        _Pragma("unroll") for (int c = 0; c < 3; ++c) {                                                  \
          x0[c] = __floats2half2_rn(h0[c].re, h0[c].im);                                                 \
          x1[c] = __floats2half2_rn(h1[c].re, h1[c].im);                                                 \
        }                                                                                                \
        load_link_h(a.U[p], s, Vh, MU, uh, a.recon ? 12 : 0);                                           \
        hop_mul_h<false>(uh, x0, x1, g0, g1);                                                            \
      } else {                                                                                           \
        load_link<PG, R>(a.U[p], s, Vh, MU, u, (PG != P64 && a.recon) ? 12 : 0);                                        \
        hop_mul<false, R>(u, h0, h1, g0, g1);                                                            \
      }                                                                                                  \
      hop_reconstruct<MU, TF, R>(acc, g0, g1, sg);                                                       \
    } else {                                                                                             \
      const int nl = nb_fwd(a.g, sc, MU);                                                                \
      R sg = (MU == 0 && sc.c[0] == a.g.n[0] - 1) ? (R)a.g.t_bc : (R)1;                                  \
      hop_from<PG, PIN, MU, TF, false, R>(acc, a.in[q], a.gstride, (int64_t)(nl >> 1) * a.nrhs + r, a.U[p], s, \
                                          Vh, sg, (PG != P64 && a.recon) ? 12 : 0);                                     \
    }                                                                                                    \
    if (BOUNDARY && A.d.xch[MU] && sc.c[MU] == 0) {                                                      \
      const int64_t nf = A.d.nface[MU] * a.nrhs;                                                         \
      cx<R> g0[3], g1[3];                                                                                \
      const R scl = face_load<R>(A.f.chi_recv[MU], nf, face_index<MU>(a.g, sc.c) * a.nrhs + r, g0, g1,    \
                                 PIN == P16);                                                            \
      R sg = (MU == 0 && sc.c[0] + A.d.off[0] == 0) ? (R)a.g.t_bc : (R)1;                                \
      sg *= scl;                                                                                         \
      hop_reconstruct<MU, TB, R>(acc, g0, g1, sg);                                                       \
    } else {                                                                                             \
      const int nl = nb_bwd(a.g, sc, MU);                                                                \
      R sg = (MU == 0 && sc.c[0] == 0) ? (R)a.g.t_bc : (R)1;                                             \
      hop_from<PG, PIN, MU, TB, true, R>(acc, a.in[q], a.gstride, (int64_t)(nl >> 1) * a.nrhs + r, a.U[q],    \
                                         nl >> 1, Vh, sg, (PG != P64 && a.recon) ? 12 : 0);                             \
    }                                                                                                    \
  }
  DD_DHOP(0)
  DD_DHOP(1)
  DD_DHOP(2)
  DD_DHOP(3)
#undef DD_DHOP

  hop_epilogue<PG, PIN, POUT, EPI, false, R>(a, p, s, r, acc);
}

// Host launchers (instantiated per precision triple in dd_decomp_f*.cu).
template <int PG, int PIN>
cudaError_t launch_face_pack(const DomHopArgs& A, bool dagger, cudaStream_t st) {
  for (int mu = 0; mu < 4; ++mu) {
    if (!A.d.xch[mu]) continue;
    const int64_t n = 2 * A.d.nface[mu] * A.h.nrhs;
    const unsigned bl = (unsigned)((n + 127) / 128);
    const int key = mu * 2 + (dagger ? 1 : 0);
    switch (key) {
      case 0: k_face_pack<PG, PIN, false, 0><<<bl, 128, 0, st>>>(A); break;
      case 1: k_face_pack<PG, PIN, true, 0><<<bl, 128, 0, st>>>(A); break;
      case 2: k_face_pack<PG, PIN, false, 1><<<bl, 128, 0, st>>>(A); break;
      case 3: k_face_pack<PG, PIN, true, 1><<<bl, 128, 0, st>>>(A); break;
      case 4: k_face_pack<PG, PIN, false, 2><<<bl, 128, 0, st>>>(A); break;
      case 5: k_face_pack<PG, PIN, true, 2><<<bl, 128, 0, st>>>(A); break;
      case 6: k_face_pack<PG, PIN, false, 3><<<bl, 128, 0, st>>>(A); break;
      default: k_face_pack<PG, PIN, true, 3><<<bl, 128, 0, st>>>(A); break;
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int PG, int PIN, int POUT>
cudaError_t launch_hop_dd(const DomHopArgs& args, bool dagger, int epi, bool boundary, cudaStream_t st) {
  DomHopArgs A = args;
  prepare_divs(A.h.g);
  A.h.fblk = make_fastdiv((uint32_t)A.h.nrhs);
  const int64_t sites = boundary ? (A.h.npar == 2 ? A.nb[0] + A.nb[1] : A.nb[A.h.p0]) : A.h.g.Vh * A.h.npar;
  const int64_t n = sites * A.h.nrhs;
  if (n == 0) return cudaSuccess;
  if (n >= (int64_t)1 << 31) return cudaErrorInvalidValue;
  const unsigned bl = (unsigned)((n + 127) / 128);
  if (epi != EPI_D && epi != EPI_AINV) return cudaErrorInvalidValue;
  const int key = (epi == EPI_D ? 0 : 4) + (dagger ? 2 : 0) + (boundary ? 1 : 0);
  switch (key) {
    case 0: k_hop_dd<PG, PIN, POUT, false, EPI_D, false><<<bl, 128, 0, st>>>(A); break;
    case 1: k_hop_dd<PG, PIN, POUT, false, EPI_D, true><<<bl, 128, 0, st>>>(A); break;
    case 2: k_hop_dd<PG, PIN, POUT, true, EPI_D, false><<<bl, 128, 0, st>>>(A); break;
    case 3: k_hop_dd<PG, PIN, POUT, true, EPI_D, true><<<bl, 128, 0, st>>>(A); break;
    case 4: k_hop_dd<PG, PIN, POUT, false, EPI_AINV, false><<<bl, 128, 0, st>>>(A); break;
    case 5: k_hop_dd<PG, PIN, POUT, false, EPI_AINV, true><<<bl, 128, 0, st>>>(A); break;
    case 6: k_hop_dd<PG, PIN, POUT, true, EPI_AINV, false><<<bl, 128, 0, st>>>(A); break;
    default: k_hop_dd<PG, PIN, POUT, true, EPI_AINV, true><<<bl, 128, 0, st>>>(A); break;
  }
  return cudaGetLastError();
}

#define DD_INSTANTIATE_DECOMP(PG, PIN, POUT)                                                              \
  template cudaError_t launch_face_pack<PG, PIN>(const DomHopArgs&, bool, cudaStream_t);                 \
  template cudaError_t launch_hop_dd<PG, PIN, POUT>(const DomHopArgs&, bool, int, bool, cudaStream_t);

}  // namespace dd
