// Link derivative of L = Re <phi, D psi> = Re sum_x phi(x)^H (D psi)(x).
//
// G_mu(x) = dL/dRe U_mu(x) + i dL/dIm U_mu(x); F = P(G U^H) with
// P(M) = (M - M^H)/2 - tr(M - M^H)/6 I (the su(3) component).
//
// Hopping terms (Eq. 1.13).  The link U = U_mu(x) enters the forward hop at
// x and the backward hop at y = x + mu.  Because (I -+ gamma_mu) / 2 are
// Hermitian projectors of rank two, each spin sum reduces to the two
// independent components of the projected spinors (the same half-spinors
// h = u -+ B_mu l that the stencil forms; nothing is stored, they are
// recomputed here):
//   G[a][b] = -1/2 s sum_{k=0,1} ( h-(phi(x))_{k,a} conj(h-(psi(y))_{k,b})
//                                 + h+(psi(x))_{k,a} conj(h+(phi(y))_{k,b}) )
// with s the time-boundary sign of the hop, summed over right-hand sides.
//
// Self coupling (Eq. 1.11, 1.12).  Since Q_numu = Q_munu^H,
//   L_sc = const + Re sum_x sum_{mu<nu} tr(Q_munu(x) T'_munu(x)),
//   T'_munu = 2 (T_munu - T_munu^H),
//   T_munu[b][a] = -(c_sw/32) sum_{s,s'} (gamma_mu gamma_nu)[s][s'] psi(x)[s'][b] conj(phi(x)[s][a]).
// For a leaf F1 F2 F3 F4 of Q_munu(x), tr(F1..F4 T') = tr(F_k R_k) with
// R_k = F_{k+1}..F4 T' F1..F_{k-1}; the link of factor k receives R_k^H if
// F_k = U and R_k if F_k = U^H (accumulated with atomic adds).
#include "dd_internal.h"

namespace dd {

namespace {

struct FGeom {
  int n[4];
  int stride[4];
  int64_t V, Vh;
  double t_bc;
};

FGeom fgeom(const dd_lattice* lat) {
  FGeom g;
  for (int i = 0; i < 4; ++i) g.n[i] = lat->dims[i];
  g.stride[3] = 1;
  g.stride[2] = g.n[3];
  g.stride[1] = g.n[3] * g.n[2];
  g.stride[0] = g.n[3] * g.n[2] * g.n[1];
  g.V = lat->V;
  g.Vh = lat->Vh;
  g.t_bc = lat->t_bc;
  return g;
}

__device__ __forceinline__ void coords_of(const FGeom& g, int lex, int c[4]) {
  c[3] = lex % g.n[3];
  int r = lex / g.n[3];
  c[2] = r % g.n[2];
  r /= g.n[2];
  c[1] = r % g.n[1];
  c[0] = r / g.n[1];
}

template <typename R>
struct M3 {
  cx<R> m[9];
};

template <typename R>
__device__ __forceinline__ M3<R> load_link(const FGeom& g, const double2* U64, const int c[4], int mu) {
  const int lex = ((c[0] * g.n[1] + c[1]) * g.n[2] + c[2]) * g.n[3] + c[3];
  const int p = (c[0] + c[1] + c[2] + c[3]) & 1;
  const double2* b = U64 + (int64_t)p * 36 * g.Vh + (int64_t)mu * 9 * g.Vh + (lex >> 1);
  M3<R> r;
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    double2 v = b[e * g.Vh];
    r.m[e] = mk<R>((R)v.x, (R)v.y);
  }
  return r;
}

// The same from the FP32 native copy: element E = 9 mu + e of a site in
// slot E & 1 of float4 group E / 2, [parity][18 groups][Vh]
template <typename R>
__device__ __forceinline__ M3<R> load_link(const FGeom& g, const float2* U32, const int c[4], int mu) {
  const int lex = ((c[0] * g.n[1] + c[1]) * g.n[2] + c[2]) * g.n[3] + c[3];
  const int p = (c[0] + c[1] + c[2] + c[3]) & 1;
  const float2* b = U32 + (int64_t)p * 36 * g.Vh + 2 * (int64_t)(lex >> 1);
  M3<R> r;
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    const int E = 9 * mu + e;
    const float2 v = b[(int64_t)(E >> 1) * 2 * g.Vh + (E & 1)];
    r.m[e] = mk<R>((R)v.x, (R)v.y);
  }
  return r;
}

template <typename R>
__device__ __forceinline__ M3<R> mmul(const M3<R>& a, const M3<R>& b) {
  M3<R> r;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cx<R> acc = zero<R>();
#pragma unroll
      for (int k = 0; k < 3; ++k) acc = cfma(a.m[3 * i + k], b.m[3 * k + j], acc);
      r.m[3 * i + j] = acc;
    }
  return r;
}

template <typename R>
__device__ __forceinline__ M3<R> mdag(const M3<R>& a) {
  M3<R> r;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) r.m[3 * i + j] = mk(a.m[3 * j + i].re, -a.m[3 * j + i].im);
  return r;
}

// h = u + t B_mu l for a spinor given as 12 complex (3 spin + colour)
template <typename R>
__device__ __forceinline__ void half_spinor(int mu, int t, const cx<R> v[12], cx<R> h[2][3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const cx<R> l0 = v[6 + c], l1 = v[9 + c];
    cx<R> b0, b1;
    switch (mu) {
      case 0: b0 = l0; b1 = l1; break;
      case 1: b0 = mul_mi(l0); b1 = mul_i(l1); break;
      case 2: b0 = neg(l1); b1 = l0; break;
      default: b0 = mul_mi(l1); b1 = mul_mi(l0); break;
    }
    h[0][c] = t > 0 ? v[c] + b0 : v[c] - b0;
    h[1][c] = t > 0 ? v[3 + c] + b1 : v[3 + c] - b1;
  }
}

template <typename R>
__device__ __forceinline__ void load_canon(const double2* f, int64_t site, cx<R> v[12]) {
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    double2 d = f[site * 12 + c];
    v[c] = mk<R>((R)d.x, (R)d.y);
  }
}
// canonical FP32 copy ([nrhs][V][12] float2, 16-byte loads)
template <typename R>
__device__ __forceinline__ void load_canon(const float2* f, int64_t site, cx<R> v[12]) {
  const float4* q = reinterpret_cast<const float4*>(f + site * 12);
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const float4 d = q[c];
    v[2 * c] = mk<R>((R)d.x, (R)d.y);
    v[2 * c + 1] = mk<R>((R)d.z, (R)d.w);
  }
}

// canonical FP64 spinors -> FP32 (the input of the FP32 force kernels)
__global__ void k_canon_to_f32(int64_t n, const double2* __restrict__ in, float2* out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const double2 v = in[t];
  out[t] = make_float2((float)v.x, (float)v.y);
}

// G storage: FP64 as 9 double2 per link; the FP32 path accumulates in 20
// floats per link (18 used) and converts at the end.
__device__ __forceinline__ void store_link_g(double2* G, int64_t t, const cx<double> v[9]) {
#pragma unroll
  for (int e = 0; e < 9; ++e) G[t * 9 + e] = make_double2(v[e].re, v[e].im);
}
__device__ __forceinline__ void store_link_g(float* G, int64_t t, const cx<float> v[9]) {
  float4* o = reinterpret_cast<float4*>(G + t * 20);
  o[0] = make_float4(v[0].re, v[0].im, v[1].re, v[1].im);
  o[1] = make_float4(v[2].re, v[2].im, v[3].re, v[3].im);
  o[2] = make_float4(v[4].re, v[4].im, v[5].re, v[5].im);
  o[3] = make_float4(v[6].re, v[6].im, v[7].re, v[7].im);
  o[4] = make_float4(v[8].re, v[8].im, 0.f, 0.f);
}

// One thread per link (x, mu): hopping contribution, written (not added).
template <typename R, typename GT, typename ST>
__global__ void k_force_hop(FGeom g, const ST* __restrict__ phi, const ST* __restrict__ psi, int nrhs, GT* G) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.V * 4) return;
  const int x = (int)(t >> 2), mu = (int)(t & 3);
  int c[4];
  coords_of(g, x, c);
  R s = 1;
  int y;
  if (c[mu] == g.n[mu] - 1) {
    y = x - (g.n[mu] - 1) * g.stride[mu];
    if (mu == 0) s = (R)g.t_bc;
  } else {
    y = x + g.stride[mu];
  }
  cx<R> acc[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) acc[e] = zero<R>();
  for (int r = 0; r < nrhs; ++r) {
    const ST* ph = phi + (int64_t)r * g.V * 12;
    const ST* ps = psi + (int64_t)r * g.V * 12;
    cx<R> v[12], hA[2][3], hB[2][3];
    // h-(phi(x)) (x) conj(h-(psi(y)))
    load_canon<R>(ph, x, v);
    half_spinor<R>(mu, -1, v, hA);
    load_canon<R>(ps, y, v);
    half_spinor<R>(mu, -1, v, hB);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int k = 0; k < 2; ++k) acc[3 * a + b] = cfmac(hB[k][b], hA[k][a], acc[3 * a + b]);
    // h+(psi(x)) (x) conj(h+(phi(y)))
    load_canon<R>(ps, x, v);
    half_spinor<R>(mu, +1, v, hA);
    load_canon<R>(ph, y, v);
    half_spinor<R>(mu, +1, v, hB);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int k = 0; k < 2; ++k) acc[3 * a + b] = cfmac(hB[k][b], hA[k][a], acc[3 * a + b]);
  }
  const R f = (R)(-0.5) * s;
#pragma unroll
  for (int e = 0; e < 9; ++e) acc[e] = f * acc[e];
  store_link_g(G, t, acc);
}

__device__ __forceinline__ cx<double> Bm(int mu, int i, int j) {
  if (mu == 0) return mk(i == j ? 1.0 : 0.0, 0.0);
  if (mu == 1) return i != j ? mk(0.0, 0.0) : mk(0.0, i == 0 ? -1.0 : 1.0);
  if (mu == 2) return i == j ? mk(0.0, 0.0) : mk(i == 0 ? -1.0 : 1.0, 0.0);
  return i == j ? mk(0.0, 0.0) : mk(0.0, -1.0);
}

// (gamma_mu gamma_nu)[s][s'] in the chiral basis: block diagonal,
// upper B_mu B_nu^H, lower B_mu^H B_nu.
__device__ __forceinline__ cx<double> gg(int mu, int nu, int s, int sp) {
  if ((s < 2) != (sp < 2)) return mk(0.0, 0.0);
  const int i = s & 1, j = sp & 1;
  cx<double> acc = zero<double>();
  for (int k = 0; k < 2; ++k) {
    if (s < 2) {
      cx<double> b = Bm(nu, j, k);
      acc = cfma(Bm(mu, i, k), mk(b.re, -b.im), acc);
    } else {
      cx<double> a = Bm(mu, k, i);
      acc = cfma(mk(a.re, -a.im), Bm(nu, k, j), acc);
    }
  }
  return acc;
}

template <typename R>
__device__ __forceinline__ void atomic_add_m3(double2* G, const M3<R>& m, bool dagger) {
  double* g = reinterpret_cast<double*>(G);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const cx<R> v = dagger ? mk(m.m[3 * j + i].re, -m.m[3 * j + i].im) : m.m[3 * i + j];
      atomicAdd(g + 2 * (3 * i + j), (double)v.re);
      atomicAdd(g + 2 * (3 * i + j) + 1, (double)v.im);
    }
}

// FP32 accumulator: a link's 3x3 complex matrix as 18 floats padded to 20
// (80 bytes, 16-byte aligned), added with 16-byte vector reductions.
constexpr int kGf = 20;

__device__ __forceinline__ void red_add_v4(float* p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
}

__device__ __forceinline__ void atomic_add_m3(float* G, const M3<float>& m, bool dagger) {
  float v[kGf];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const cx<float> e = dagger ? mk(m.m[3 * j + i].re, -m.m[3 * j + i].im) : m.m[3 * i + j];
      v[2 * (3 * i + j)] = e.re;
      v[2 * (3 * i + j) + 1] = e.im;
    }
  v[18] = v[19] = 0.f;
#pragma unroll
  for (int q = 0; q < kGf / 4; ++q) red_add_v4(G + 4 * q, v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

// The self-coupling contribution of site c for plane (mu, nu): T' from the
// spinors (summed over right-hand sides), then for each of the four leaves
// of Q_munu(x) (Eq. 1.12) the derivatives R_k of its four factors, handed to
// emit(site coordinates, direction, R_k, add R_k^H instead).
template <typename R, int mu, int nu, typename UT, typename ST, typename Emit>
__device__ __forceinline__ void clover_plane_leaves(const FGeom& g, const UT* __restrict__ U,
                                                    const ST* __restrict__ phi, const ST* __restrict__ psi,
                                                    int nrhs, double csw, const int c[4], Emit emit) {
  const int x = ((c[0] * g.n[1] + c[1]) * g.n[2] + c[2]) * g.n[3] + c[3];
  cx<R> ph[12], ps[12];
  // T[b][a] = -(c_sw/32) sum_{s,s'} gg[s][s'] psi[s'][b] conj(phi[s][a]), summed over RHS
  M3<R> T;
#pragma unroll
  for (int e = 0; e < 9; ++e) T.m[e] = zero<R>();
  for (int r = 0; r < nrhs; ++r) {
    load_canon<R>(phi + (int64_t)r * g.V * 12, x, ph);
    load_canon<R>(psi + (int64_t)r * g.V * 12, x, ps);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int sp = 0; sp < 4; ++sp) {
        const cx<double> w = gg(mu, nu, s, sp);
        if (w.re == 0.0 && w.im == 0.0) continue;
        const cx<R> wr = mk<R>((R)w.re, (R)w.im);
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
          for (int a = 0; a < 3; ++a)
            T.m[3 * b + a] = cfmac(ph[3 * s + a], cmul(wr, ps[3 * sp + b]), T.m[3 * b + a]);
      }
  }
  // T' = 2 (T - T^H) scaled by -(c_sw / 32)
  M3<R> Tp;
  const R f = (R)(-2.0 * csw / 32.0);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      Tp.m[3 * i + j] = f * mk(T.m[3 * i + j].re - T.m[3 * j + i].re, T.m[3 * i + j].im + T.m[3 * j + i].im);
  // the four leaves of Q_munu(x), Eq. 1.12.  Factor k of leaf l sits at
  // c + dm mu^ + dn nu^ (the offsets below), points along mu when l + k is
  // even (else nu), and enters daggered when (l + k) mod 4 >= 2:
  //   l = 0: U_mu(c) U_nu(c+mu) U_mu(c+nu)^H U_nu(c)^H
  //   l = 1: U_nu(c) U_mu(c-mu+nu)^H U_nu(c-mu)^H U_mu(c-mu)
  //   l = 2: U_mu(c-mu)^H U_nu(c-mu-nu)^H U_mu(c-mu-nu) U_nu(c-nu)
  //   l = 3: U_nu(c-nu)^H U_mu(c-nu) U_nu(c-nu+mu) U_mu(c)^H
  constexpr signed char kDm[4][4] = {{0, 1, 0, 0}, {0, -1, -1, -1}, {-1, -1, -1, 0}, {0, 0, 1, 0}};
  constexpr signed char kDn[4][4] = {{0, 0, 1, 0}, {0, 1, 0, 0}, {0, -1, -1, -1}, {-1, -1, -1, 0}};
  for (int l = 0; l < 4; ++l) {
    M3<R> F[4];
    int fs[4][4];  // factor sites (coordinates)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int dm = kDm[l][k], dn = kDn[l][k];
#pragma unroll
      for (int i = 0; i < 4; ++i) fs[k][i] = c[i];
      fs[k][mu] = (c[mu] + dm + g.n[mu]) % g.n[mu];
      fs[k][nu] = (c[nu] + dn + g.n[nu]) % g.n[nu];
      const M3<R> u = load_link<R>(g, U, fs[k], ((l + k) & 1) ? nu : mu);
      F[k] = ((l + k) & 3) >= 2 ? mdag(u) : u;
    }
    auto dirk = [&](int k) { return ((l + k) & 1) ? nu : mu; };
    auto plain = [&](int k) { return ((l + k) & 3) < 2; };  // factor k is U (not U^H)
    // R_k = F_{k+1} .. F_3 T' F_0 .. F_{k-1} from the suffix products
    // S_k = F_{k+1} .. F_3 T' and the prefix products P_k = F_0 .. F_{k-1}:
    // eight 3x3 products per leaf instead of twelve
    const M3<R> S2 = mmul(F[3], Tp);
    const M3<R> S1 = mmul(F[2], S2);
    emit(fs[0], dirk(0), mmul(F[1], S1), plain(0));
    emit(fs[1], dirk(1), mmul(S1, F[0]), plain(1));
    const M3<R> P2 = mmul(F[0], F[1]);
    emit(fs[2], dirk(2), mmul(S2, P2), plain(2));
    emit(fs[3], dirk(3), mmul(Tp, mmul(P2, F[2])), plain(3));
  }
}

// One thread per site and plane (mu, nu) (grid row blockIdx.y): self-coupling
// contribution, accumulated atomically in G (FP64 atomics) or in the padded
// FP32 workspace (16-byte vector reductions).
template <typename R, typename GT, typename UT, typename ST>
__global__ void k_force_clover(FGeom g, const UT* __restrict__ U, const ST* __restrict__ phi,
                               const ST* __restrict__ psi, int nrhs, double csw, GT* G) {
  constexpr int kStride = sizeof(GT) == sizeof(float) ? kGf : 9;  // elements of GT per link
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.V) return;
  int c[4];
  coords_of(g, x, c);
  auto emit = [&](const int* sc, int d, const M3<R>& Rk, bool dagger) {
    const int lex = ((sc[0] * g.n[1] + sc[1]) * g.n[2] + sc[2]) * g.n[3] + sc[3];
    atomic_add_m3(G + ((int64_t)lex * 4 + d) * kStride, Rk, dagger);
  };
  // one plane (mu, nu) per grid row: every index into the coordinate arrays
  // is a compile-time constant
  switch (blockIdx.y) {
    case 0: clover_plane_leaves<R, 0, 1>(g, U, phi, psi, nrhs, csw, c, emit); break;
    case 1: clover_plane_leaves<R, 0, 2>(g, U, phi, psi, nrhs, csw, c, emit); break;
    case 2: clover_plane_leaves<R, 0, 3>(g, U, phi, psi, nrhs, csw, c, emit); break;
    case 3: clover_plane_leaves<R, 1, 2>(g, U, phi, psi, nrhs, csw, c, emit); break;
    case 4: clover_plane_leaves<R, 1, 3>(g, U, phi, psi, nrhs, csw, c, emit); break;
    default: clover_plane_leaves<R, 2, 3>(g, U, phi, psi, nrhs, csw, c, emit); break;
  }
}

__device__ __forceinline__ cx<double> load_g(const double2* G, int64_t t, int e) {
  return mk(G[t * 9 + e].x, G[t * 9 + e].y);
}
__device__ __forceinline__ cx<double> load_g(const float* G, int64_t t, int e) {
  return mk((double)G[t * kGf + 2 * e], (double)G[t * kGf + 2 * e + 1]);
}

// FP32 accumulator -> the caller's FP64 G
__global__ void k_force_widen(int64_t nlinks, const float* __restrict__ Gf, double2* G) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nlinks) return;
  for (int e = 0; e < 9; ++e) G[t * 9 + e] = make_double2((double)Gf[t * kGf + 2 * e], (double)Gf[t * kGf + 2 * e + 1]);
}

// F = P(G U^H), in R (FP64, or FP32 for the FP32 accumulator and links)
template <typename R, typename GT, typename UT>
__global__ void k_force_project(FGeom g, const UT* __restrict__ U, const GT* __restrict__ G, double2* F) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.V * 4) return;
  const int x = (int)(t >> 2), mu = (int)(t & 3);
  int c[4];
  coords_of(g, x, c);
  M3<R> u = load_link<R>(g, U, c, mu), gm;
  for (int e = 0; e < 9; ++e) {
    const cx<double> v = load_g(G, t, e);
    gm.m[e] = mk<R>((R)v.re, (R)v.im);
  }
  M3<R> M = mmul(gm, mdag(u));
  cx<R> f[9];
  const R half = (R)0.5, third = (R)(1.0 / 3.0);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      f[3 * i + j] = mk(half * (M.m[3 * i + j].re - M.m[3 * j + i].re), half * (M.m[3 * i + j].im + M.m[3 * j + i].im));
  const cx<R> tr = mk((f[0].re + f[4].re + f[8].re) * third, (f[0].im + f[4].im + f[8].im) * third);
  for (int i = 0; i < 3; ++i) f[4 * i] = f[4 * i] - tr;
  for (int e = 0; e < 9; ++e) F[t * 9 + e] = make_double2((double)f[e].re, (double)f[e].im);
}

}  // namespace

int force(dd_clover* op, int prec, const double* phi, const double* psi, int nrhs, int with_clover, double* G,
          double* F, cudaStream_t st) {
  const dd_lattice* lat = op->lat;
  const FGeom g = fgeom(lat);
  const double2* ph = reinterpret_cast<const double2*>(phi);
  const double2* ps = reinterpret_cast<const double2*>(psi);
  const double2* U64 = reinterpret_cast<const double2*>(op->gauge->links[0].ptr);
  const int64_t nl = lat->V * 4;
  const unsigned bl = (unsigned)((nl + 127) / 128);
  const unsigned bs = (unsigned)((lat->V + 63) / 64);
  const bool clover = with_clover && op->csw != 0.0;
  if (prec == P64) {
    DevBuf gtmp;
    double2* Gd = reinterpret_cast<double2*>(G);
    if (!Gd) {
      DD_TRY(gtmp.alloc((size_t)nl * 9 * sizeof(double2)));
      Gd = reinterpret_cast<double2*>(gtmp.ptr);
    }
    k_force_hop<double, double2, double2><<<bl, 128, 0, st>>>(g, ph, ps, nrhs, Gd);
    if (clover) k_force_clover<double, double2, double2, double2><<<dim3(bs, 6), 64, 0, st>>>(g, U64, ph, ps, nrhs, op->csw, Gd);
    if (F) k_force_project<double, double2, double2><<<bl, 128, 0, st>>>(g, U64, Gd, reinterpret_cast<double2*>(F));
    DD_CUDA(cudaGetLastError());
    if (!G) DD_CUDA(cudaStreamSynchronize(st));  // the temporary G is released on return
    return DD_OK;
  }
  // FP32: the spinors converted once to FP32 (canonical), the links read from
  // the FP32 native copy when the gauge handle has one; accumulate in the
  // operator's padded FP32 workspace (vector reductions), then widen into G
  // and / or project into F in FP32
  const size_t nsp = (size_t)nrhs * lat->V * 12;
  DD_TRY(op->ws_force.ensure((size_t)nl * kGf * sizeof(float) + 2 * nsp * sizeof(float2)));
  float* Gf = reinterpret_cast<float*>(op->ws_force.ptr);
  float2* ph32 = reinterpret_cast<float2*>(Gf + (size_t)nl * kGf);
  float2* ps32 = ph32 + nsp;
  const unsigned bc = (unsigned)((nsp + 255) / 256);
  k_canon_to_f32<<<bc, 256, 0, st>>>((int64_t)nsp, ph, ph32);
  k_canon_to_f32<<<bc, 256, 0, st>>>((int64_t)nsp, ps, ps32);
  k_force_hop<float, float, float2><<<bl, 128, 0, st>>>(g, ph32, ps32, nrhs, Gf);
  const float2* U32 = reinterpret_cast<const float2*>(op->gauge->links[1].ptr);
  if (U32) {
    if (clover) k_force_clover<float, float, float2, float2><<<dim3(bs, 6), 64, 0, st>>>(g, U32, ph32, ps32, nrhs, op->csw, Gf);
    if (F) k_force_project<float, float, float2><<<bl, 128, 0, st>>>(g, U32, Gf, reinterpret_cast<double2*>(F));
  } else {
    if (clover) k_force_clover<float, float, double2, float2><<<dim3(bs, 6), 64, 0, st>>>(g, U64, ph32, ps32, nrhs, op->csw, Gf);
    if (F) k_force_project<float, float, double2><<<bl, 128, 0, st>>>(g, U64, Gf, reinterpret_cast<double2*>(F));
  }
  if (G) k_force_widen<<<bl, 128, 0, st>>>(nl, Gf, reinterpret_cast<double2*>(G));
  DD_CUDA(cudaGetLastError());
  return DD_OK;
}

}  // namespace dd
