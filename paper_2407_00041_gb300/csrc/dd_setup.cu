// Setup kernels: native link layout, self-coupling construction (Eq. 1.11,
// 1.12, 2.5) and inversion, precision copies, and canonical <-> native field
// conversion.
#include <cstring>

#include "dd_internal.h"
#include "dd_link8.cuh"
#include "dd_pair.cuh"

namespace dd {

namespace {

struct LexGeom {
  int n[4];
  int stride[4];
  int64_t Vh;
};

LexGeom lex_geom(const dd_lattice* lat) {
  LexGeom g;
  for (int i = 0; i < 4; ++i) g.n[i] = lat->dims[i];
  g.stride[3] = 1;
  g.stride[2] = g.n[3];
  g.stride[1] = g.n[3] * g.n[2];
  g.stride[0] = g.n[3] * g.n[2] * g.n[1];
  g.Vh = lat->Vh;
  return g;
}

__device__ __forceinline__ void lex_to_coords(const LexGeom& g, int lex, int c[4]) {
  c[3] = lex % g.n[3];
  int r = lex / g.n[3];
  c[2] = r % g.n[2];
  r /= g.n[2];
  c[1] = r % g.n[1];
  c[0] = r / g.n[1];
}

__device__ __forceinline__ int coords_to_lex(const LexGeom& g, const int c[4]) {
  return ((c[0] * g.n[1] + c[1]) * g.n[2] + c[2]) * g.n[3] + c[3];
}

// ---------------------------------------------------------------- links
// Store link (lex, mu), nine complex elements row-major, in every native
// copy that exists (U32 / U16 may be null).
__device__ __forceinline__ void put_link_native(const LexGeom& g, int lex, int mu, const double2 v[9], double2* U64,
                                                float2* U32, __half2* U16) {
  int c[4];
  lex_to_coords(g, lex, c);
  const int p = (c[0] + c[1] + c[2] + c[3]) & 1;
  const int64_t s = lex >> 1;
  const int64_t base = (int64_t)p * 36 * g.Vh + (int64_t)mu * 9 * g.Vh + s;
  // FP32 / FP16 copies: element E = 9 mu + e in 16-byte groups of 2 / 4
  const int64_t pbase = (int64_t)p * 36 * g.Vh;
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    U64[base + e * g.Vh] = v[e];
    const int E = 9 * mu + e;
    if (U32) U32[pbase + ((int64_t)(E >> 1) * g.Vh + s) * 2 + (E & 1)] = make_float2((float)v[e].x, (float)v[e].y);
    if (U16)
      U16[pbase + ((int64_t)(E >> 2) * g.Vh + s) * 4 + (E & 3)] = __floats2half2_rn((float)v[e].x, (float)v[e].y);
  }
}

__global__ void k_links_to_native(LexGeom g, const double2* __restrict__ Uc, double2* U64, float2* U32,
                                  __half2* U16) {
  const int64_t V = 2 * g.Vh;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= V * 4) return;
  double2 v[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) v[e] = Uc[t * 9 + e];
  put_link_native(g, (int)(t >> 2), (int)(t & 3), v, U64, U32, U16);
}

// ---------------------------------------------------------------- link generator
// Counter-based synthetic links (not part of the thesis; it stands in for its
// gauge configurations).  SplitMix64 (Steele, Lea and Flood, "Fast splittable
// pseudorandom number generators", 2014) keyed by the seed gives word k of
// the stream as mix64(mix64(seed) + (k + 1) * golden gamma); pair k of
// uniforms u1 = ((word(2k) >> 11) + 1) 2^-53 in (0, 1], u2 = (word(2k+1) >> 11)
// 2^-53 turns into one complex Gaussian by Box-Muller,
// sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2).  Link (x, mu) uses pairs
// (4 x + mu) 9 + j, j = 0..8, as the entries of a 3x3 matrix A; with
// H = (A + A^H) / 2 - tr / 3 (traceless Hermitian) the link is U = exp(i eps H),
// special unitary.  The exponential is scaling and squaring of a 14-term
// Taylor series in Horner form (Higham 2005), exact to rounding here.
__device__ __forceinline__ uint64_t gen_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double2 gen_normal_pair(uint64_t key, uint64_t pair) {
  const uint64_t w1 = gen_mix64(key + (2 * pair + 1ULL) * 0x9E3779B97F4A7C15ULL);
  const uint64_t w2 = gen_mix64(key + (2 * pair + 2ULL) * 0x9E3779B97F4A7C15ULL);
  const double two53 = 1.0 / 9007199254740992.0;
  const double u1 = (double)((w1 >> 11) + 1ULL) * two53;
  const double u2 = (double)(w2 >> 11) * two53;
  const double r = sqrt(-2.0 * log(u1));
  double sn, cs;
  sincos(6.283185307179586476925286766559 * u2, &sn, &cs);
  return make_double2(r * cs, r * sn);
}

// C = A B for 3x3 complex matrices (row-major); C may alias neither operand
__device__ __forceinline__ void gen_m3_mul(const double2* A, const double2* B, double2* C) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      double re = 0.0, im = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double2 x = A[3 * a + k], y = B[3 * k + b];
        re += x.x * y.x - x.y * y.y;
        im += x.x * y.y + x.y * y.x;
      }
      C[3 * a + b] = make_double2(re, im);
    }
}

__global__ void k_links_generate(LexGeom g, uint64_t key, double eps, double2* U64, float2* U32, __half2* U16) {
  const int64_t V = 2 * g.Vh;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= V * 4) return;
  double2 A[9], X[9];
#pragma unroll
  for (int j = 0; j < 9; ++j) A[j] = gen_normal_pair(key, (uint64_t)t * 9ULL + (uint64_t)j);
  // X = i eps H, H = (A + A^H) / 2 - (tr / 3) I
  double tr = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) tr += A[4 * a].x;
  tr /= 3.0;
  double nrm = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      double hre = 0.5 * (A[3 * a + b].x + A[3 * b + a].x);
      const double him = 0.5 * (A[3 * a + b].y - A[3 * b + a].y);
      if (a == b) hre -= tr;
      X[3 * a + b] = make_double2(-eps * him, eps * hre);
      nrm += X[3 * a + b].x * X[3 * a + b].x + X[3 * a + b].y * X[3 * a + b].y;
    }
  nrm = sqrt(nrm);
  int k = 0;
  double scale = 1.0;
  while (nrm * scale > 0.25) {
    scale *= 0.5;
    ++k;
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) X[i] = make_double2(X[i].x * scale, X[i].y * scale);
  double2 E[9], T[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) E[i] = make_double2(i % 4 == 0 ? 1.0 : 0.0, 0.0);
  for (int n = 14; n >= 1; --n) {
    gen_m3_mul(X, E, T);
#pragma unroll
    for (int i = 0; i < 9; ++i) E[i] = make_double2(T[i].x / (double)n + (i % 4 == 0 ? 1.0 : 0.0), T[i].y / (double)n);
  }
  for (int s = 0; s < k; ++s) {
    gen_m3_mul(E, E, T);
#pragma unroll
    for (int i = 0; i < 9; ++i) E[i] = T[i];
  }
  put_link_native(g, (int)(t >> 2), (int)(t & 3), E, U64, U32, U16);
}

// max(|U U^H - 1|, |det U - 1|) of every link, reduced with an atomic max on
// the bit pattern of the (non-negative) float
__global__ void k_su3_deviation(int64_t nlinks, const double2* __restrict__ U64, int64_t Vh, unsigned* out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float dev = 0.f;
  if (t < nlinks) {
    // t = (parity * 4 + mu) * Vh + s
    const int64_t s = t % Vh, pm = t / Vh;
    const double2* b = U64 + pm * 9 * Vh + s;
    double2 u[9];
    for (int e = 0; e < 9; ++e) u[e] = b[e * Vh];
    double m = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double re = 0.0, im = 0.0;  // (U U^H)_ij
        for (int k = 0; k < 3; ++k) {
          const double2 a = u[3 * i + k], c = u[3 * j + k];
          re += a.x * c.x + a.y * c.y;
          im += a.y * c.x - a.x * c.y;
        }
        if (i == j) re -= 1.0;
        m = fmax(m, fmax(fabs(re), fabs(im)));
      }
    auto cm = [](double2 a, double2 c) { return make_double2(a.x * c.x - a.y * c.y, a.x * c.y + a.y * c.x); };
    auto cs = [](double2 a, double2 c) { return make_double2(a.x - c.x, a.y - c.y); };
    const double2 m0 = cs(cm(u[4], u[8]), cm(u[5], u[7]));
    const double2 m1 = cs(cm(u[5], u[6]), cm(u[3], u[8]));
    const double2 m2 = cs(cm(u[3], u[7]), cm(u[4], u[6]));
    const double2 det = make_double2(cm(u[0], m0).x + cm(u[1], m1).x + cm(u[2], m2).x,
                                     cm(u[0], m0).y + cm(u[1], m1).y + cm(u[2], m2).y);
    m = fmax(m, fmax(fabs(det.x - 1.0), fabs(det.y)));
    dev = isfinite(m) ? (float)fmin(m, 1e30) : 1e30f;
  }
  // block max, then one atomic per block
  __shared__ float red[256];
  red[threadIdx.x] = dev;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicMax(out, __float_as_uint(red[0]));
}

// FP32 copy with rows 0 and 1: element E = 6 mu + e (e < 6) of a site in
// float4 group E / 2, [parity][12 groups][Vh]
__global__ void k_links_recon32(int64_t nlinks, const double2* __restrict__ U64, int64_t Vh, float2* U32) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nlinks) return;
  const int64_t s = t % Vh, pm = t / Vh;
  const int64_t p = pm / 4, mu = pm % 4;
  const double2* b = U64 + pm * 9 * Vh + s;
  for (int e = 0; e < 6; ++e) {
    const double2 v = b[e * Vh];
    const int64_t E = 6 * mu + e;
    U32[p * 24 * Vh + ((E >> 1) * Vh + s) * 2 + (E & 1)] = make_float2((float)v.x, (float)v.y);
  }
}

// FP16 copy with rows 0 and 1: element E = 6 mu + e (e < 6) of a site in
// slot E % 4 of uint4 group E / 4, [parity][6 groups][Vh], rounded as the
// three-row FP16 links
__global__ void k_links_recon16(int64_t nlinks, const double2* __restrict__ U64, int64_t Vh, __half2* U16) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nlinks) return;
  const int64_t s = t % Vh, pm = t / Vh;
  const int64_t p = pm / 4, mu = pm % 4;
  const double2* b = U64 + pm * 9 * Vh + s;
  for (int e = 0; e < 6; ++e) {
    const double2 v = b[e * Vh];
    const int64_t E = 6 * mu + e;
    U16[p * 24 * Vh + ((E >> 2) * Vh + s) * 4 + (E & 3)] = __floats2half2_rn((float)v.x, (float)v.y);
  }
}

// Eight-real FP32 copy: link (parity p, mu) of site s in float4 groups
// 2 mu, 2 mu + 1 of [p][8 groups][Vh] (dd_link8.cuh)
__global__ void k_links_recon8(int64_t nlinks, const double2* __restrict__ U64, int64_t Vh, float4* U8) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nlinks) return;
  const int64_t s = t % Vh, pm = t / Vh;
  const int64_t p = pm / 4, mu = pm % 4;
  const double2* b = U64 + pm * 9 * Vh + s;
  double2 u[9];
  for (int e = 0; e < 9; ++e) u[e] = b[e * Vh];
  float4 w0, w1;
  link8_encode(u, w0, w1);
  U8[(p * 8 + 2 * mu) * Vh + s] = w0;
  U8[(p * 8 + 2 * mu + 1) * Vh + s] = w1;
}

// max |decoded - U| over the elements of every link (the decoder of the
// stencil), reduced like k_su3_deviation
__global__ void k_links_recon8_error(int64_t nlinks, const double2* __restrict__ U64, const float4* __restrict__ U8,
                                     int64_t Vh, unsigned* out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float dev = 0.f;
  if (t < nlinks) {
    const int64_t s = t % Vh, pm = t / Vh;
    const int64_t p = pm / 4, mu = pm % 4;
    float2 u[9];
    link8_decode(U8[(p * 8 + 2 * mu) * Vh + s], U8[(p * 8 + 2 * mu + 1) * Vh + s], u);
    const double2* b = U64 + pm * 9 * Vh + s;
    double m = 0.0;
    for (int e = 0; e < 9; ++e) {
      const double2 v = b[e * Vh];
      m = fmax(m, fmax(fabs((double)u[e].x - v.x), fabs((double)u[e].y - v.y)));
    }
    dev = isfinite(m) ? (float)fmin(m, 1e30) : 1e30f;
  }
  __shared__ float red[256];
  red[threadIdx.x] = dev;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicMax(out, __float_as_uint(red[0]));
}

// FP64 complex elements -> FP32 pairs (re.h, re.l, im.h, im.l), the same
// element order (links, self-coupling blocks, A_ee^-1)
__global__ void k_split_pairs(int64_t n, const double2* __restrict__ in, float4* out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const double2 v = in[t];
  const df re(v.x), im(v.y);
  out[t] = make_float4(re.h, re.l, im.h, im.l);
}

__global__ void k_links_to_canonical(LexGeom g, const double2* __restrict__ U64, double2* Uc) {
  const int64_t V = 2 * g.Vh;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= V * 4) return;
  const int lex = (int)(t >> 2), mu = (int)(t & 3);
  int c[4];
  lex_to_coords(g, lex, c);
  const int p = (c[0] + c[1] + c[2] + c[3]) & 1;
  const int64_t base = (int64_t)p * 36 * g.Vh + (int64_t)mu * 9 * g.Vh + (lex >> 1);
  for (int e = 0; e < 9; ++e) Uc[t * 9 + e] = U64[base + e * g.Vh];
}

// ---------------------------------------------------------------- 3x3 algebra (FP64)
struct M3 {
  cx<double> m[9];
};

__device__ __forceinline__ M3 m3_load(const LexGeom& g, const double2* U64, const int c[4], int mu) {
  const int lex = coords_to_lex(g, c);
  const int p = (c[0] + c[1] + c[2] + c[3]) & 1;
  const double2* b = U64 + (int64_t)p * 36 * g.Vh + (int64_t)mu * 9 * g.Vh + (lex >> 1);
  M3 r;
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    double2 v = b[e * g.Vh];
    r.m[e] = mk(v.x, v.y);
  }
  return r;
}

__device__ __forceinline__ M3 m3_dag(const M3& a) {
  M3 r;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) r.m[3 * i + j] = mk(a.m[3 * j + i].re, -a.m[3 * j + i].im);
  return r;
}

__device__ __forceinline__ M3 m3_mul(const M3& a, const M3& b) {
  M3 r;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cx<double> acc = zero<double>();
#pragma unroll
      for (int k = 0; k < 3; ++k) acc = cfma(a.m[3 * i + k], b.m[3 * k + j], acc);
      r.m[3 * i + j] = acc;
    }
  return r;
}

__device__ __forceinline__ void shifted(const LexGeom& g, const int c[4], int mu, int d, int out[4]) {
  for (int i = 0; i < 4; ++i) out[i] = c[i];
  out[mu] = (c[mu] + d + g.n[mu]) % g.n[mu];
}

// Q_munu(x), Eq. 1.12: the four plaquettes in the mu-nu plane that start and
// end at x (gauge links are periodic).
__device__ M3 clover_leaves(const LexGeom& g, const double2* U, const int x[4], int mu, int nu) {
  int xpm[4], xpn[4], xmm[4], xmn[4], xmm_pn[4], xmm_mn[4], xmn_pm[4];
  shifted(g, x, mu, +1, xpm);
  shifted(g, x, nu, +1, xpn);
  shifted(g, x, mu, -1, xmm);
  shifted(g, x, nu, -1, xmn);
  shifted(g, xmm, nu, +1, xmm_pn);
  shifted(g, xmm, nu, -1, xmm_mn);
  shifted(g, xmn, mu, +1, xmn_pm);
  // U_mu(x) U_nu(x+mu) U_mu(x+nu)^H U_nu(x)^H
  M3 l = m3_mul(m3_mul(m3_load(g, U, x, mu), m3_load(g, U, xpm, nu)),
                m3_mul(m3_dag(m3_load(g, U, xpn, mu)), m3_dag(m3_load(g, U, x, nu))));
  M3 q = l;
  // U_nu(x) U_mu(x-mu+nu)^H U_nu(x-mu)^H U_mu(x-mu)
  l = m3_mul(m3_mul(m3_load(g, U, x, nu), m3_dag(m3_load(g, U, xmm_pn, mu))),
             m3_mul(m3_dag(m3_load(g, U, xmm, nu)), m3_load(g, U, xmm, mu)));
  for (int e = 0; e < 9; ++e) q.m[e] = q.m[e] + l.m[e];
  // U_mu(x-mu)^H U_nu(x-mu-nu)^H U_mu(x-mu-nu) U_nu(x-nu)
  l = m3_mul(m3_mul(m3_dag(m3_load(g, U, xmm, mu)), m3_dag(m3_load(g, U, xmm_mn, nu))),
             m3_mul(m3_load(g, U, xmm_mn, mu), m3_load(g, U, xmn, nu)));
  for (int e = 0; e < 9; ++e) q.m[e] = q.m[e] + l.m[e];
  // U_nu(x-nu)^H U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^H
  l = m3_mul(m3_mul(m3_dag(m3_load(g, U, xmn, nu)), m3_load(g, U, xmn, mu)),
             m3_mul(m3_load(g, U, xmn_pm, nu), m3_dag(m3_load(g, U, x, mu))));
  for (int e = 0; e < 9; ++e) q.m[e] = q.m[e] + l.m[e];
  return q;
}

// 2x2 spin blocks of the chiral basis: gamma_mu = [[0, B_mu], [B_mu^H, 0]]
__device__ __forceinline__ cx<double> Bmat(int mu, int i, int j) {
  // B_T = I, B_Z = diag(-i, i), B_Y = [[0, -1], [1, 0]], B_X = [[0, -i], [-i, 0]]
  if (mu == 0) return mk(i == j ? 1.0 : 0.0, 0.0);
  if (mu == 1) return i != j ? mk(0.0, 0.0) : mk(0.0, i == 0 ? -1.0 : 1.0);
  if (mu == 2) return i == j ? mk(0.0, 0.0) : mk(i == 0 ? -1.0 : 1.0, 0.0);
  return i == j ? mk(0.0, 0.0) : mk(0.0, -1.0);
}

// Element (i, j) of gamma_mu gamma_nu restricted to chirality block b:
// b = 0: B_mu B_nu^H, b = 1: B_mu^H B_nu.
__device__ __forceinline__ cx<double> gg_block(int b, int mu, int nu, int i, int j) {
  cx<double> acc = zero<double>();
  for (int k = 0; k < 2; ++k) {
    cx<double> x, y;
    if (b == 0) {
      x = Bmat(mu, i, k);
      cx<double> t = Bmat(nu, j, k);
      y = mk(t.re, -t.im);
    } else {
      cx<double> t = Bmat(mu, k, i);
      x = mk(t.re, -t.im);
      y = Bmat(nu, k, j);
    }
    acc = cfma(x, y, acc);
  }
  return acc;
}

// One thread per site: both 6x6 blocks of A(x) = (m0 + 4) I
//   - (c_sw / 16) sum_{mu < nu} (gamma_mu gamma_nu) (x) (Q_munu - Q_munu^H).
__global__ void k_clover_build(LexGeom g, const double2* __restrict__ U, double m0, double csw, double2* clov) {
  const int64_t V = 2 * g.Vh;
  const int lex = blockIdx.x * blockDim.x + threadIdx.x;
  if (lex >= V) return;
  int x[4];
  lex_to_coords(g, lex, x);
  const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
  const int64_t s = lex >> 1;
  cx<double> A[2][6][6];
  for (int b = 0; b < 2; ++b)
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) A[b][i][j] = mk(i == j ? m0 + 4.0 : 0.0, 0.0);
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = mu + 1; nu < 4; ++nu) {
      M3 Q = clover_leaves(g, U, x, mu, nu);
      M3 F;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
          F.m[3 * i + j] = mk(Q.m[3 * i + j].re - Q.m[3 * j + i].re, Q.m[3 * i + j].im + Q.m[3 * j + i].im);
      for (int b = 0; b < 2; ++b)
        for (int si = 0; si < 2; ++si)
          for (int sj = 0; sj < 2; ++sj) {
            cx<double> gg = gg_block(b, mu, nu, si, sj);
            if (gg.re == 0.0 && gg.im == 0.0) continue;
            for (int a = 0; a < 3; ++a)
              for (int c = 0; c < 3; ++c) {
                cx<double> t = cmul(gg, F.m[3 * a + c]);
                A[b][3 * si + a][3 * sj + c] = A[b][3 * si + a][3 * sj + c] - (csw / 16.0) * t;
              }
          }
    }
  double2* out = clov + (int64_t)p * 36 * g.Vh + s;
  for (int b = 0; b < 2; ++b) {
    double2* o = out + (int64_t)18 * b * g.Vh;
    for (int k = 0; k < 3; ++k) o[k * g.Vh] = make_double2(A[b][2 * k][2 * k].re, A[b][2 * k + 1][2 * k + 1].re);
    int k = 3;
    for (int i = 0; i < 6; ++i)
      for (int j = i + 1; j < 6; ++j, ++k) o[k * g.Vh] = make_double2(A[b][i][j].re, A[b][i][j].im);
  }
}

__device__ void unpack_block(const double2* m, int64_t Vh, cx<double> A[6][6]) {
  for (int k = 0; k < 3; ++k) {
    double2 d = m[k * Vh];
    A[2 * k][2 * k] = mk(d.x, 0.0);
    A[2 * k + 1][2 * k + 1] = mk(d.y, 0.0);
  }
  int k = 3;
  for (int i = 0; i < 6; ++i)
    for (int j = i + 1; j < 6; ++j, ++k) {
      double2 v = m[k * Vh];
      A[i][j] = mk(v.x, v.y);
      A[j][i] = mk(v.x, -v.y);
    }
}

// A_ee^{-1}: Gauss-Jordan elimination with partial pivoting on each 6x6 block
// of every even site.  A block whose pivot falls below 1e-12 of the block's
// largest entry raises `flag`.
__global__ void k_clover_invert(int64_t Vh, const double2* __restrict__ clov_even, double2* ainv, int* flag) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= Vh) return;
  for (int b = 0; b < 2; ++b) {
    cx<double> A[6][6], X[6][6];
    unpack_block(clov_even + (int64_t)18 * b * Vh + s, Vh, A);
    double amax = 0.0;
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) {
        X[i][j] = mk(i == j ? 1.0 : 0.0, 0.0);
        amax = fmax(amax, fabs(A[i][j].re) + fabs(A[i][j].im));
      }
    for (int col = 0; col < 6; ++col) {
      int piv = col;
      double best = -1.0;
      for (int r = col; r < 6; ++r) {
        double m = A[r][col].re * A[r][col].re + A[r][col].im * A[r][col].im;
        if (m > best) {
          best = m;
          piv = r;
        }
      }
      if (!(sqrt(best) > 1e-12 * amax)) {
        atomicExch(flag, 1);
        return;
      }
      if (piv != col)
        for (int j = 0; j < 6; ++j) {
          cx<double> t = A[col][j];
          A[col][j] = A[piv][j];
          A[piv][j] = t;
          t = X[col][j];
          X[col][j] = X[piv][j];
          X[piv][j] = t;
        }
      const cx<double> d = A[col][col];
      const double dn = d.re * d.re + d.im * d.im;
      const cx<double> inv = mk(d.re / dn, -d.im / dn);
      for (int j = 0; j < 6; ++j) {
        A[col][j] = cmul(inv, A[col][j]);
        X[col][j] = cmul(inv, X[col][j]);
      }
      for (int r = 0; r < 6; ++r) {
        if (r == col) continue;
        const cx<double> f = A[r][col];
        for (int j = 0; j < 6; ++j) {
          A[r][j] = A[r][j] - cmul(f, A[col][j]);
          X[r][j] = X[r][j] - cmul(f, X[col][j]);
        }
      }
    }
    double2* o = ainv + (int64_t)18 * b * Vh + s;
    for (int k = 0; k < 3; ++k) o[k * Vh] = make_double2(X[2 * k][2 * k].re, X[2 * k + 1][2 * k + 1].re);
    int k = 3;
    for (int i = 0; i < 6; ++i)
      for (int j = i + 1; j < 6; ++j, ++k) o[k * Vh] = make_double2(X[i][j].re, X[i][j].im);
  }
}

// Block arrays [nsets][36 elements][Vh] (FP64) -> 16-byte groups
// [nsets][36 / PER][Vh] with PER = 2 (FP32, float4) or 4 (FP16, 8 halves).
__global__ void k_group32(const double2* __restrict__ in, float4* out, int64_t nsets, int64_t Vh) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // over nsets * 18 * Vh
  if (t >= nsets * 18 * Vh) return;
  const int64_t s = t % Vh, g = (t / Vh) % 18, set = t / (18 * Vh);
  const double2 a = in[(set * 36 + 2 * g) * Vh + s], b = in[(set * 36 + 2 * g + 1) * Vh + s];
  out[t] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
}
__global__ void k_group16(const double2* __restrict__ in, uint4* out, int64_t nsets, int64_t Vh) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // over nsets * 9 * Vh
  if (t >= nsets * 9 * Vh) return;
  const int64_t s = t % Vh, g = (t / Vh) % 9, set = t / (9 * Vh);
  unsigned int w[4];
  for (int q = 0; q < 4; ++q) {
    const double2 v = in[(set * 36 + 4 * g + q) * Vh + s];
    __half2 h = __floats2half2_rn((float)v.x, (float)v.y);
    w[q] = *reinterpret_cast<unsigned int*>(&h);
  }
  out[t] = make_uint4(w[0], w[1], w[2], w[3]);
}

__global__ void k_clover_dense(LexGeom g, const double2* __restrict__ clov, double2* A) {
  const int64_t V = 2 * g.Vh;
  const int lex = blockIdx.x * blockDim.x + threadIdx.x;
  if (lex >= V) return;
  int x[4];
  lex_to_coords(g, lex, x);
  const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
  double2* o = A + (int64_t)lex * 144;
  for (int i = 0; i < 144; ++i) o[i] = make_double2(0.0, 0.0);
  for (int b = 0; b < 2; ++b) {
    cx<double> B[6][6];
    unpack_block(clov + (int64_t)p * 36 * g.Vh + (int64_t)18 * b * g.Vh + (lex >> 1), g.Vh, B);
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) o[(6 * b + i) * 12 + 6 * b + j] = make_double2(B[i][j].re, B[i][j].im);
  }
}

// ---------------------------------------------------------------- fields
struct PackArgs {
  LexGeom g;
  int nrhs;
  int subset;  // 0 full, 1 odd, 2 even
  int p0, npar;
  int64_t gstride;
  HalfField h[2];
  int64_t s0, ns;  // compact sites s0 .. s0 + ns - 1 of each parity (a range of time slices)
};

__device__ __forceinline__ int64_t canon_offset(const PackArgs& a, int p, int64_t s, int r) {
  if (a.subset == 0 || a.subset >= 3) {  // full-lattice canonical array
    // lexicographic index of compact site s of parity p
    const int lex2 = (int)(2 * s);
    const int r1 = lex2 / a.g.n[3];
    const int x0 = lex2 - r1 * a.g.n[3];
    const int r2 = r1 / a.g.n[2];
    const int y = r1 - r2 * a.g.n[2];
    const int t = r2 / a.g.n[1];
    const int z = r2 - t * a.g.n[1];
    const int lex = r1 * a.g.n[3] + x0 + ((p ^ (t + z + y)) & 1);
    return ((int64_t)r * 2 * a.g.Vh + lex) * 12;
  }
  return ((int64_t)r * a.g.Vh + s) * 12;
}

// CT: the canonical element, double2 (complex128) or float2 (complex64)
template <int P, typename CT = double2>
__global__ void k_pack(PackArgs a, const CT* __restrict__ canon) {
  using R = typename SpinorStore<P>::real;
  const int64_t nper = a.ns * a.nrhs;
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nper * a.npar) return;
  int p = a.p0;
  if (t >= nper) {
    t -= nper;
    p ^= 1;
  }
  t += a.s0 * a.nrhs;
  const int64_t s = t / a.nrhs;
  const int r = (int)(t - s * a.nrhs);
  const CT* src = canon + canon_offset(a, p, s, r);
  cx<R> v[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    const CT d = src[c];
    v[c] = mk<R>((R)d.x, (R)d.y);
  }
  store_spinor<P, R>(a.h[p], a.gstride, t, v);
}

template <int P, typename CT = double2>
__global__ void k_unpack(PackArgs a, CT* canon) {
  using R = typename SpinorStore<P>::real;
  const int64_t nper = a.ns * a.nrhs;
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nper * a.npar) return;
  int p = a.p0;
  if (t >= nper) {
    t -= nper;
    p ^= 1;
  }
  t += a.s0 * a.nrhs;
  const int64_t s = t / a.nrhs;
  const int r = (int)(t - s * a.nrhs);
  cx<R> v[12];
  load_spinor<P, R>(a.h[p], a.gstride, t, v);
  CT* dst = canon + canon_offset(a, p, s, r);
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    if constexpr (std::is_same<CT, float2>::value)
      dst[c] = make_float2((float)v[c].re, (float)v[c].im);
    else
      dst[c] = make_double2((double)v[c].re, (double)v[c].im);
  }
}

// The paired-RHS layouts (dd_pair.cuh): one thread per (site, RHS pair j),
// which holds RHS 2j and 2j + 1; a.gstride = Vh * nrhs / 2.
template <int P>
__global__ void k_pack_pair(PackArgs a, const double2* __restrict__ canon) {
  const int NP = a.nrhs >> 1;
  const int64_t nper = a.ns * NP;
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nper * a.npar) return;
  int p = a.p0;
  if (t >= nper) {
    t -= nper;
    p ^= 1;
  }
  t += a.s0 * NP;
  const int64_t s = t / NP;
  const int j = (int)(t - s * NP);
  const double2* sa = canon + canon_offset(a, p, s, 2 * j);
  const double2* sb = canon + canon_offset(a, p, s, 2 * j + 1);
  cx2 v[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    const double2 da = sa[c], db = sb[c];
    v[c].re = make_float2((float)da.x, (float)db.x);
    v[c].im = make_float2((float)da.y, (float)db.y);
  }
  store_pair<P, false>(a.h[p], a.gstride, t, v);
}

template <int P>
__global__ void k_unpack_pair(PackArgs a, double2* canon) {
  const int NP = a.nrhs >> 1;
  const int64_t nper = a.ns * NP;
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nper * a.npar) return;
  int p = a.p0;
  if (t >= nper) {
    t -= nper;
    p ^= 1;
  }
  t += a.s0 * NP;
  const int64_t s = t / NP;
  const int j = (int)(t - s * NP);
  cx2 v[12];
  const float2 sc = load_pair<P>(a.h[p], a.gstride, t, v);
  double2* da = canon + canon_offset(a, p, s, 2 * j);
  double2* db = canon + canon_offset(a, p, s, 2 * j + 1);
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    da[c] = make_double2((double)(v[c].re.x * sc.x), (double)(v[c].im.x * sc.x));
    db[c] = make_double2((double)(v[c].re.y * sc.y), (double)(v[c].im.y * sc.y));
  }
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

PackArgs pack_args(const dd_lattice* lat, int subset, const Field& f) {
  PackArgs a;
  a.g = lex_geom(lat);
  a.nrhs = f.nrhs;
  a.subset = subset;
  a.p0 = (subset == 1 || subset == 4) ? 1 : 0;
  a.npar = subset == 0 ? 2 : 1;
  a.gstride = lat->Vh * f.nrhs;
  a.h[0] = f.h[0];
  a.h[1] = f.h[1];
  a.s0 = 0;
  a.ns = lat->Vh;
  return a;
}

}  // namespace

int links_to_native(const dd_lattice* lat, const double* Uc, dd_gauge* g, cudaStream_t st) {
  const int64_t n = lat->V * 4;
  k_links_to_native<<<nblk(n, 128), 128, 0, st>>>(
      lex_geom(lat), reinterpret_cast<const double2*>(Uc), reinterpret_cast<double2*>(g->links[0].ptr),
      reinterpret_cast<float2*>(g->links[1].ptr), reinterpret_cast<__half2*>(g->links[2].ptr));
  DD_CUDA(cudaGetLastError());
  return DD_OK;
}

int links_generate(const dd_lattice* lat, uint64_t seed, double eps, dd_gauge* g, cudaStream_t st) {
  const int64_t n = lat->V * 4;
  // the stream key is mix64(seed), as in the host-side generator
  uint64_t z = seed;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  const uint64_t key = z ^ (z >> 31);
  k_links_generate<<<nblk(n, 128), 128, 0, st>>>(
      lex_geom(lat), key, eps, reinterpret_cast<double2*>(g->links[0].ptr),
      reinterpret_cast<float2*>(g->links[1].ptr), reinterpret_cast<__half2*>(g->links[2].ptr));
  DD_CUDA(cudaGetLastError());
  return DD_OK;
}

int links_su3_deviation(const dd_gauge* g, double* dev, cudaStream_t st) {
  const int64_t n = g->lat->V * 4;
  DevBuf out;
  DD_TRY(out.alloc(sizeof(unsigned)));
  DD_CUDA(cudaMemsetAsync(out.ptr, 0, sizeof(unsigned), st));
  k_su3_deviation<<<nblk(n, 256), 256, 0, st>>>(n, reinterpret_cast<const double2*>(g->links[0].ptr), g->lat->Vh,
                                                reinterpret_cast<unsigned*>(out.ptr));
  DD_CUDA(cudaGetLastError());
  unsigned bits = 0;
  DD_CUDA(cudaMemcpyAsync(&bits, out.ptr, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  DD_CUDA(cudaStreamSynchronize(st));
  float f;
  memcpy(&f, &bits, sizeof(f));
  *dev = f;
  return DD_OK;
}

int links_to_recon32(dd_gauge* g, cudaStream_t st) {
  const int64_t n = g->lat->V * 4;
  DD_TRY(g->links32r.alloc((size_t)g->lat->V * 24 * sizeof(float2)));
  k_links_recon32<<<nblk(n, 128), 128, 0, st>>>(n, reinterpret_cast<const double2*>(g->links[0].ptr), g->lat->Vh,
                                               reinterpret_cast<float2*>(g->links32r.ptr));
  DD_CUDA(cudaGetLastError());
  g->recon32 = 12;
  return DD_OK;
}

int links_to_recon16(dd_gauge* g, cudaStream_t st) {
  const int64_t n = g->lat->V * 4;
  DD_TRY(g->links16r.alloc((size_t)g->lat->V * 6 * sizeof(uint4)));
  k_links_recon16<<<nblk(n, 128), 128, 0, st>>>(n, reinterpret_cast<const double2*>(g->links[0].ptr), g->lat->Vh,
                                               reinterpret_cast<__half2*>(g->links16r.ptr));
  DD_CUDA(cudaGetLastError());
  g->recon16 = 12;
  return DD_OK;
}

int links_to_recon8(dd_gauge* g, double* dev, cudaStream_t st) {
  const int64_t n = g->lat->V * 4;
  DD_TRY(g->links32r.alloc((size_t)g->lat->V * 8 * sizeof(float4)));
  g->recon32 = 8;
  const double2* U64 = reinterpret_cast<const double2*>(g->links[0].ptr);
  float4* U8 = reinterpret_cast<float4*>(g->links32r.ptr);
  k_links_recon8<<<nblk(n, 128), 128, 0, st>>>(n, U64, g->lat->Vh, U8);
  DD_CUDA(cudaGetLastError());
  DevBuf out;
  DD_TRY(out.alloc(sizeof(unsigned)));
  DD_CUDA(cudaMemsetAsync(out.ptr, 0, sizeof(unsigned), st));
  k_links_recon8_error<<<nblk(n, 256), 256, 0, st>>>(n, U64, U8, g->lat->Vh, reinterpret_cast<unsigned*>(out.ptr));
  DD_CUDA(cudaGetLastError());
  unsigned bits = 0;
  DD_CUDA(cudaMemcpyAsync(&bits, out.ptr, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  DD_CUDA(cudaStreamSynchronize(st));
  float f;
  memcpy(&f, &bits, sizeof(f));
  *dev = f;
  return DD_OK;
}

int links_to_canonical(const dd_gauge* g, double* Uc, cudaStream_t st) {
  const int64_t n = g->lat->V * 4;
  k_links_to_canonical<<<nblk(n, 128), 128, 0, st>>>(lex_geom(g->lat),
                                                     reinterpret_cast<const double2*>(g->links[0].ptr),
                                                     reinterpret_cast<double2*>(Uc));
  DD_CUDA(cudaGetLastError());
  return DD_OK;
}

int clover_build(dd_clover* op, cudaStream_t st) {
  const dd_lattice* lat = op->lat;
  const int64_t Vh = lat->Vh;
  const int64_t nclov = 2 * 36 * Vh, nainv = 36 * Vh;
  DD_TRY(op->clov[0].alloc(nclov * sizeof(double2)));
  DD_TRY(op->ainv[0].alloc(nainv * sizeof(double2)));
  k_clover_build<<<nblk(lat->V, 64), 64, 0, st>>>(lex_geom(lat),
                                                  reinterpret_cast<const double2*>(op->gauge->links[0].ptr), op->m0,
                                                  op->csw, reinterpret_cast<double2*>(op->clov[0].ptr));
  DD_CUDA(cudaGetLastError());
  DevBuf flag;
  DD_TRY(flag.alloc(sizeof(int)));
  DD_CUDA(cudaMemsetAsync(flag.ptr, 0, sizeof(int), st));
  k_clover_invert<<<nblk(Vh, 64), 64, 0, st>>>(Vh, reinterpret_cast<const double2*>(op->clov[0].ptr),
                                                reinterpret_cast<double2*>(op->ainv[0].ptr),
                                                reinterpret_cast<int*>(flag.ptr));
  DD_CUDA(cudaGetLastError());
  int hflag = 0;
  DD_CUDA(cudaMemcpyAsync(&hflag, flag.ptr, sizeof(int), cudaMemcpyDeviceToHost, st));
  DD_CUDA(cudaStreamSynchronize(st));
  if (hflag) return fail(DD_ERR_SINGULAR, "an even-site self-coupling block is singular");
  if (op->prec_mask & P32) {
    DD_TRY(op->clov[1].alloc(nclov * sizeof(float2)));
    DD_TRY(op->ainv[1].alloc(nainv * sizeof(float2)));
    k_group32<<<nblk(2 * 18 * Vh, 256), 256, 0, st>>>((const double2*)op->clov[0].ptr, (float4*)op->clov[1].ptr, 2, Vh);
    k_group32<<<nblk(18 * Vh, 256), 256, 0, st>>>((const double2*)op->ainv[0].ptr, (float4*)op->ainv[1].ptr, 1, Vh);
  }
  if (op->prec_mask & P16) {
    DD_TRY(op->clov[2].alloc(nclov * sizeof(__half2)));
    DD_TRY(op->ainv[2].alloc(nainv * sizeof(__half2)));
    k_group16<<<nblk(2 * 9 * Vh, 256), 256, 0, st>>>((const double2*)op->clov[0].ptr, (uint4*)op->clov[2].ptr, 2, Vh);
    k_group16<<<nblk(9 * Vh, 256), 256, 0, st>>>((const double2*)op->ainv[0].ptr, (uint4*)op->ainv[2].ptr, 1, Vh);
  }
  if (op->prec_mask & PDF) {
    DD_TRY(op->clov[3].alloc(nclov * sizeof(float4)));
    DD_TRY(op->ainv[3].alloc(nainv * sizeof(float4)));
    k_split_pairs<<<nblk(nclov, 256), 256, 0, st>>>(nclov, (const double2*)op->clov[0].ptr, (float4*)op->clov[3].ptr);
    k_split_pairs<<<nblk(nainv, 256), 256, 0, st>>>(nainv, (const double2*)op->ainv[0].ptr, (float4*)op->ainv[3].ptr);
  }
  DD_CUDA(cudaGetLastError());
  return DD_OK;
}

int links_to_pairs(dd_gauge* g, cudaStream_t st) {
  const int64_t n = g->lat->V * 36;
  DD_TRY(g->links[3].alloc((size_t)n * sizeof(float4)));
  k_split_pairs<<<nblk(n, 256), 256, 0, st>>>(n, reinterpret_cast<const double2*>(g->links[0].ptr),
                                              reinterpret_cast<float4*>(g->links[3].ptr));
  DD_CUDA(cudaGetLastError());
  return DD_OK;
}

int clover_to_dense(const dd_clover* op, double* A_dev, cudaStream_t st) {
  k_clover_dense<<<nblk(op->lat->V, 64), 64, 0, st>>>(lex_geom(op->lat), (const double2*)op->clov[0].ptr,
                                                      reinterpret_cast<double2*>(A_dev));
  DD_CUDA(cudaGetLastError());
  return DD_OK;
}

template <typename CT>
int pack_native(const PackArgs& a, int prec, int nrhs, const CT* c, cudaStream_t st) {
  const int64_t n = a.ns * nrhs * a.npar;
  if (prec == P64)
    k_pack<P64, CT><<<nblk(n, 128), 128, 0, st>>>(a, c);
  else if (prec == PDF)
    k_pack<PDF, CT><<<nblk(n, 128), 128, 0, st>>>(a, c);
  else if (prec == P32)
    k_pack<P32, CT><<<nblk(n, 128), 128, 0, st>>>(a, c);
  else
    k_pack<P16, CT><<<nblk(n, 128), 128, 0, st>>>(a, c);
  DD_CUDA(cudaGetLastError());
  return DD_OK;
}

template <typename CT>
int unpack_native(const PackArgs& a, int prec, int nrhs, CT* c, cudaStream_t st) {
  const int64_t n = a.ns * nrhs * a.npar;
  if (prec == P64)
    k_unpack<P64, CT><<<nblk(n, 128), 128, 0, st>>>(a, c);
  else if (prec == PDF)
    k_unpack<PDF, CT><<<nblk(n, 128), 128, 0, st>>>(a, c);
  else if (prec == P32)
    k_unpack<P32, CT><<<nblk(n, 128), 128, 0, st>>>(a, c);
  else
    k_unpack<P16, CT><<<nblk(n, 128), 128, 0, st>>>(a, c);
  DD_CUDA(cudaGetLastError());
  return DD_OK;
}

int pack(const dd_lattice* lat, int prec, int subset, const double* canon, const Field& f, cudaStream_t st, int t0,
         int nt) {
  PackArgs a = pack_args(lat, subset, f);
  if (nt > 0) {  // time slices t0 .. t0 + nt - 1 of a full field
    const int64_t slice = (int64_t)lat->dims[1] * lat->dims[2] * lat->dims[3];
    a.s0 = t0 * slice / 2;
    a.ns = nt * slice / 2;
  }
  const double2* c = reinterpret_cast<const double2*>(canon);
  if (f.paired) {
    if (f.nrhs % 2 != 0 || (prec != P32 && prec != P16)) return fail(DD_ERR_ARG, "paired layout: FP32 / FP16, even nrhs");
    a.gstride = lat->Vh * (f.nrhs / 2);
    const int64_t np = a.ns * (f.nrhs / 2) * a.npar;
    if (prec == P32)
      k_pack_pair<P32><<<nblk(np, 128), 128, 0, st>>>(a, c);
    else
      k_pack_pair<P16><<<nblk(np, 128), 128, 0, st>>>(a, c);
    DD_CUDA(cudaGetLastError());
    return DD_OK;
  }
  return pack_native(a, prec, f.nrhs, c, st);
}

// complex64 canonical fields (native layout only)
int pack_c64(const dd_lattice* lat, int prec, int subset, const float* canon, const Field& f, cudaStream_t st,
             int t0, int nt) {
  if (f.paired) return fail(DD_ERR_ARG, "complex64 fields take the native layout");
  PackArgs a = pack_args(lat, subset, f);
  if (nt > 0) {
    const int64_t slice = (int64_t)lat->dims[1] * lat->dims[2] * lat->dims[3];
    a.s0 = t0 * slice / 2;
    a.ns = nt * slice / 2;
  }
  return pack_native(a, prec, f.nrhs, reinterpret_cast<const float2*>(canon), st);
}

int unpack(const dd_lattice* lat, int prec, int subset, const Field& f, double* canon, cudaStream_t st, int t0,
           int nt) {
  PackArgs a = pack_args(lat, subset, f);
  if (nt > 0) {
    const int64_t slice = (int64_t)lat->dims[1] * lat->dims[2] * lat->dims[3];
    a.s0 = t0 * slice / 2;
    a.ns = nt * slice / 2;
  }
  double2* c = reinterpret_cast<double2*>(canon);
  if (f.paired) {
    if (f.nrhs % 2 != 0 || (prec != P32 && prec != P16)) return fail(DD_ERR_ARG, "paired layout: FP32 / FP16, even nrhs");
    a.gstride = lat->Vh * (f.nrhs / 2);
    const int64_t np = a.ns * (f.nrhs / 2) * a.npar;
    if (prec == P32)
      k_unpack_pair<P32><<<nblk(np, 128), 128, 0, st>>>(a, c);
    else
      k_unpack_pair<P16><<<nblk(np, 128), 128, 0, st>>>(a, c);
    DD_CUDA(cudaGetLastError());
    return DD_OK;
  }
  return unpack_native(a, prec, f.nrhs, c, st);
}

int unpack_c64(const dd_lattice* lat, int prec, int subset, const Field& f, float* canon, cudaStream_t st, int t0,
               int nt) {
  if (f.paired) return fail(DD_ERR_ARG, "complex64 fields take the native layout");
  PackArgs a = pack_args(lat, subset, f);
  if (nt > 0) {
    const int64_t slice = (int64_t)lat->dims[1] * lat->dims[2] * lat->dims[3];
    a.s0 = t0 * slice / 2;
    a.ns = nt * slice / 2;
  }
  return unpack_native(a, prec, f.nrhs, reinterpret_cast<float2*>(canon), st);
}

}  // namespace dd
