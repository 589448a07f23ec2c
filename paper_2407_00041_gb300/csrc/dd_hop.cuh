// Fused Wilson-clover stencil kernel.
//
// One thread computes one (output site, right-hand side) pair of one parity:
//   acc(x) = sum_mu (I + s gamma_mu) (x) U_mu(x)       psi(x + mu)
//          + sum_mu (I - s gamma_mu) (x) U_mu^H(x - mu) psi(x - mu)
// with s = -1 for D (the hopping sum of Eq. 1.13 / Eq. 2.6, without the
// factor 1/2) and s = +1 for D^H = gamma5 D gamma5.  The sum is formed the
// way the back-substitution after Algorithm 3 of the thesis shows: each
// neighbour spinor is projected to two independent spin components
// (6 complex), multiplied by the link, and reconstructed.  Nothing is staged
// through memory: projection, SU(3) products, reconstruction and the
// self-coupling epilogue (Eq. 2.5, 2.7) run in registers in one pass.
//
// In the chiral basis gamma_mu = [[0, B_mu], [B_mu^H, 0]] with
//   B_T = I, B_Z = -i sigma_3, B_Y = -i sigma_2, B_X = -i sigma_1,
// so for psi = (u, l) (upper and lower spin pairs)
//   (I + t gamma_mu) psi = (h, t B_mu^H h),  h = u + t B_mu l,  t = +-1.
#pragma once

#include <cstdlib>

#include "dd_blas.h"
#include "dd_link8.cuh"
#include "dd_ops.h"

namespace dd {

__device__ __forceinline__ float ffma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double ffma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ df ffma(df a, df b, df c) { return df_fma(a, b, c); }

// (B_mu l) for spin component 0 / 1 of the lower pair
template <int MU, typename R>
__device__ __forceinline__ void b_times(cx<R> l0, cx<R> l1, cx<R>& b0, cx<R>& b1) {
  if constexpr (MU == 0) {
    b0 = l0;
    b1 = l1;
  } else if constexpr (MU == 1) {  // -i sigma_3
    b0 = mul_mi(l0);
    b1 = mul_i(l1);
  } else if constexpr (MU == 2) {  // -i sigma_2 = [[0, -1], [1, 0]]
    b0 = neg(l1);
    b1 = l0;
  } else {  // -i sigma_1 = [[0, -i], [-i, 0]]
    b0 = mul_mi(l1);
    b1 = mul_mi(l0);
  }
}

// (B_mu^H g)
template <int MU, typename R>
__device__ __forceinline__ void bh_times(cx<R> g0, cx<R> g1, cx<R>& b0, cx<R>& b1) {
  if constexpr (MU == 0) {
    b0 = g0;
    b1 = g1;
  } else if constexpr (MU == 1) {  // i sigma_3
    b0 = mul_i(g0);
    b1 = mul_mi(g1);
  } else if constexpr (MU == 2) {  // i sigma_2 = [[0, 1], [-1, 0]]
    b0 = g1;
    b1 = neg(g0);
  } else {  // i sigma_1
    b0 = mul_i(g1);
    b1 = mul_i(g0);
  }
}

// The three stages of one hop, acc += (I + T gamma_mu) (x) W psi with
// W = U (ADJ = false) or U^H (ADJ = true), scaled by `sign` (the time-boundary
// sign, times any overall factor).  Split so that a domain-decomposed apply
// can run the first stage (projection, and for the backward hop the link
// product) on the rank that owns psi and the rest on the rank that owns the
// output site, with the same arithmetic as the fused hop.
// Stage 1: the two independent spin components h = u + T B_mu l.
template <int MU, int T, typename R>
__device__ __forceinline__ void hop_project(const cx<R> psi[12], cx<R> h0[3], cx<R> h1[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    cx<R> b0, b1;
    b_times<MU>(psi[6 + c], psi[9 + c], b0, b1);
    if constexpr (T > 0) {
      h0[c] = psi[c] + b0;
      h1[c] = psi[3 + c] + b1;
    } else {
      h0[c] = psi[c] - b0;
      h1[c] = psi[3 + c] - b1;
    }
  }
}

// Stage 2: g = W h for both spin components (the nine elements of U in
// registers).
template <bool ADJ, typename R>
__device__ __forceinline__ void hop_mul(const cx<R> u[9], const cx<R> h0[3], const cx<R> h1[3], cx<R> g0[3],
                                        cx<R> g1[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    g0[a] = zero<R>();
    g1[a] = zero<R>();
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if constexpr (ADJ) {
        g0[a] = cfmac(u[3 * b + a], h0[b], g0[a]);
        g1[a] = cfmac(u[3 * b + a], h1[b], g1[a]);
      } else {
        g0[a] = cfma(u[3 * a + b], h0[b], g0[a]);
        g1[a] = cfma(u[3 * a + b], h1[b], g1[a]);
      }
    }
    renorm(g0[a]);
    renorm(g1[a]);
  }
}

// Stage 3: reconstruct the lower spin pair as T B_mu^H g and accumulate.
template <int MU, int T, typename R>
__device__ __forceinline__ void hop_reconstruct(cx<R> acc[12], const cx<R> g0[3], const cx<R> g1[3], R sign) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    acc[c] = caxpy(sign, g0[c], acc[c]);
    acc[3 + c] = caxpy(sign, g1[c], acc[3 + c]);
    cx<R> b0, b1;
    bh_times<MU>(g0[c], g1[c], b0, b1);
    const R sb = T > 0 ? sign : -sign;
    acc[6 + c] = caxpy(sb, b0, acc[6 + c]);
    acc[9 + c] = caxpy(sb, b1, acc[9 + c]);
  }
}

// All three stages: acc += (I + T gamma_mu) (x) W psi.
template <int MU, int T, bool ADJ, typename R>
__device__ __forceinline__ void hop_regs(cx<R> acc[12], const cx<R> psi[12], const cx<R> u[9], R sign) {
  cx<R> h0[3], h1[3], g0[3], g1[3];
  hop_project<MU, T, R>(psi, h0, h1);
  hop_mul<ADJ, R>(u, h0, h1, g0, g1);
  hop_reconstruct<MU, T, R>(acc, g0, g1, sign);
}

// Link storage: the 36 elements of a site's four links (direction-major,
// 3x3 row-major) are stored in 16-byte groups [group][Vh] per parity: FP64
// one element per group, FP32 two, FP16 four.  Direction mu uses elements
// 9 mu .. 9 mu + 8, i.e. 9, 5 or 3 group loads; a group shared by two
// directions is read twice (the second time from cache).
// FP32 with `recon` = 12: the copy keeps rows 0 and 1 only ([12 groups][Vh],
// direction mu in groups 3 mu .. 3 mu + 2) and row 2 of the SU(3) matrix is
// rebuilt as the complex conjugate of the cross product of rows 0 and 1.
// FP32 with `recon` = 8: eight reals per link ([8 groups][Vh], direction mu
// in groups 2 mu, 2 mu + 1), rebuilt by link8_decode.  FP16 with `recon`
// (12): rows 0 and 1 ([6 groups][Vh], elements 6 mu .. 6 mu + 5 four per
// group), row 2 rebuilt in R from the widened rows.
template <int PG, typename R>
__device__ __forceinline__ void load_link(const void* Ubase, int64_t s, int64_t Vh, int mu, cx<R> u[9],
                                          int recon = 0) {
  if constexpr (PG == P32) {
    if (recon == 8) {
      const float4* p = reinterpret_cast<const float4*>(Ubase) + s;
      const float4 w0 = __ldg(p + (int64_t)(2 * mu) * Vh), w1 = __ldg(p + (int64_t)(2 * mu + 1) * Vh);
      float2 f[9];
      link8_decode(w0, w1, f);
#pragma unroll
      for (int e = 0; e < 9; ++e) u[e] = mk<R>(f[e].x, f[e].y);
      return;
    }
    if (recon) {
      const float4* p = reinterpret_cast<const float4*>(Ubase) + s;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float4 v = __ldg(p + (int64_t)(3 * mu + k) * Vh);
        u[2 * k] = mk<R>(v.x, v.y);
        u[2 * k + 1] = mk<R>(v.z, v.w);
      }
      auto cross = [](cx<R> a, cx<R> b, cx<R> c, cx<R> d) {  // conj(a b - c d)
        const cx<R> t = cfma(neg(c), d, cmul(a, b));
        return mk(t.re, -t.im);
      };
      u[6] = cross(u[1], u[5], u[2], u[4]);
      u[7] = cross(u[2], u[3], u[0], u[5]);
      u[8] = cross(u[0], u[4], u[1], u[3]);
      return;
    }
  }
  if constexpr (PG == PDF) {
    const float4* p = reinterpret_cast<const float4*>(Ubase) + (int64_t)(9 * mu) * Vh + s;
#pragma unroll
    for (int e = 0; e < 9; ++e) u[e] = df_cx(__ldg(p + e * Vh));
  } else if constexpr (PG == P64) {
    const double2* p = reinterpret_cast<const double2*>(Ubase) + (int64_t)(9 * mu) * Vh + s;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      const double2 v = __ldg(p + e * Vh);
      u[e] = mk<R>(v.x, v.y);
    }
  } else if constexpr (PG == P32) {
    const float4* p = reinterpret_cast<const float4*>(Ubase) + s;
    const int g0 = (9 * mu) >> 1, off = (9 * mu) & 1;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const float4 v = __ldg(p + (int64_t)(g0 + k) * Vh);
      const int e0 = 2 * k - off;  // element index of v.xy within this link
      if (e0 >= 0 && e0 < 9) u[e0] = mk<R>(v.x, v.y);
      if (e0 + 1 >= 0 && e0 + 1 < 9) u[e0 + 1] = mk<R>(v.z, v.w);
    }
  } else {
    const uint4* p = reinterpret_cast<const uint4*>(Ubase) + s;
    if (recon) {  // FP16 rows 0 and 1 ([6 groups][Vh], elements 6 mu .. 6 mu + 5)
      const int g0 = (6 * mu) >> 2, off = (6 * mu) & 3;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const uint4 v = __ldg(p + (int64_t)(g0 + k) * Vh);
        unsigned int w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int e = 4 * k + q - off;
          if (e >= 0 && e < 6) {
            const float2 f = __half22float2(*reinterpret_cast<__half2*>(&w[q]));
            u[e] = mk<R>(f.x, f.y);
          }
        }
      }
      auto cross = [](cx<R> a, cx<R> b, cx<R> c, cx<R> d) {  // conj(a b - c d)
        const cx<R> t = cfma(neg(c), d, cmul(a, b));
        return mk(t.re, -t.im);
      };
      u[6] = cross(u[1], u[5], u[2], u[4]);
      u[7] = cross(u[2], u[3], u[0], u[5]);
      u[8] = cross(u[0], u[4], u[1], u[3]);
      return;
    }
    const int g0 = (9 * mu) >> 2, off = (9 * mu) & 3;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const uint4 v = __ldg(p + (int64_t)(g0 + k) * Vh);
      unsigned int w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int e = 4 * k + q - off;
        if (e >= 0 && e < 9) {
          const float2 f = __half22float2(*reinterpret_cast<__half2*>(&w[q]));
          u[e] = mk<R>(f.x, f.y);
        }
      }
    }
  }
}

// The same with the link read from its native layout.
template <int PG, int MU, int T, bool ADJ, typename R>
__device__ __forceinline__ void hop(cx<R> acc[12], const cx<R> psi[12], const void* Ubase, int64_t s, int64_t Vh,
                                    R sign, int recon) {
  cx<R> u[9];
  load_link<PG, R>(Ubase, s, Vh, MU, u, recon);
  hop_regs<MU, T, ADJ, R>(acc, psi, u, sign);
}

// ---- FP16 storage with half2 projection and FP16 x FP16 -> FP32 products ----
// For FP16 spinors with FP16 links and blocks the hop runs without widening
// the stored values: the spin projection h = u + T B l is formed in half2
// arithmetic (each component the exact sum rounded once to FP16), and every
// product of a link or block element with an FP16 value is one mixed FMA,
// fma.rn.f32.f16 (exact product of the two FP16 values, FP32 accumulation,
// one rounding to FP32), in the order of cfma / cfmac.  The reconstruction
// and the accumulation of the hops stay in FP32.  Compared with widening
// every value first, the only extra rounding is that of h to FP16.

// c + a b for FP16 a, b with one rounding to FP32
__device__ __forceinline__ float mfma_h(__half a, __half b, float c) {
  float d;
  asm("fma.rn.f32.f16 %0, %1, %2, %3;" : "=f"(d) : "h"(__half_as_ushort(a)), "h"(__half_as_ushort(b)), "f"(c));
  return d;
}

// (re, im) -> (im, re)
__device__ __forceinline__ __half2 h2_swap(__half2 z) { return __lowhigh2highlow(z); }

// h = u + T (B_mu l) per colour on half2 (re, im) words; -i z = swap(z) (1, -1),
// i z = swap(z) (-1, 1)
template <int MU, int T>
__device__ __forceinline__ void hop_project_h(const __half2 psi[12], __half2 h0[3], __half2 h1[3]) {
  const __half2 pm = __floats2half2_rn((float)T, (float)-T);
  const __half2 mp = __floats2half2_rn((float)-T, (float)T);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const __half2 u0 = psi[c], u1 = psi[3 + c], l0 = psi[6 + c], l1 = psi[9 + c];
    if constexpr (MU == 0) {  // b0 = l0, b1 = l1
      h0[c] = T > 0 ? __hadd2(u0, l0) : __hsub2(u0, l0);
      h1[c] = T > 0 ? __hadd2(u1, l1) : __hsub2(u1, l1);
    } else if constexpr (MU == 1) {  // b0 = -i l0, b1 = i l1
      h0[c] = __hfma2(h2_swap(l0), pm, u0);
      h1[c] = __hfma2(h2_swap(l1), mp, u1);
    } else if constexpr (MU == 2) {  // b0 = -l1, b1 = l0
      h0[c] = T > 0 ? __hsub2(u0, l1) : __hadd2(u0, l1);
      h1[c] = T > 0 ? __hadd2(u1, l0) : __hsub2(u1, l0);
    } else {  // b0 = -i l1, b1 = -i l0
      h0[c] = __hfma2(h2_swap(l1), pm, u0);
      h1[c] = __hfma2(h2_swap(l0), pm, u1);
    }
  }
}

// g += w h (ADJ = false) or conj(w) h (ADJ = true) for FP16 w, h (nh = -h),
// in the order of cfma / cfmac
template <bool ADJ>
__device__ __forceinline__ void cmac_h(__half2 w, __half2 h, __half2 nh, cx<float>& g) {
  const __half wr = __low2half(w), wi = __high2half(w);
  g.re = mfma_h(wr, __low2half(h), g.re);
  g.re = mfma_h(wi, ADJ ? __high2half(h) : __high2half(nh), g.re);
  g.im = mfma_h(wr, __high2half(h), g.im);
  g.im = mfma_h(wi, ADJ ? __low2half(nh) : __low2half(h), g.im);
}

// g = W h for both spin components (W = U, or U^H with ADJ)
template <bool ADJ>
__device__ __forceinline__ void hop_mul_h(const __half2 u[9], const __half2 h0[3], const __half2 h1[3],
                                          cx<float> g0[3], cx<float> g1[3]) {
  __half2 n0[3], n1[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) n0[b] = __hneg2(h0[b]), n1[b] = __hneg2(h1[b]);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    g0[a] = zero<float>();
    g1[a] = zero<float>();
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const __half2 w = ADJ ? u[3 * b + a] : u[3 * a + b];
      cmac_h<ADJ>(w, h0[b], n0[b], g0[a]);
      cmac_h<ADJ>(w, h1[b], n1[b], g1[a]);
    }
  }
}

// The nine FP16 elements of link mu of site s, as stored (four per 16-byte
// group).  With `recon` (12) the copy holds rows 0 and 1 ([6 groups][Vh]);
// row 2 = conj(row 0 x row 1) is formed with mixed FMAs (exact products of
// the stored FP16 values, FP32 sums) and rounded once to FP16.
__device__ __forceinline__ void load_link_h(const void* Ubase, int64_t s, int64_t Vh, int mu, __half2 u[9],
                                            int recon = 0) {
  const uint4* p = reinterpret_cast<const uint4*>(Ubase) + s;
  if (recon) {
    const int g0 = (6 * mu) >> 2, off = (6 * mu) & 3;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const uint4 v = __ldg(p + (int64_t)(g0 + k) * Vh);
      const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int e = 4 * k + q - off;
        if (e >= 0 && e < 6) u[e] = *reinterpret_cast<const __half2*>(&w[q]);
      }
    }
    // conj(a b - c d): re = ar br - ai bi - cr dr + ci di, im = -(ar bi + ai br - cr di - ci dr)
    auto cross = [](__half2 a, __half2 b, __half2 c, __half2 d) {
      const __half2 nc = __hneg2(c);
      const __half ar = __low2half(a), ai = __high2half(a), br = __low2half(b), bi = __high2half(b);
      const __half ci = __high2half(c), ncr = __low2half(nc), nci = __high2half(nc);
      const __half dr = __low2half(d), di = __high2half(d);
      float re = mfma_h(ar, br, 0.f);
      re = mfma_h(__hneg(ai), bi, re);
      re = mfma_h(ncr, dr, re);
      re = mfma_h(ci, di, re);
      float im = mfma_h(ar, bi, 0.f);
      im = mfma_h(ai, br, im);
      im = mfma_h(ncr, di, im);
      im = mfma_h(nci, dr, im);
      return __floats2half2_rn(re, -im);
    };
    u[6] = cross(u[1], u[5], u[2], u[4]);
    u[7] = cross(u[2], u[3], u[0], u[5]);
    u[8] = cross(u[0], u[4], u[1], u[3]);
    return;
  }
  const int g0 = (9 * mu) >> 2, off = (9 * mu) & 3;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const uint4 v = __ldg(p + (int64_t)(g0 + k) * Vh);
    const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = 4 * k + q - off;
      if (e >= 0 && e < 9) u[e] = *reinterpret_cast<const __half2*>(&w[q]);
    }
  }
}

// The 12 stored FP16 components of index i (site * N + r); returns the site scale
__device__ __forceinline__ float load_spinor_h(const HalfField& f, int64_t gstride, int64_t i, __half2 v[12]) {
  const uint4* b = reinterpret_cast<const uint4*>(f.base) + i;
  const float sc = __ldg(f.scale + i);
#pragma unroll
  for (int g = 0; g < 3; ++g) {
    const uint4 t = __ldg(b + g * gstride);
    const unsigned w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) v[4 * g + k] = *reinterpret_cast<const __half2*>(&w[k]);
  }
  return sc;
}

// acc += sign (I + T gamma_mu) (x) W psi for FP16 psi and links
template <int MU, int T, bool ADJ>
__device__ __forceinline__ void hop_h(cx<float> acc[12], const __half2 psi[12], const void* Ubase, int64_t s,
                                      int64_t Vh, float sign, int recon = 0) {
  __half2 u[9], h0[3], h1[3];
  load_link_h(Ubase, s, Vh, MU, u, recon);
  hop_project_h<MU, T>(psi, h0, h1);
  cx<float> g0[3], g1[3];
  hop_mul_h<ADJ>(u, h0, h1, g0, g1);
  hop_reconstruct<MU, T, float>(acc, g0, g1, sign);
}

// One hop from the stored neighbour spinor i of field f: FP16 spinors with
// FP16 links take the half2 / mixed-FMA path above, every other precision
// pair widens to R first.  sg: the boundary sign (the FP16 site scale is
// folded in here).
template <int PG, int PIN, int MU, int T, bool ADJ, typename R>
__device__ __forceinline__ void hop_from(cx<R> acc[12], const HalfField& f, int64_t gstride, int64_t i,
                                         const void* Ubase, int64_t s, int64_t Vh, R sg, int recon) {
  if constexpr (PG == P16 && PIN == P16) {
    __half2 psi[12];
    sg *= load_spinor_h(f, gstride, i, psi);
    hop_h<MU, T, ADJ>(acc, psi, Ubase, s, Vh, sg, recon);
  } else {
    cx<R> psi[12];
    sg *= load_spinor_unscaled<PIN, R>(f, gstride, i, psi);
    hop<PG, MU, T, ADJ, R>(acc, psi, Ubase, s, Vh, sg, recon);
  }
}

// Self-coupling / A_ee^{-1} storage: two Hermitian 6x6 blocks per site, 18
// elements each: elements 0..2 hold the real diagonal in pairs (d0, d1),
// (d2, d3), (d4, d5); elements 3..17 the strict upper triangle row by row.
// The 36 elements of a site are stored in 16-byte groups, [group][Vh]:
// FP64 one element per group (double2), FP32 two (float4), FP16 four
// (8 halves), so a site's blocks take 36, 18 or 9 loads.
template <int PG>
struct BlockGroups {
  static constexpr int PER = (PG == P64 || PG == PDF) ? 1 : PG == P32 ? 2 : 4;  // elements per group
};

// (i, j) of the strict upper-triangle element o = 0..14 of a 6x6 block
__device__ __forceinline__ void tri_ij(int o, int& i, int& j) {
  i = o < 5 ? 0 : o < 9 ? 1 : o < 12 ? 2 : o < 14 ? 3 : 4;
  const int start = i == 0 ? 0 : i == 1 ? 5 : i == 2 ? 9 : i == 3 ? 12 : 14;
  j = i + 1 + (o - start);
}

// group g of site s: the PER elements it holds
template <int PG, typename R>
__device__ __forceinline__ void load_block_group(const void* M, int64_t s, int64_t Vh, int g, cx<R> e[4],
                                                 bool streaming) {
  if constexpr (PG == PDF) {
    const float4* p = reinterpret_cast<const float4*>(M) + (int64_t)g * Vh + s;
    e[0] = df_cx(streaming ? __ldcs(p) : __ldg(p));
  } else if constexpr (PG == P64) {
    const double2* p = reinterpret_cast<const double2*>(M) + (int64_t)g * Vh + s;
    const double2 v = streaming ? __ldcs(p) : __ldg(p);
    e[0] = mk<R>(v.x, v.y);
  } else if constexpr (PG == P32) {
    const float4* p = reinterpret_cast<const float4*>(M) + (int64_t)g * Vh + s;
    const float4 v = streaming ? __ldcs(p) : __ldg(p);
    e[0] = mk<R>(v.x, v.y);
    e[1] = mk<R>(v.z, v.w);
  } else {
    const uint4* p = reinterpret_cast<const uint4*>(M) + (int64_t)g * Vh + s;
    const uint4 v = streaming ? __ldcs(p) : __ldg(p);
    unsigned int w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float2 f = __half22float2(*reinterpret_cast<__half2*>(&w[q]));
      e[q] = mk<R>(f.x, f.y);
    }
  }
}

// out (+)= M x for the two blocks of site s (ADD = false overwrites out).
template <int PG, bool ADD, typename R>
__device__ __forceinline__ void block_apply_g(const void* M, int64_t s, int64_t Vh, const cx<R> x[12], cx<R> out[12],
                                              bool streaming) {
  constexpr int PER = BlockGroups<PG>::PER;
  cx<R> grp[4];
#pragma unroll
  for (int E = 0; E < 36; ++E) {
    if (E % PER == 0) load_block_group<PG, R>(M, s, Vh, E / PER, grp, streaming);
    const cx<R> m = grp[E % PER];
    const int b = E / 18, k = E % 18;
    if (k < 3) {
      if (ADD) {
        out[6 * b + 2 * k] = out[6 * b + 2 * k] + m.re * x[6 * b + 2 * k];
        out[6 * b + 2 * k + 1] = out[6 * b + 2 * k + 1] + m.im * x[6 * b + 2 * k + 1];
      } else {
        out[6 * b + 2 * k] = m.re * x[6 * b + 2 * k];
        out[6 * b + 2 * k + 1] = m.im * x[6 * b + 2 * k + 1];
      }
    } else {
      int i, j;
      tri_ij(k - 3, i, j);
      out[6 * b + i] = cfma(m, x[6 * b + j], out[6 * b + i]);
      out[6 * b + j] = cfmac(m, x[6 * b + i], out[6 * b + j]);
    }
  }
#pragma unroll
  for (int c = 0; c < 12; ++c) renorm(out[c]);
}

// out = M x with M the parity base pointer of the block array and s the site
template <int PG, typename R>
__device__ __forceinline__ void block_apply(const void* M, int64_t s, int64_t Vh, const cx<R> x[12], cx<R> out[12]) {
  block_apply_g<PG, false, R>(M, s, Vh, x, out, true);
}

// out = M x for FP16 blocks and an FP16 spinor x (stored values, without the
// site scale), by mixed FMAs in the order of block_apply_g.
__device__ __forceinline__ void block_apply_h(const void* M, int64_t s, int64_t Vh, const __half2 x[12],
                                              cx<float> out[12]) {
  __half2 nx[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) nx[c] = __hneg2(x[c]);
  const uint4* p = reinterpret_cast<const uint4*>(M) + s;
  unsigned w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
  for (int E = 0; E < 36; ++E) {
    if (E % 4 == 0) {
      const uint4 v = __ldcs(p + (int64_t)(E / 4) * Vh);
      w[0] = v.x, w[1] = v.y, w[2] = v.z, w[3] = v.w;
    }
    const __half2 m = *reinterpret_cast<const __half2*>(&w[E % 4]);
    const int b = E / 18, k = E % 18;
    if (k < 3) {
      const int i0 = 6 * b + 2 * k, i1 = i0 + 1;
      const __half d0 = __low2half(m), d1 = __high2half(m);
      out[i0].re = mfma_h(d0, __low2half(x[i0]), 0.f);
      out[i0].im = mfma_h(d0, __high2half(x[i0]), 0.f);
      out[i1].re = mfma_h(d1, __low2half(x[i1]), 0.f);
      out[i1].im = mfma_h(d1, __high2half(x[i1]), 0.f);
    } else {
      int i, j;
      tri_ij(k - 3, i, j);
      i += 6 * b;
      j += 6 * b;
      cmac_h<false>(m, x[j], nx[j], out[i]);  // out_i += m x_j
      cmac_h<true>(m, x[i], nx[i], out[j]);   // out_j += conj(m) x_i
    }
  }
}

// Epilogue of the one-thread-per-(site, RHS) stencil: combine the hopping
// sum acc of output site s (parity p), right-hand side r, with the self
// coupling as EPI says and store.  With NORM it returns |out|^2 of the stored
// FP32 result (summed in FP32 over the 12 components), else 0.
template <int PG, int PIN, int POUT, int EPI, bool NORM, typename R>
__device__ __forceinline__ float hop_epilogue(const HopArgs& a, int p, int s, int r, cx<R> acc[12]) {
#pragma unroll
  for (int c = 0; c < 12; ++c) renorm(acc[c]);  // FP32 pairs: the hops accumulate lazily
  const int64_t Vh = a.g.Vh;
  const R beta = (R)a.beta;
  const int64_t i = (int64_t)s * a.nrhs + r;
  const void* M = a.M[p];
  cx<R> res[12];
  if constexpr (EPI == EPI_D && PG == P16 && PIN == P16) {
    // M y from the stored FP16 values, then the site scale
    __half2 yh[12];
    const float ys = load_spinor_h(a.y[p], a.gstride, i, yh);
    block_apply_h(M, s, Vh, yh, res);
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      res[c].re = ffma(beta, acc[c].re, res[c].re * ys);
      res[c].im = ffma(beta, acc[c].im, res[c].im * ys);
    }
  } else if constexpr (EPI == EPI_D || EPI == EPI_RESID) {
    cx<R> y[12];
    if constexpr (EPI == EPI_D)
      load_spinor<PIN, R>(a.y[p], a.gstride, i, y);
    else
      load_spinor<POUT, R>(a.y[p], a.gstride, i, y);
    block_apply<PG, R>(M, s, Vh, y, res);
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      res[c].re = ffma(beta, acc[c].re, res[c].re);
      res[c].im = ffma(beta, acc[c].im, res[c].im);
    }
    if constexpr (EPI == EPI_RESID) {
      cx<R> z[12];
      load_spinor<POUT, R>(a.z[p], a.gstride, i, z);
#pragma unroll
      for (int c = 0; c < 12; ++c) res[c] = z[c] - res[c];
    }
  } else if constexpr (EPI == EPI_AINV) {
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[c] = beta * acc[c];
    block_apply<PG, R>(M, s, Vh, acc, res);
  } else if constexpr (EPI == EPI_ADD) {
    load_spinor<POUT, R>(a.y[p], a.gstride, i, res);
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      res[c].re = ffma(beta, acc[c].re, res[c].re);
      res[c].im = ffma(beta, acc[c].im, res[c].im);
    }
  } else {  // EPI_AINV_ADD
    cx<R> y[12];
    load_spinor<POUT, R>(a.y[p], a.gstride, i, y);
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      y[c].re = ffma(beta, acc[c].re, y[c].re);
      y[c].im = ffma(beta, acc[c].im, y[c].im);
    }
    block_apply<PG, R>(M, s, Vh, y, res);
  }
  store_spinor<POUT, R, true>(a.out[p], a.gstride, i, res);
  float n2 = 0.f;
  if constexpr (NORM) {
    // the FP32 result before it is stored (for FP16 output: before the
    // rounding to halves, within 2^-11 of the stored vector's norm)
    static_assert(POUT == P32 || POUT == P16, "the fused norm reads an FP32 result");
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      n2 = __fmaf_rn((float)res[c].re, (float)res[c].re, n2);
      n2 = __fmaf_rn((float)res[c].im, (float)res[c].im, n2);
    }
  }
  return n2;
}

// FP32-pair arithmetic: the eight hops of a site in one rolled loop.  Each
// pair operation takes 7-15 FP32 instructions, and the unrolled eight hops
// (4 directions x 2, each with its own projection and colour product code)
// did not fit the instruction cache (ncu at 48 x 24^3: warps stalled on
// instruction fetch 7.7 times per issue, issue active 27%); here one copy of
// the colour product serves all hops: the backward hops take U^H by
// conjugating and transposing the nine elements in registers, and the
// projection B_mu l and reconstruction B_mu^H g select their components and
// factors (1, i, -1, -i) from small tables.
// f z for f = i^k, k = 0..3
template <typename R>
__device__ __forceinline__ cx<R> mul_ipow(cx<R> z, int k) {
  const bool sw = k & 1;
  const R re = sw ? z.im : z.re, im = sw ? z.re : z.im;
  return mk((k == 1 || k == 2) ? -re : re, (k >= 2) ? -im : im);
}

template <int PG, int PIN, bool DAG, typename R>
__device__ __forceinline__ void hops_rolled(const HopArgs& a, const SiteCoord& sc, int p, int s, int r,
                                            cx<R> acc[12]) {
  const int q = p ^ 1;
  const int64_t Vh = a.g.Vh;
  constexpr int TF = DAG ? +1 : -1;
  int nidx[8];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    nidx[2 * m] = nb_fwd(a.g, sc, m);
    nidx[2 * m + 1] = nb_bwd(a.g, sc, m);
  }
  const R sf0 = sc.c[0] == a.g.n[0] - 1 ? (R)a.g.t_bc : (R)1;
  const R sb0 = sc.c[0] == 0 ? (R)a.g.t_bc : (R)1;
#pragma unroll 1
  for (int k = 0; k < 8; ++k) {
    const int mu = k >> 1;
    const bool bwd = k & 1;
    int nl = nidx[0];
#pragma unroll
    for (int j = 1; j < 8; ++j)
      if (k == j) nl = nidx[j];
    const int T = bwd ? -TF : TF;
    const R sign = mu == 0 ? (bwd ? sb0 : sf0) : (R)1;
    cx<R> psi[12], u[9];
    load_spinor<PIN, R>(a.in[q], a.gstride, (int64_t)(nl >> 1) * a.nrhs + r, psi);
    if (bwd)
      load_link<PG, R>(a.U[q], nl >> 1, Vh, mu, u);
    else
      load_link<PG, R>(a.U[p], s, Vh, mu, u);
    if (bwd) {  // U^H
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        u[4 * i] = mk(u[4 * i].re, -u[4 * i].im);
#pragma unroll
        for (int j = i + 1; j < 3; ++j) {
          const cx<R> t = u[3 * i + j];
          u[3 * i + j] = mk(u[3 * j + i].re, -u[3 * j + i].im);
          u[3 * j + i] = mk(t.re, -t.im);
        }
      }
    }
    // B_mu l: b0 = i^k0 l_j0, b1 = i^k1 l_j1; B_mu^H g: b0 = i^m0 g_i0, b1 = i^m1 g_i1
    const int j0 = mu >= 2, j1 = mu < 2;
    const int k0 = mu == 0 ? 0 : mu == 1 ? 3 : mu == 2 ? 2 : 3;
    const int k1 = mu == 0 ? 0 : mu == 1 ? 1 : mu == 2 ? 0 : 3;
    const int i0 = mu == 2 || mu == 3, i1 = mu < 2;
    const int m0 = mu == 0 ? 0 : mu == 1 ? 1 : mu == 2 ? 0 : 1;
    const int m1 = mu == 0 ? 0 : mu == 1 ? 3 : mu == 2 ? 2 : 1;
    cx<R> h0[3], h1[3], g0[3], g1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const cx<R> b0 = mul_ipow(j0 ? psi[9 + c] : psi[6 + c], k0);
      const cx<R> b1 = mul_ipow(j1 ? psi[9 + c] : psi[6 + c], k1);
      h0[c] = T > 0 ? psi[c] + b0 : psi[c] - b0;
      h1[c] = T > 0 ? psi[3 + c] + b1 : psi[3 + c] - b1;
    }
    hop_mul<false, R>(u, h0, h1, g0, g1);
    const R sb = T > 0 ? sign : -sign;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      acc[c] = caxpy(sign, g0[c], acc[c]);
      acc[3 + c] = caxpy(sign, g1[c], acc[3 + c]);
      acc[6 + c] = caxpy(sb, mul_ipow(i0 ? g1[c] : g0[c], m0), acc[6 + c]);
      acc[9 + c] = caxpy(sb, mul_ipow(i1 ? g1[c] : g0[c], m1), acc[9 + c]);
    }
  }
}

// The work of one thread: output slot `tid` in [0, npar * Vh * nrhs).  With
// NORM it returns |out|^2 of the stored FP32 result (summed in FP32 over the
// 12 components), else 0.
// LF: the form of the links the launch reads: 0 three rows, 12 rows 0 and 1
// (FP16), 8 eight reals (FP32), fixed at compile time; -1 (FP32) three or
// two rows by a.recon at run time (ptxas allocates this variant of the FP32
// stencil without the spills of the compile-time two-row one).
template <int PG, int PIN, int POUT, bool DAG, int EPI, bool NORM = false, int LF = 0>
__device__ __forceinline__ float hop_thread(const HopArgs& a, int64_t tid) {
  using R = typename Store<PG>::real;
  using E = typename Store<PG>::elem;
  int p, s, r;
  SiteCoord sc;
  if (a.npar == 2) {
    // both parities: threads follow the lexicographic site order, so the two
    // uses of every link (forward hop at x, backward hop at x + mu) and the
    // reads of a neighbour spinor fall within about one time slice of traffic
    const int lex = fdiv((int)tid, a.fblk);
    r = (int)tid - lex * a.nrhs;
    sc = traversal_coords(a.g, lex);
    p = (sc.c[0] + sc.c[1] + sc.c[2] + sc.c[3]) & 1;
    s = sc.lex >> 1;
  } else {
    p = a.p0;
    s = fdiv((int)tid, a.fblk);
    r = (int)tid - s * a.nrhs;
    sc = site_coords(a.g, s, p);
  }
  const int q = p ^ 1;
  const int64_t Vh = a.g.Vh;
  // forward hop: (I - gamma) for D, (I + gamma) for D^H; backward the opposite
  constexpr int TF = DAG ? +1 : -1;
  constexpr int TB = -TF;
  const int rc = LF >= 0 ? LF : (a.recon ? 12 : 0);

  cx<R> acc[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) acc[c] = zero<R>();

#define DD_HOP_DIR(MU)                                                                                 \
  {                                                                                                    \
    int nl = nb_fwd(a.g, sc, MU);                                                                      \
    R sg = (MU == 0 && sc.c[0] == a.g.n[0] - 1) ? (R)a.g.t_bc : (R)1;                                  \
    hop_from<PG, PIN, MU, TF, false, R>(acc, a.in[q], a.gstride, (int64_t)(nl >> 1) * a.nrhs + r, a.U[p], s, \
                                        Vh, sg, rc);                                                   \
    nl = nb_bwd(a.g, sc, MU);                                                                          \
    sg = (MU == 0 && sc.c[0] == 0) ? (R)a.g.t_bc : (R)1;                                               \
    hop_from<PG, PIN, MU, TB, true, R>(acc, a.in[q], a.gstride, (int64_t)(nl >> 1) * a.nrhs + r, a.U[q],    \
                                       nl >> 1, Vh, sg, rc);                                           \
  }
  if constexpr (PG == PDF) {
    hops_rolled<PG, PIN, DAG, R>(a, sc, p, s, r, acc);
  } else {
    DD_HOP_DIR(0)
    DD_HOP_DIR(1)
    DD_HOP_DIR(2)
    DD_HOP_DIR(3)
  }
#undef DD_HOP_DIR

  return hop_epilogue<PG, PIN, POUT, EPI, NORM, R>(a, p, s, r, acc);
}

// RHS-blocked variant for several right-hand sides (three-row links only): one thread handles NB
// right-hand sides r = rb + k * (N / NB), k < NB, of one site, so each link
// element is loaded once per NB spinors (link reuse across RHS in
// registers).  The strided RHS choice keeps every load instruction of a warp
// on consecutive addresses.  EPI_D builds A(x) psi(x) first and folds beta
// into the hops; EPI_AINV applies the block to beta * acc at the end.  The
// self-coupling elements are re-read from L1 for each of the NB spinors.
template <int PG, int PIN, int POUT, bool DAG, int EPI, int NB>
__device__ __forceinline__ void hop_thread_rb(const HopArgs& a, int64_t tid) {
  using R = typename Store<PG>::real;
  using E = typename Store<PG>::elem;
  const int nrb = (a.nrhs + NB - 1) / NB;  // RHS blocks; the last one may be short
  int p, s, rb;
  SiteCoord sc;
  if (a.npar == 2) {
    const int lex = fdiv((int)tid, a.fblk);
    rb = (int)tid - lex * nrb;
    sc = traversal_coords(a.g, lex);
    p = (sc.c[0] + sc.c[1] + sc.c[2] + sc.c[3]) & 1;
    s = sc.lex >> 1;
  } else {
    p = a.p0;
    s = fdiv((int)tid, a.fblk);
    rb = (int)tid - s * nrb;
    sc = site_coords(a.g, s, p);
  }
  const int q = p ^ 1;
  const int64_t Vh = a.g.Vh;
  constexpr int TF = DAG ? +1 : -1;
  constexpr int TB = -TF;
  const R beta = (R)a.beta;
  const void* M = a.M[p];
  const int64_t ibase = (int64_t)s * a.nrhs + rb;
  // offset of RHS k of the block; a RHS past the end (N not a multiple of
  // NB) recomputes RHS rb and is not stored
  int koff[NB];
#pragma unroll
  for (int k = 0; k < NB; ++k) koff[k] = rb + k * nrb < a.nrhs ? k * nrb : 0;

  cx<R> res[NB][12];
#pragma unroll
  for (int k = 0; k < NB; ++k) {
#pragma unroll
    for (int c = 0; c < 12; ++c) res[k][c] = zero<R>();
    if constexpr (EPI == EPI_D) {
      cx<R> y[12];
      load_spinor<PIN, R>(a.y[p], a.gstride, ibase + koff[k], y);
      block_apply_g<PG, true, R>(M, s, Vh, y, res[k], false);
    }
  }
  const R hop_scale = EPI == EPI_D ? beta : (R)1;

#define DD_RB_HOP(MU, FWD)                                                                          \
  {                                                                                                 \
    const int nl = FWD ? nb_fwd(a.g, sc, MU) : nb_bwd(a.g, sc, MU);                                 \
    R sg = hop_scale;                                                                               \
    if (MU == 0 && sc.c[0] == (FWD ? a.g.n[0] - 1 : 0)) sg = sg * (R)a.g.t_bc;                      \
    cx<R> u[9];                                                                                     \
    load_link<PG, R>(FWD ? a.U[p] : a.U[q], FWD ? (int64_t)s : (int64_t)(nl >> 1), Vh, MU, u);     \
    const int64_t ib = (int64_t)(nl >> 1) * a.nrhs + rb;                                            \
    _Pragma("unroll") for (int k = 0; k < NB; ++k) {                                                \
      cx<R> psi[12];                                                                                \
      const R sk = sg * load_spinor_unscaled<PIN, R>(a.in[q], a.gstride, ib + koff[k], psi);        \
      hop_regs<MU, FWD ? TF : TB, !FWD, R>(res[k], psi, u, sk);                                     \
    }                                                                                               \
  }
  DD_RB_HOP(0, true)
  DD_RB_HOP(0, false)
  DD_RB_HOP(1, true)
  DD_RB_HOP(1, false)
  DD_RB_HOP(2, true)
  DD_RB_HOP(2, false)
  DD_RB_HOP(3, true)
  DD_RB_HOP(3, false)
#undef DD_RB_HOP

#pragma unroll
  for (int k = 0; k < NB; ++k) {
    if (koff[k] != k * nrb) continue;  // past the last RHS
    if constexpr (EPI == EPI_AINV) {
      // out_k = M (beta acc_k)
#pragma unroll
      for (int c = 0; c < 12; ++c) res[k][c] = beta * res[k][c];
      cx<R> out[12];
#pragma unroll
      for (int c = 0; c < 12; ++c) out[c] = zero<R>();
      block_apply_g<PG, true, R>(M, s, Vh, res[k], out, false);
      store_spinor<POUT, R, true>(a.out[p], a.gstride, ibase + k * nrb, out);
    } else {
      store_spinor<POUT, R, true>(a.out[p], a.gstride, ibase + k * nrb, res[k]);
    }
  }
}

template <int PG, int PIN, int POUT, bool DAG, int EPI, int NB>
__global__ void __launch_bounds__(128, NB >= 4 ? 2 : 3) k_hop_rb(const HopArgs a) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= launch_sites(a.g, a.npar) * ((a.nrhs + NB - 1) / NB)) return;
  hop_thread_rb<PG, PIN, POUT, DAG, EPI, NB>(a, tid);
}

// Memory-bound FP32 variants ask for at least 5 resident CTAs of 128
// threads (at most 102 registers): measured on the 48^3 x 96 lattice this
// beats the unconstrained 108-register build by about 5%.  The FP16-storage
// stencil (half2 projection, mixed FMAs) asks for 7 (at most 72 registers):
// 0.738 ms against 0.762 ms with 5 and 0.857 ms with 3 at 48^3 x 96 (with
// two-row links 0.698 ms against 0.709 with 6 and 0.724 with 8).  FP16 links
// with FP32 vectors (the FP16-inner solve) take 4: the solve 1.468 s against
// 1.502 s with 5 and 1.513 s with 6.  The FP32-pair stencil takes 3 (at most
// 168 registers: 7.6 ms against 11.3 ms with 4, which spills).  FP64 is
// bound by the FP64 pipe and keeps the unconstrained allocation.
template <int PG, int PIN = PG>
struct HopMinBlocks {
  static constexpr int value = PG == P64 ? 1 : PG == PDF ? 3 : (PG == P16 && PIN == P16) ? 7 : PG == P16 ? 4 : 5;
};

template <int PG, int PIN, int POUT, bool DAG, int EPI, int LF = 0>
__global__ void __launch_bounds__(128, (HopMinBlocks<PG, PIN>::value)) k_hop(const HopArgs a) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= launch_sites(a.g, a.npar) * a.nrhs) return;
  hop_thread<PG, PIN, POUT, DAG, EPI, false, LF>(a, tid);
}

// EPI_D stencil of one right-hand side that also reduces |out|^2 over the
// block: FP32 warp shuffles (32 sites, as the dot kernel sums short runs in
// FP32), then the four warps' sums in FP64 in order, one partial per block
// (partials[blockIdx.x].x); threads past the end contribute zero.
template <int PG, int PIN, int POUT, bool DAG, int LF = 0>
__global__ void __launch_bounds__(128, (HopMinBlocks<PG, PIN>::value)) k_hop_norm(const HopArgs a, double2* partials) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float v = 0.f;
  if (tid < launch_sites(a.g, a.npar)) v = hop_thread<PG, PIN, POUT, DAG, EPI_D, true, LF>(a, tid);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  __shared__ float sw[4];
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0)
    partials[blockIdx.x] = make_double2((((double)sw[0] + (double)sw[1]) + (double)sw[2]) + (double)sw[3], 0.0);
}

template <int PG, int PIN, int POUT>
__global__ void __launch_bounds__(128) k_block(const BlockArgs a) {
  using R = typename Store<PG>::real;
  using E = typename Store<PG>::elem;
  const int64_t nper = a.Vh * a.nrhs;
  int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= nper * a.npar) return;
  int p = a.p0;
  if (tid >= nper) {
    tid -= nper;
    p ^= 1;
  }
  const int s = (int)(tid / a.nrhs);
  cx<R> y[12], res[12];
  load_spinor<PIN, R>(a.y[p], a.gstride, tid, y);
  block_apply<PG, R>(a.M[p], s, a.Vh, y, res);
  store_spinor<POUT, R>(a.out[p], a.gstride, tid, res);
}

}  // namespace dd

#include "dd_stage.cuh"

namespace dd {

// RHS counts for which the batched kernel (one register allocation for all
// its lattices, sized for blocks of two) takes the RHS-blocked body: every
// even count, and odd counts from 5 up (one thread of every site then carries
// a short block).  Separate launches block even counts only: for odd counts
// the one-thread-per-RHS kernel at its higher occupancy is faster (32^4:
// 5 RHS 0.57 vs 0.64 ms, 17 RHS 1.68 vs 1.73 ms).
inline bool rb_worth(int nrhs) { return nrhs >= 2 && (nrhs % 2 == 0 || nrhs >= 5); }

// One thread per (site, RHS) with the epilogue `epi`.
template <int PG, int PIN, int POUT, int LF>
cudaError_t launch_hop_single(const HopArgs& a, bool dagger, int epi, unsigned blocks, int threads, cudaStream_t st) {
  switch (epi * 2 + (dagger ? 1 : 0)) {
    case EPI_D * 2:
      k_hop<PG, PIN, POUT, false, EPI_D, LF><<<blocks, threads, 0, st>>>(a);
      break;
    case EPI_D * 2 + 1:
      k_hop<PG, PIN, POUT, true, EPI_D, LF><<<blocks, threads, 0, st>>>(a);
      break;
    case EPI_AINV * 2:
      k_hop<PG, PIN, POUT, false, EPI_AINV, LF><<<blocks, threads, 0, st>>>(a);
      break;
    case EPI_AINV * 2 + 1:
      k_hop<PG, PIN, POUT, true, EPI_AINV, LF><<<blocks, threads, 0, st>>>(a);
      break;
    case EPI_RESID * 2:
      k_hop<PG, PIN, POUT, false, EPI_RESID, LF><<<blocks, threads, 0, st>>>(a);
      break;
    case EPI_ADD * 2:
      k_hop<PG, PIN, POUT, false, EPI_ADD, LF><<<blocks, threads, 0, st>>>(a);
      break;
    case EPI_AINV_ADD * 2:
      k_hop<PG, PIN, POUT, false, EPI_AINV_ADD, LF><<<blocks, threads, 0, st>>>(a);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Host launchers; the instantiation units explicitly instantiate one
// precision triple each, other units only see the declarations in dd_ops.h.
template <int PG, int PIN, int POUT>
cudaError_t launch_hop(const HopArgs& args, bool dagger, int epi, cudaStream_t st) {
  HopArgs a = args;
  prepare_divs(a.g);
  a.fblk = make_fastdiv((uint32_t)a.nrhs);
  const int64_t n = launch_sites(a.g, a.npar) * a.nrhs;
  if (n == 0) return cudaSuccess;
  if (n >= (int64_t)1 << 31) return cudaErrorInvalidValue;  // thread indices are 32-bit
  const int threads = 128;
  const unsigned blocks = (unsigned)((n + threads - 1) / threads);
  // several right-hand sides: RHS-blocked variant (not for FP64, which is
  // bound by the FP64 pipe, nor for the residual / add epilogues)
  const int rbmax = rhs_block_limit();

  if constexpr (PIN == P32 && POUT == P32 && PG != P64) {
    cudaError_t e = cudaSuccess;
    if (epi == EPI_D && launch_stage<PG>(a, dagger, st, &e)) return e;
  }

  if constexpr (PG != P64 && PG != PDF) {
  if (rbmax >= 2 && (epi == EPI_D || epi == EPI_AINV) && a.nrhs >= 2 && a.nrhs % 2 == 0) {
    // measured on 32^4: blocks of 4 win from 16 RHS up, blocks of 2 below
    const int NBsel = (a.nrhs % 4 == 0 && a.nrhs >= 16 && rbmax >= 4) ? 4 : 2;
    a.fblk = make_fastdiv((uint32_t)((a.nrhs + NBsel - 1) / NBsel));
    const int64_t nt = launch_sites(a.g, a.npar) * ((a.nrhs + NBsel - 1) / NBsel);
    const unsigned bl = (unsigned)((nt + threads - 1) / threads);
    const int key = (epi == EPI_D ? 0 : 4) + (dagger ? 2 : 0) + (NBsel == 4 ? 1 : 0);
    switch (key) {
      case 0: k_hop_rb<PG, PIN, POUT, false, EPI_D, 2><<<bl, threads, 0, st>>>(a); break;
      case 1: k_hop_rb<PG, PIN, POUT, false, EPI_D, 4><<<bl, threads, 0, st>>>(a); break;
      case 2: k_hop_rb<PG, PIN, POUT, true, EPI_D, 2><<<bl, threads, 0, st>>>(a); break;
      case 3: k_hop_rb<PG, PIN, POUT, true, EPI_D, 4><<<bl, threads, 0, st>>>(a); break;
      case 4: k_hop_rb<PG, PIN, POUT, false, EPI_AINV, 2><<<bl, threads, 0, st>>>(a); break;
      case 5: k_hop_rb<PG, PIN, POUT, false, EPI_AINV, 4><<<bl, threads, 0, st>>>(a); break;
      case 6: k_hop_rb<PG, PIN, POUT, true, EPI_AINV, 2><<<bl, threads, 0, st>>>(a); break;
      default: k_hop_rb<PG, PIN, POUT, true, EPI_AINV, 4><<<bl, threads, 0, st>>>(a); break;
    }
    return cudaGetLastError();
  }
  }
  if constexpr (PG == P32) {
    if (a.recon == 8) return launch_hop_single<PG, PIN, POUT, 8>(a, dagger, epi, blocks, threads, st);
    return launch_hop_single<PG, PIN, POUT, -1>(a, dagger, epi, blocks, threads, st);
  } else {
    if (PG == P16 && a.recon) return launch_hop_single<PG, PIN, POUT, PG == P16 ? 12 : 0>(a, dagger, epi, blocks, threads, st);
    return launch_hop_single<PG, PIN, POUT, 0>(a, dagger, epi, blocks, threads, st);
  }
}

// One right-hand side, EPI_D, out written in FP32 or FP16: the stencil plus
// norm_out[0] = (|out|^2, 0), reduced in a fixed order (deterministic).
// `partials` holds at least hop_norm_blocks(launch sites) complex doubles
// plus the reduction's own scratch (blas_reduce_scratch(blocks, 1)).
template <int PG, int PIN, int POUT>
cudaError_t launch_hop_norm(const HopArgs& args, bool dagger, double2* partials, int64_t npartials,
                            double2* norm_out, cudaStream_t st) {
  if (args.nrhs != 1) return cudaErrorInvalidValue;
  HopArgs a = args;
  prepare_divs(a.g);
  a.fblk = make_fastdiv(1u);
  const int64_t n = launch_sites(a.g, a.npar);
  if (n == 0 || n >= (int64_t)1 << 31) return cudaErrorInvalidValue;
  const int threads = 128;
  const int64_t blocks = hop_norm_blocks(n);
  if (blocks > INT32_MAX || blocks + blas_reduce_scratch((int)blocks, 1) > npartials) return cudaErrorInvalidValue;
  const unsigned nb = (unsigned)blocks;
  if constexpr (PG == P32) {
    if (a.recon == 8) {
      if (dagger)
        k_hop_norm<PG, PIN, POUT, true, 8><<<nb, threads, 0, st>>>(a, partials);
      else
        k_hop_norm<PG, PIN, POUT, false, 8><<<nb, threads, 0, st>>>(a, partials);
    } else if (dagger) {
      k_hop_norm<PG, PIN, POUT, true, -1><<<nb, threads, 0, st>>>(a, partials);
    } else {
      k_hop_norm<PG, PIN, POUT, false, -1><<<nb, threads, 0, st>>>(a, partials);
    }
  } else {
    constexpr int LF = PG == P16 ? 12 : 0;
    if (PG == P16 && a.recon) {
      if (dagger)
        k_hop_norm<PG, PIN, POUT, true, LF><<<nb, threads, 0, st>>>(a, partials);
      else
        k_hop_norm<PG, PIN, POUT, false, LF><<<nb, threads, 0, st>>>(a, partials);
    } else if (dagger) {
      k_hop_norm<PG, PIN, POUT, true><<<nb, threads, 0, st>>>(a, partials);
    } else {
      k_hop_norm<PG, PIN, POUT, false><<<nb, threads, 0, st>>>(a, partials);
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return blas_reduce_partials(partials, (int)blocks, 1, norm_out, 0, st, partials + blocks) == 0 ? cudaSuccess
                                                                                   : cudaErrorLaunchFailure;
}

template <int PG, int PIN, int POUT>
cudaError_t launch_block(const BlockArgs& a, cudaStream_t st) {
  const int64_t n = a.Vh * a.nrhs * a.npar;
  if (n == 0) return cudaSuccess;
  const int threads = 128;
  k_block<PG, PIN, POUT><<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(a);
  return cudaGetLastError();
}

#define DD_INSTANTIATE_HOP(PG, PIN, POUT)                                                                  \
  template cudaError_t launch_hop<PG, PIN, POUT>(const HopArgs&, bool, int, cudaStream_t);                \
  template cudaError_t launch_block<PG, PIN, POUT>(const BlockArgs&, cudaStream_t);
#define DD_INSTANTIATE_HOP_NORM(PG, PIN, POUT) \
  template cudaError_t launch_hop_norm<PG, PIN, POUT>(const HopArgs&, bool, double2*, int64_t, double2*, cudaStream_t);

}  // namespace dd
