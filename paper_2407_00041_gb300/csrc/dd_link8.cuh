// Eight-real FP32 storage of an SU(3) link (Section 2.3 stores the links of
// the stencil; an SU(3) matrix has eight real degrees of freedom, Section
// 1.1).  Two float4 words per link:
//   w0 = (W01, W02)                       row 0 without its pivot
//   w1 = (W10, arg(W00) / pi, arg(W20) / pi)
// of the matrix W = S U C_k, where C_k cyclically shifts the columns so that
// the pivot W00 is the element of row 0 of largest modulus (|W00|^2 >= 1/3),
// and S either keeps rows 1, 2 or replaces them by (row 2, -row 1) so that
// the stored W10 is the smaller of the two lower entries of column 0
// (|W20|^2 >= n / 2 with n = |W01|^2 + |W02|^2).  Both maps keep det = 1.
// The choice (k in 0..2, swap) sits in the lowest mantissa bits of w1.z
// (k & 1), w1.w (k >> 1) and w1.x (swap), a change of at most one unit in
// the last place of those values.
//
// Reconstruction, from unitarity and det W = 1:
//   |W00| = sqrt(1 - n),  |W20| = sqrt(n - |W10|^2)
//   (W11, W12) solves  W11 conj(W01) + W12 conj(W02) = -W10 conj(W00)
//                      W01 W12 - W02 W11             = conj(W20)
//   (determinant n), and row 2 = conj(row 0 x row 1).
// With both magnitudes taken where they are large and the 2 x 2 solve scaled
// by n, every element is recovered to a few FP32 units in the last place.
#pragma once

#include <cuda_runtime.h>

namespace dd {

__device__ __forceinline__ unsigned link8_bit(float v) { return __float_as_uint(v) & 1u; }
__device__ __forceinline__ float link8_with_bit(float v, unsigned b) {
  return __uint_as_float((__float_as_uint(v) & ~1u) | b);
}

// Encode one link (row-major double2 u[9]) into the two words.
__device__ __forceinline__ void link8_encode(const double2 u[9], float4& w0, float4& w1) {
  auto m2 = [](double2 a) { return a.x * a.x + a.y * a.y; };
  int k = 0;
  if (m2(u[1]) > m2(u[k])) k = 1;
  if (m2(u[2]) > m2(u[k])) k = 2;
  double2 w[9];  // W[:, j] = U[:, (j + k) mod 3]
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int j = 0; j < 3; ++j) w[3 * r + j] = u[3 * r + (j + k) % 3];
  const bool swap = m2(w[3]) > m2(w[6]);
  if (swap) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const double2 t = w[3 + j];
      w[3 + j] = w[6 + j];
      w[6 + j] = make_double2(-t.x, -t.y);
    }
  }
  const double inv_pi = 0.31830988618379067154;
  w0 = make_float4((float)w[1].x, (float)w[1].y, (float)w[2].x, (float)w[2].y);
  const float ta = (float)(atan2(w[0].y, w[0].x) * inv_pi);
  const float tc = (float)(atan2(w[6].y, w[6].x) * inv_pi);
  w1 = make_float4(link8_with_bit((float)w[3].x, swap ? 1u : 0u), (float)w[3].y, link8_with_bit(ta, k & 1),
                   link8_with_bit(tc, (unsigned)k >> 1));
}

// Decode the two words into the row-major FP32 link u[9] (re, im pairs).
__device__ __forceinline__ void link8_decode(const float4 w0, const float4 w1, float2 u[9]) {
  const float a1r = w0.x, a1i = w0.y, a2r = w0.z, a2i = w0.w, b0r = w1.x, b0i = w1.y;
  const float n = fmaf(a1r, a1r, fmaf(a1i, a1i, fmaf(a2r, a2r, a2i * a2i)));
  const float ma = sqrtf(fmaxf(1.f - n, 0.f));
  const float mc = sqrtf(fmaxf(n - fmaf(b0r, b0r, b0i * b0i), 0.f));
  float sa, ca, sc, cc;
  sincospif(w1.z, &sa, &ca);
  sincospif(w1.w, &sc, &cc);
  const float a0r = ma * ca, a0i = ma * sa, c0r = mc * cc, c0i = mc * sc;
  // X = -W10 conj(W00), Y = conj(W20)
  const float xr = -fmaf(b0r, a0r, b0i * a0i), xi = -fmaf(b0i, a0r, -b0r * a0i);
  const float yr = c0r, yi = -c0i;
  const float in = 1.f / n;
  // W11 = (W01 X - conj(W02) Y) / n,  W12 = (W02 X + conj(W01) Y) / n
  const float b1r = (fmaf(a1r, xr, -a1i * xi) - fmaf(a2r, yr, a2i * yi)) * in;
  const float b1i = (fmaf(a1r, xi, a1i * xr) - fmaf(a2r, yi, -a2i * yr)) * in;
  const float b2r = (fmaf(a2r, xr, -a2i * xi) + fmaf(a1r, yr, a1i * yi)) * in;
  const float b2i = (fmaf(a2r, xi, a2i * xr) + fmaf(a1r, yi, -a1i * yr)) * in;
  // row 2 = conj(row 0 x row 1): W21 = conj(W02 W10 - W00 W12), W22 = conj(W00 W11 - W01 W10)
  const float c1r = fmaf(a2r, b0r, -a2i * b0i) - fmaf(a0r, b2r, -a0i * b2i);
  const float c1i = -(fmaf(a2r, b0i, a2i * b0r) - fmaf(a0r, b2i, a0i * b2r));
  const float c2r = fmaf(a0r, b1r, -a0i * b1i) - fmaf(a1r, b0r, -a1i * b0i);
  const float c2i = -(fmaf(a0r, b1i, a0i * b1r) - fmaf(a1r, b0i, a1i * b0r));
  float2 w[9] = {make_float2(a0r, a0i), make_float2(a1r, a1i), make_float2(a2r, a2i),
                 make_float2(b0r, b0i), make_float2(b1r, b1i), make_float2(b2r, b2i),
                 make_float2(c0r, c0i), make_float2(c1r, c1i), make_float2(c2r, c2i)};
  if (link8_bit(w1.x)) {  // stored rows were (row 2, -row 1)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float2 t = w[3 + j];
      w[3 + j] = make_float2(-w[6 + j].x, -w[6 + j].y);
      w[6 + j] = t;
    }
  }
  const unsigned k = link8_bit(w1.z) | (link8_bit(w1.w) << 1);
  // U[:, (j + k) mod 3] = W[:, j]
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float2 x0 = w[3 * r], x1 = w[3 * r + 1], x2 = w[3 * r + 2];
    u[3 * r] = k == 0 ? x0 : k == 1 ? x2 : x1;
    u[3 * r + 1] = k == 0 ? x1 : k == 1 ? x0 : x2;
    u[3 * r + 2] = k == 0 ? x2 : k == 1 ? x1 : x0;
  }
}

}  // namespace dd
