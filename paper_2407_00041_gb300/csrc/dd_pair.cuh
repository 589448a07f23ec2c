// Paired-RHS fields: the same spinor component of two right-hand sides side
// by side, so that packed FP32x2 instructions (fma.rn.f32x2 and friends)
// process both.  Layouts (N even, NP = N / 2 pairs, RHS 2j and 2j + 1 form
// pair j):
//   FP32 half field: [12 components c][Vh][NP] of float4
//                    (re_2j, re_2j+1, im_2j, im_2j+1)
//   FP16 half field: [6 component pairs g][Vh][NP] of 4 half2
//                    (re of c = 2g, im of c = 2g, re of c = 2g + 1,
//                     im of c = 2g + 1; .x RHS 2j, .y RHS 2j + 1, each divided
//                     by its site scale), then [Vh][N] float scales (scale of
//                     RHS r of site s at s * N + r: the unpaired order)
// Both take the bytes of the unpaired native half field of the same N.
#pragma once

#include "dd_device.cuh"

namespace dd {

// one complex component of two right-hand sides: RHS a in .x, RHS b in .y
struct cx2 {
  float2 re, im;
};

__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// one complex component of two right-hand sides as stored in the paired FP16
// layout: re and im as half2 (RHS a in .x, RHS b in .y), in units of each
// RHS's site scale
struct hx2 {
  __half2 re, im;
};

__device__ __forceinline__ __half2 add2(__half2 a, __half2 b) { return __hadd2(a, b); }
__device__ __forceinline__ __half2 sub2(__half2 a, __half2 b) { return __hsub2(a, b); }

// ---- paired field access ----
// Load the 12 components of RHS pair index i (= site * NP + j); FP16 values
// come without their site scales, which are returned (FP32: (1, 1)).
template <int P>
__device__ __forceinline__ float2 load_pair(const HalfField& f, int64_t gstride, int64_t i, cx2 v[12]) {
  if constexpr (P == P32) {
    const float4* b = reinterpret_cast<const float4*>(f.base) + i;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      const float4 t = __ldg(b + c * gstride);
      v[c].re = make_float2(t.x, t.y);
      v[c].im = make_float2(t.z, t.w);
    }
    return make_float2(1.f, 1.f);
  } else {
    static_assert(P == P16, "paired fields are FP32 or FP16");
    const uint4* b = reinterpret_cast<const uint4*>(f.base) + i;
#pragma unroll
    for (int g = 0; g < 6; ++g) {
      const uint4 t = __ldg(b + g * gstride);
      v[2 * g].re = __half22float2(*reinterpret_cast<const __half2*>(&t.x));
      v[2 * g].im = __half22float2(*reinterpret_cast<const __half2*>(&t.y));
      v[2 * g + 1].re = __half22float2(*reinterpret_cast<const __half2*>(&t.z));
      v[2 * g + 1].im = __half22float2(*reinterpret_cast<const __half2*>(&t.w));
    }
    // scales of RHS 2j and 2j + 1 of the site: floats site * N + 2j = 2 i
    return __ldg(reinterpret_cast<const float2*>(f.scale) + i);
  }
}

// The 12 stored FP16 components of RHS pair index i without widening; returns
// the site scales of the two RHS.
__device__ __forceinline__ float2 load_pair_h(const HalfField& f, int64_t gstride, int64_t i, hx2 v[12]) {
  const uint4* b = reinterpret_cast<const uint4*>(f.base) + i;
#pragma unroll
  for (int g = 0; g < 6; ++g) {
    const uint4 t = __ldg(b + g * gstride);
    v[2 * g].re = *reinterpret_cast<const __half2*>(&t.x);
    v[2 * g].im = *reinterpret_cast<const __half2*>(&t.y);
    v[2 * g + 1].re = *reinterpret_cast<const __half2*>(&t.z);
    v[2 * g + 1].im = *reinterpret_cast<const __half2*>(&t.w);
  }
  return __ldg(reinterpret_cast<const float2*>(f.scale) + i);
}

// Store RHS pair index i; FP16 divides each RHS by its own site scale
// (max |re|, |im| over its 24 reals), as store_spinor does.
template <int P, bool STREAM = true>
__device__ __forceinline__ void store_pair(const HalfField& f, int64_t gstride, int64_t i, const cx2 v[12]) {
  if constexpr (P == P32) {
    float4* b = reinterpret_cast<float4*>(f.base) + i;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      const float4 d = make_float4(v[c].re.x, v[c].re.y, v[c].im.x, v[c].im.y);
      if (STREAM) __stcs(b + c * gstride, d); else b[c * gstride] = d;
    }
  } else {
    float ma = 0.f, mb = 0.f;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      ma = fmaxf(ma, fmaxf(fabsf(v[c].re.x), fabsf(v[c].im.x)));
      mb = fmaxf(mb, fmaxf(fabsf(v[c].re.y), fabsf(v[c].im.y)));
    }
    const float ia = ma > 0.f ? 1.f / ma : 0.f, ib = mb > 0.f ? 1.f / mb : 0.f;
    uint4* b = reinterpret_cast<uint4*>(f.base) + i;
#pragma unroll
    for (int g = 0; g < 6; ++g) {
      const cx2 a0 = v[2 * g], a1 = v[2 * g + 1];
      const __half2 q0 = __floats2half2_rn(a0.re.x * ia, a0.re.y * ib);
      const __half2 q1 = __floats2half2_rn(a0.im.x * ia, a0.im.y * ib);
      const __half2 q2 = __floats2half2_rn(a1.re.x * ia, a1.re.y * ib);
      const __half2 q3 = __floats2half2_rn(a1.im.x * ia, a1.im.y * ib);
      const uint4 d = make_uint4(*reinterpret_cast<const unsigned*>(&q0), *reinterpret_cast<const unsigned*>(&q1),
                                 *reinterpret_cast<const unsigned*>(&q2), *reinterpret_cast<const unsigned*>(&q3));
      if (STREAM) __stcs(b + g * gstride, d); else b[g * gstride] = d;
    }
    const float2 m = make_float2(ma, mb);
    float2* sp = reinterpret_cast<float2*>(f.scale) + i;
    if (STREAM) __stcs(sp, m); else *sp = m;
  }
}

}  // namespace dd
