// Device-side types shared by the library's kernels: complex arithmetic,
// precision traits, native field accessors and even-odd lattice geometry.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace dd {

// ---------------------------------------------------------------- complex
template <typename R>
struct cx {
  R re, im;
};

template <typename R>
__device__ __forceinline__ cx<R> mk(R a, R b) {
  cx<R> c;
  c.re = a;
  c.im = b;
  return c;
}
template <typename R>
__device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) {
  return mk(a.re + b.re, a.im + b.im);
}
template <typename R>
__device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) {
  return mk(a.re - b.re, a.im - b.im);
}
template <typename R>
__device__ __forceinline__ cx<R> operator*(R s, cx<R> a) {
  return mk(s * a.re, s * a.im);
}
// a * b
template <typename R>
__device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
// acc + a * b
template <typename R>
__device__ __forceinline__ cx<R> cfma(cx<R> a, cx<R> b, cx<R> acc) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
  return acc;
}
// acc + conj(a) * b
template <typename R>
__device__ __forceinline__ cx<R> cfmac(cx<R> a, cx<R> b, cx<R> acc) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
  return acc;
}
// acc + s * a (s real)
template <typename R>
__device__ __forceinline__ cx<R> caxpy(R s, cx<R> a, cx<R> acc) {
  acc.re = fma(s, a.re, acc.re);
  acc.im = fma(s, a.im, acc.im);
  return acc;
}
// i * a, -i * a
template <typename R>
__device__ __forceinline__ cx<R> mul_i(cx<R> a) {
  return mk(-a.im, a.re);
}
template <typename R>
__device__ __forceinline__ cx<R> mul_mi(cx<R> a) {
  return mk(a.im, -a.re);
}
template <typename R>
__device__ __forceinline__ cx<R> neg(cx<R> a) {
  return mk(-a.re, -a.im);
}
template <typename R>
__device__ __forceinline__ cx<R> zero() {
  return mk(R(0), R(0));
}


// ---------------------------------------------------------------- FP32 pairs
// A double-word number x = h + l of two FP32 values with |l| <= ulp(h) / 2
// (Dekker, "A floating-point technique for extending the available
// precision", 1971): about 48 significant bits, so FP64-level accuracy from
// the FP32 pipes.  Building blocks: Knuth's TwoSum and Dekker's Fast2Sum
// (exact sums), and the exact product error by FMA.  The sum below adds the
// low parts without a second TwoSum (an error of about 2^-48 (|a| + |b|)),
// the product drops l_a l_b (about 2^-48 |a b|).  Every operation is an
// intrinsic with its own rounding, so the compiler cannot contract a
// product into a following sum.
struct df;
__device__ __forceinline__ df df_fma(df a, df b, df c);
struct df {
  float h, l;
  df() = default;
  __host__ __device__ __forceinline__ df(float hi, float lo) : h(hi), l(lo) {}
  __host__ __device__ __forceinline__ df(float x) : h(x), l(0.f) {}
  __host__ __device__ __forceinline__ df(int x) : h((float)x), l(0.f) {}
  // round to the nearest FP32, then the FP32 nearest to the exact remainder
  // (x - h is exact in FP64)
  __host__ __device__ __forceinline__ df(double x) : h((float)x), l((float)(x - (double)(float)x)) {}
  __host__ __device__ __forceinline__ explicit operator double() const { return (double)h + (double)l; }
  __host__ __device__ __forceinline__ explicit operator float() const { return h + l; }
  // fma(df, df, df) for the generic complex helpers, defined as a friend so
  // that only argument-dependent lookup finds it (an ordinary fma in this
  // namespace would hide ::fma for the FP32 / FP64 callers)
  friend __device__ __forceinline__ df fma(df a, df b, df c) { return df_fma(a, b, c); }
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// |a| >= |b| (or a = 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ df operator-(df a) { return df(-a.h, -a.l); }
__device__ __forceinline__ df operator+(df a, df b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  df r;
  fast_two_sum(s, e, r.h, r.l);
  return r;
}
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  df r;
  fast_two_sum(p, e, r.h, r.l);
  return r;
}
__device__ __forceinline__ df& operator*=(df& a, df b) { return a = a * b; }
// c + a b
__device__ __forceinline__ df df_fma(df a, df b, df c) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  float s, t;
  two_sum(c.h, p, s, t);
  t = __fadd_rn(t, __fadd_rn(c.l, e));
  df r;
  fast_two_sum(s, t, r.h, r.l);
  return r;
}

// An FP64 value as a pair without FP64 instructions (the FP64 pipe of this
// GPU runs at 1/64 of the FP32 rate): h = x truncated to 24 significant
// bits, built from the sign, the rebased exponent and the top 23 fraction
// bits; l = the next 23 fraction bits as an exact integer (the 2^23 magic
// constant) times the power of two of their place.  |x - h - l| < 2^-46 |x|.
// |x| < 2^-126 (and zero) gives (0, 0); |x| >= 2^128 is outside the range.
__device__ __forceinline__ df df_split(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
  const int e = (int)((hi >> 20) & 0x7FFu);
  const unsigned sgn = hi & 0x80000000u;
  const float h = __uint_as_float(sgn | ((unsigned)(e - 896) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
  const float r = __fsub_rn(__uint_as_float(0x4B000000u | ((lo >> 6) & 0x7FFFFFu)), 8388608.f);
  const int se = e - 942;  // FP32 exponent field of 2^(e - 1023 - 46)
  const float l = __fmul_rn(r, __uint_as_float(sgn | ((unsigned)(se > 0 ? se : 0) << 23)));
  return e > 896 ? df(h, l) : df(0.f, 0.f);
}

// Complex multiply-accumulate of FP32 pairs for the short sums of the stencil
// (three terms of a colour product, six of a block row): each step keeps the
// exact product error and the exact error of the high-part sum in the low
// part without renormalising; renorm restores |l| <= ulp(h) / 2 at the end
// of the sum.  About 20% fewer FP32 operations than df_fma per step.
__device__ __forceinline__ df df_fma_lazy(df a, df b, df c) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  float s, t;
  two_sum(c.h, p, s, t);
  return df(s, __fadd_rn(c.l, __fadd_rn(t, e)));
}
__device__ __forceinline__ cx<df> cfma(cx<df> a, cx<df> b, cx<df> acc) {
  acc.re = df_fma_lazy(a.re, b.re, acc.re);
  acc.re = df_fma_lazy(-a.im, b.im, acc.re);
  acc.im = df_fma_lazy(a.re, b.im, acc.im);
  acc.im = df_fma_lazy(a.im, b.re, acc.im);
  return acc;
}
__device__ __forceinline__ cx<df> cfmac(cx<df> a, cx<df> b, cx<df> acc) {
  acc.re = df_fma_lazy(a.re, b.re, acc.re);
  acc.re = df_fma_lazy(a.im, b.im, acc.re);
  acc.im = df_fma_lazy(a.re, b.im, acc.im);
  acc.im = df_fma_lazy(-a.im, b.re, acc.im);
  return acc;
}
// c + s a: for s = +-1 (the sign of a hop) a sum of the high parts with its
// exact error kept in the low part, else df_fma_lazy
__device__ __forceinline__ df df_axpy_lazy(df s, df a, df c) {
  if (s.l == 0.f && fabsf(s.h) == 1.f) {
    const float ah = s.h > 0.f ? a.h : -a.h, al = s.h > 0.f ? a.l : -a.l;
    float h, t;
    two_sum(c.h, ah, h, t);
    return df(h, __fadd_rn(c.l, __fadd_rn(t, al)));
  }
  return df_fma_lazy(s, a, c);
}
__device__ __forceinline__ cx<df> caxpy(df s, cx<df> a, cx<df> acc) {
  acc.re = df_axpy_lazy(s, a.re, acc.re);
  acc.im = df_axpy_lazy(s, a.im, acc.im);
  return acc;
}
template <typename R>
__device__ __forceinline__ void renorm(cx<R>&) {}
__device__ __forceinline__ void renorm(cx<df>& z) {
  float h, l;
  fast_two_sum(z.re.h, z.re.l, h, l);
  z.re = df(h, l);
  fast_two_sum(z.im.h, z.im.l, h, l);
  z.im = df(h, l);
}

// ---------------------------------------------------------------- precisions
// PDF: FP64-accurate arithmetic in FP32 pairs (df) on fields, links and
// blocks stored as FP32 pairs (one complex = float4 (re.h, re.l, im.h, im.l),
// 16 bytes like FP64, in the FP64 layouts).
enum { P64 = 1, P32 = 2, P16 = 4, PDF = 8 };

// Storage of links and self-coupling blocks: one complex (or one pair of
// reals) per element.
template <int P>
struct Store;
template <>
struct Store<P64> {
  using real = double;
  using elem = double2;  // complex
};
template <>
struct Store<P32> {
  using real = float;
  using elem = float2;
};
template <>
struct Store<P16> {
  using real = float;
  using elem = __half2;
};
template <>
struct Store<PDF> {
  using real = df;
  using elem = float4;
};

__device__ __forceinline__ cx<df> df_cx(float4 v) { return mk(df(v.x, v.y), df(v.z, v.w)); }

template <int P>
__device__ __forceinline__ cx<typename Store<P>::real> ld_elem(const typename Store<P>::elem* p) {
  if constexpr (P == PDF) {
    return df_cx(__ldg(p));
  } else if constexpr (P == P64) {
    double2 v = __ldg(p);
    return mk(v.x, v.y);
  } else if constexpr (P == P32) {
    float2 v = __ldg(p);
    return mk(v.x, v.y);
  } else {
    unsigned int u = __ldg(reinterpret_cast<const unsigned int*>(p));
    __half2 h = *reinterpret_cast<__half2*>(&u);
    float2 f = __half22float2(h);
    return mk(f.x, f.y);
  }
}

// Streaming load (data touched once per apply: self-coupling blocks).
template <int P>
__device__ __forceinline__ cx<typename Store<P>::real> ld_elem_stream(const typename Store<P>::elem* p) {
  if constexpr (P == PDF) {
    return df_cx(__ldcs(p));
  } else if constexpr (P == P64) {
    double2 v = __ldcs(p);
    return mk(v.x, v.y);
  } else if constexpr (P == P32) {
    float2 v = __ldcs(p);
    return mk(v.x, v.y);
  } else {
    unsigned int u = __ldcs(reinterpret_cast<const unsigned int*>(p));
    __half2 h = *reinterpret_cast<__half2*>(&u);
    float2 f = __half22float2(h);
    return mk(f.x, f.y);
  }
}

template <int P>
__device__ __forceinline__ void st_elem(typename Store<P>::elem* p, cx<typename Store<P>::real> v) {
  if constexpr (P == PDF) {
    *p = make_float4(v.re.h, v.re.l, v.im.h, v.im.l);
  } else if constexpr (P == P64) {
    *p = make_double2(v.re, v.im);
  } else if constexpr (P == P32) {
    *p = make_float2(v.re, v.im);
  } else {
    *p = __floats2half2_rn(v.re, v.im);
  }
}

// ---------------------------------------------------------------- spinor fields
// A half field (sites of one parity, Vh sites, N right-hand sides) in native
// layout.  `base` points at the first component group; `gstride` is the
// distance between component groups in group units (= Vh * N); FP16 fields
// carry `scale` [Vh][N].
struct HalfField {
  void* base;
  float* scale;
};

template <int P>
struct SpinorStore;
template <>
struct SpinorStore<P64> {
  static constexpr int GROUPS = 12;
  using group = double2;
  using real = double;
};
template <>
struct SpinorStore<P32> {
  static constexpr int GROUPS = 6;
  using group = float4;
  using real = float;
};
template <>
struct SpinorStore<P16> {
  static constexpr int GROUPS = 3;
  using group = uint4;
  using real = float;
};
template <>
struct SpinorStore<PDF> {
  static constexpr int GROUPS = 12;
  using group = float4;
  using real = df;
};

template <int P>
__host__ __device__ inline size_t half_field_bytes(int64_t Vh, int nrhs) {
  size_t n = (size_t)Vh * (size_t)nrhs;
  if (P == P64 || P == PDF) return n * 12 * 16;
  if (P == P32) return n * 6 * 16;
  return n * 3 * 16 + n * 4;
}

// Load the 12 components of site-rhs index `i` (= site * N + r).
template <int P, typename R>
__device__ __forceinline__ void load_spinor(const HalfField& f, int64_t gstride, int64_t i, cx<R> v[12]) {
  if constexpr (P == PDF) {
    const float4* b = reinterpret_cast<const float4*>(f.base) + i;
#pragma unroll
    for (int c = 0; c < 12; ++c) v[c] = df_cx(__ldg(b + c * gstride));
  } else if constexpr (P == P64) {
    const double2* b = reinterpret_cast<const double2*>(f.base) + i;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      double2 t = __ldg(b + c * gstride);
      if constexpr (std::is_same<R, df>::value)
        v[c] = mk(df_split(t.x), df_split(t.y));
      else
        v[c] = mk<R>(t.x, t.y);
    }
  } else if constexpr (P == P32) {
    const float4* b = reinterpret_cast<const float4*>(f.base) + i;
#pragma unroll
    for (int g = 0; g < 6; ++g) {
      float4 t = __ldg(b + g * gstride);
      v[2 * g] = mk<R>(t.x, t.y);
      v[2 * g + 1] = mk<R>(t.z, t.w);
    }
  } else {
    const uint4* b = reinterpret_cast<const uint4*>(f.base) + i;
    const float s = __ldg(f.scale + i);
#pragma unroll
    for (int g = 0; g < 3; ++g) {
      uint4 t = __ldg(b + g * gstride);
      unsigned int w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        __half2 h = *reinterpret_cast<__half2*>(&w[k]);
        float2 ff = __half22float2(h);
        v[4 * g + k] = mk<R>(ff.x * s, ff.y * s);
      }
    }
  }
}

// A neighbour spinor for the hopping term: FP16 values are returned without
// their per-site scale, which is returned instead (and folded by the caller
// into the hop's accumulation); FP32 / FP64 return 1.
template <int P, typename R>
__device__ __forceinline__ R load_spinor_unscaled(const HalfField& f, int64_t gstride, int64_t i, cx<R> v[12]) {
  if constexpr (P == P16) {
    const uint4* b = reinterpret_cast<const uint4*>(f.base) + i;
    const float s = __ldg(f.scale + i);
#pragma unroll
    for (int g = 0; g < 3; ++g) {
      uint4 t = __ldg(b + g * gstride);
      unsigned int w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float2 ff = __half22float2(*reinterpret_cast<__half2*>(&w[k]));
        v[4 * g + k] = mk<R>(ff.x, ff.y);
      }
    }
    return (R)s;
  } else {
    load_spinor<P, R>(f, gstride, i, v);
    return (R)1;
  }
}

// STREAM: evict-first stores (outputs the kernel does not read again)
template <int P, typename R, bool STREAM = false>
__device__ __forceinline__ void store_spinor(const HalfField& f, int64_t gstride, int64_t i, const cx<R> v[12]) {
  if constexpr (P == PDF) {
    float4* b = reinterpret_cast<float4*>(f.base) + i;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      const float4 d = make_float4(v[c].re.h, v[c].re.l, v[c].im.h, v[c].im.l);
      if (STREAM) __stcs(b + c * gstride, d); else b[c * gstride] = d;
    }
  } else if constexpr (P == P64) {
    double2* b = reinterpret_cast<double2*>(f.base) + i;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      const double2 d = make_double2((double)v[c].re, (double)v[c].im);
      if (STREAM) __stcs(b + c * gstride, d); else b[c * gstride] = d;
    }
  } else if constexpr (P == P32) {
    float4* b = reinterpret_cast<float4*>(f.base) + i;
#pragma unroll
    for (int g = 0; g < 6; ++g) {
      const float4 d = make_float4((float)v[2 * g].re, (float)v[2 * g].im, (float)v[2 * g + 1].re,
                                   (float)v[2 * g + 1].im);
      if (STREAM) __stcs(b + g * gstride, d); else b[g * gstride] = d;
    }
  } else {
    float m = 0.f;
#pragma unroll
    for (int c = 0; c < 12; ++c) m = fmaxf(m, fmaxf(fabsf((float)v[c].re), fabsf((float)v[c].im)));
    const float inv = m > 0.f ? 1.f / m : 0.f;
    uint4* b = reinterpret_cast<uint4*>(f.base) + i;
#pragma unroll
    for (int g = 0; g < 3; ++g) {
      unsigned int w[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        __half2 h = __floats2half2_rn((float)v[4 * g + k].re * inv, (float)v[4 * g + k].im * inv);
        w[k] = *reinterpret_cast<unsigned int*>(&h);
      }
      const uint4 d = make_uint4(w[0], w[1], w[2], w[3]);
      if (STREAM) __stcs(b + g * gstride, d); else b[g * gstride] = d;
    }
    if (STREAM) __stcs(f.scale + i, m); else f.scale[i] = m;
  }
}

// ---------------------------------------------------------------- geometry
// Even-odd geometry.  A site of parity p has compact index s = lex / 2
// (valid because nX is even), so the sites of one parity keep their
// lexicographic order.
// Division by a divisor fixed for a launch, by multiply and shift
// (Granlund and Montgomery, "Division by invariant integers using
// multiplication", 1994): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, n / d = (mulhi(n, m) + n) >> l, exact
// for 0 <= n < 2^31 (the sum then stays below 2^32).
struct FastDiv {
  uint32_t d, m, l;
};

inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  f.l = 0;
  while ((1ull << f.l) < d) ++f.l;
  f.m = (uint32_t)((((1ull << 32) * ((1ull << f.l) - d)) / d) + 1);
  return f;
}

__device__ __forceinline__ int fdiv(int n, const FastDiv& f) {
  return (int)((__umulhi((uint32_t)n, f.m) + (uint32_t)n) >> f.l);
}

struct Geom {
  int n[4];       // nT, nZ, nY, nX
  int stride[4];  // lexicographic strides of T, Z, Y, X
  int Vh;         // sites per parity
  float t_bc;     // sign of hops across the time boundary
  int zblock;     // traversal of full-lattice launches: Z-slabs of this depth (divides nZ)
  int t0, nt;     // full-lattice launches cover the time slices t0 .. t0 + nt - 1
  // full-lattice launches take the sites of `rseg` consecutive X-rows
  // parity by parity (rseg * nX / 2 a multiple of 32 where nY allows), so a
  // warp reads and writes one parity's arrays only
  int rseg;
  // divisions by nX, nY, nZ, zblock, nt, nX / 2 and the segment sizes (set by
  // prepare_divs)
  FastDiv fx, fy, fz, fzb, fnt, fhx, fseg;
};

inline void prepare_divs(Geom& g) {
  g.fx = make_fastdiv((uint32_t)g.n[3]);
  g.fy = make_fastdiv((uint32_t)g.n[2]);
  g.fz = make_fastdiv((uint32_t)g.n[1]);
  g.fzb = make_fastdiv((uint32_t)g.zblock);
  g.fnt = make_fastdiv((uint32_t)g.nt);
  const int hx = g.n[3] / 2;
  g.fhx = make_fastdiv((uint32_t)hx);
  g.rseg = 1;
  for (int r = 1; r <= g.n[2]; ++r)
    if (g.n[2] % r == 0 && (r * hx) % 32 == 0) {
      g.rseg = r;
      break;
    }
  g.fseg = make_fastdiv((uint32_t)(g.rseg * g.n[3]));
}

// Output sites of a launch: both parities of the slices t0 .. t0 + nt - 1,
// or one parity of the whole lattice.
__host__ __device__ __forceinline__ int64_t launch_sites(const Geom& g, int npar) {
  return npar == 2 ? (int64_t)g.nt * g.stride[0] : (int64_t)g.Vh;
}

struct SiteCoord {
  int c[4];  // t, z, y, x
  int lex;
};

__device__ __forceinline__ SiteCoord site_coords(const Geom& g, int s, int p) {
  SiteCoord sc;
  const int lex2 = 2 * s;
  const int r1 = fdiv(s, g.fhx);  // = lex2 / nX, nX even
  const int x0 = lex2 - r1 * g.n[3];
  const int r2 = fdiv(r1, g.fy);
  sc.c[2] = r1 - r2 * g.n[2];
  sc.c[0] = fdiv(r2, g.fz);
  sc.c[1] = r2 - sc.c[0] * g.n[1];
  sc.c[3] = x0 + ((p ^ (sc.c[0] + sc.c[1] + sc.c[2])) & 1);
  sc.lex = r1 * g.n[3] + sc.c[3];
  return sc;
}

__device__ __forceinline__ SiteCoord lex_coords(const Geom& g, int lex) {
  SiteCoord sc;
  sc.lex = lex;
  const int r1 = lex / g.n[3];
  sc.c[3] = lex - r1 * g.n[3];
  const int r2 = r1 / g.n[2];
  sc.c[2] = r1 - r2 * g.n[2];
  sc.c[0] = r2 / g.n[1];
  sc.c[1] = r2 - sc.c[0] * g.n[1];
  return sc;
}

// Traversal order of full-lattice launches: slab b of `zblock` Z-planes is
// walked time slice by time slice, rows of X fastest:
//   row = ((b * nt + t - t0) * zblock + zz) * nY + y,  z = b * zblock + zz,
// and the rows are taken in segments of `rseg`: first the parity-0 sites of
// the segment's rows, then its parity-1 sites, so that consecutive threads
// cover consecutive compact sites of one parity (a warp touches one half
// field).  The hops to t +- 1 find their data after one slab-slice of
// traffic (zblock * nY * nX sites) instead of a whole time slice, which
// keeps that reuse inside L2 on large lattices.
__device__ __forceinline__ SiteCoord traversal_coords(const Geom& g, int k) {
  SiteCoord sc;
  // segment of rseg rows: its parity-0 sites, then its parity-1 sites
  const int hx = g.n[3] >> 1;
  const int seg = fdiv(k, g.fseg);
  int w = k - seg * g.rseg * g.n[3];
  const int half = w >= g.rseg * hx ? 1 : 0;
  w -= half * g.rseg * hx;
  const int rr = fdiv(w, g.fhx);
  const int j = w - rr * hx;
  int r = seg * g.rseg + rr;  // row index in traversal order
  int r2 = fdiv(r, g.fy);
  sc.c[2] = r - r2 * g.n[2];
  r = fdiv(r2, g.fzb);
  const int zz = r2 - r * g.zblock;
  r2 = fdiv(r, g.fnt);
  sc.c[0] = r - r2 * g.nt + g.t0;
  sc.c[1] = r2 * g.zblock + zz;
  sc.c[3] = 2 * j + ((half + sc.c[0] + sc.c[1] + sc.c[2]) & 1);
  sc.lex = ((sc.c[0] * g.n[1] + sc.c[1]) * g.n[2] + sc.c[2]) * g.n[3] + sc.c[3];
  return sc;
}

// lexicographic index of the neighbour x + mu (fwd) or x - mu (bwd)
__device__ __forceinline__ int nb_fwd(const Geom& g, const SiteCoord& sc, int mu) {
  return sc.c[mu] == g.n[mu] - 1 ? sc.lex - (g.n[mu] - 1) * g.stride[mu] : sc.lex + g.stride[mu];
}
__device__ __forceinline__ int nb_bwd(const Geom& g, const SiteCoord& sc, int mu) {
  return sc.c[mu] == 0 ? sc.lex + (g.n[mu] - 1) * g.stride[mu] : sc.lex - g.stride[mu];
}

}  // namespace dd
