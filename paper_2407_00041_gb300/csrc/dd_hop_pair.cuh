// Paired-RHS Wilson-clover stencil: one thread computes one output site for
// two right-hand sides with packed FP32x2 arithmetic (fma.rn.f32x2 and
// add.rn.f32x2 through __ffma2_rn / __fadd2_rn / __fmul2_rn).
//
// The operator is the one of dd_hop.cuh (the hopping sum of Eq. 1.13 formed
// through the two-spin projection that the back-substitution after
// Algorithm 3 uses, plus the self coupling of Eq. 2.5).  With FP32 vectors
// every arithmetic step of one right-hand side is the same FP32 operation, in
// the same order, as in the RHS-blocked kernel k_hop_rb, so results are
// bit-identical to it.  With FP16 vectors (and FP16 links) each hop works in
// half2 arithmetic on the stored values, the two lanes of a half2 being the
// two right-hand sides: spin projection by add.f16x2 and the colour product
// by fma.rn.f16x2 (FP16 sums of the six products of a component), then
// widened once per component for the reconstruction; the sum over the hops,
// the site scales and the self coupling stay FP32.  A packed FP32x2 FMA
// occupies the FMA pipe for two cycles and an FP16x2 FMA for one, so this
// halves the pipe time of the colour products, which bound the FP16-storage
// kernel at many right-hand sides; the FP16 sums add about 3e-4 relative
// error per product to the 2.4e-4 of the FP16 storage itself.
// What changes is the data layout, which puts the same component of two
// right-hand sides side by side so that one packed instruction serves both:
//
//   paired FP32 half field (N even, NP = N / 2 pairs):
//     [12 components c][Vh][NP] of float4 (re_2j, re_2j+1, im_2j, im_2j+1)
//   paired FP16 half field:
//     [6 component pairs g][Vh][NP] of 4 half2
//       (re of c = 2g, im of c = 2g, re of c = 2g + 1, im of c = 2g + 1; each
//        half2 holding RHS 2j in .x and 2j + 1 in .y, divided by the site scale)
//     then [Vh][N] float scales (scale of RHS r of site s at s * N + r)
//
// Multiplication of a component by +-i only swaps which pair is the real
// part (and flips a sign), so the spin projection and reconstruction need no
// data movement; link and self-coupling elements are broadcast to both lanes.
#pragma once

#include "dd_hop.cuh"
#include "dd_pair.cuh"

namespace dd {

// Spin projection for colour c: h0 = u0 + T (B_mu l)_0, h1 = u1 + T (B_mu l)_1
// with (u0, u1) the upper and (l0, l1) the lower spin pair and
//   B_T = I, B_Z = -i sigma_3, B_Y = -i sigma_2, B_X = -i sigma_1
// (-i z = (z.im, -z.re), i z = (-z.im, z.re)).
template <int MU, int T, typename C>
__device__ __forceinline__ void proj2(C u0, C u1, C l0, C l1, C& h0, C& h1) {
  if constexpr (MU == 0) {  // b0 = l0, b1 = l1
    if constexpr (T > 0) {
      h0.re = add2(u0.re, l0.re), h0.im = add2(u0.im, l0.im);
      h1.re = add2(u1.re, l1.re), h1.im = add2(u1.im, l1.im);
    } else {
      h0.re = sub2(u0.re, l0.re), h0.im = sub2(u0.im, l0.im);
      h1.re = sub2(u1.re, l1.re), h1.im = sub2(u1.im, l1.im);
    }
  } else if constexpr (MU == 1) {  // b0 = -i l0 = (l0.im, -l0.re), b1 = i l1 = (-l1.im, l1.re)
    if constexpr (T > 0) {
      h0.re = add2(u0.re, l0.im), h0.im = sub2(u0.im, l0.re);
      h1.re = sub2(u1.re, l1.im), h1.im = add2(u1.im, l1.re);
    } else {
      h0.re = sub2(u0.re, l0.im), h0.im = add2(u0.im, l0.re);
      h1.re = add2(u1.re, l1.im), h1.im = sub2(u1.im, l1.re);
    }
  } else if constexpr (MU == 2) {  // b0 = -l1, b1 = l0
    if constexpr (T > 0) {
      h0.re = sub2(u0.re, l1.re), h0.im = sub2(u0.im, l1.im);
      h1.re = add2(u1.re, l0.re), h1.im = add2(u1.im, l0.im);
    } else {
      h0.re = add2(u0.re, l1.re), h0.im = add2(u0.im, l1.im);
      h1.re = sub2(u1.re, l0.re), h1.im = sub2(u1.im, l0.im);
    }
  } else {  // b0 = -i l1 = (l1.im, -l1.re), b1 = -i l0 = (l0.im, -l0.re)
    if constexpr (T > 0) {
      h0.re = add2(u0.re, l1.im), h0.im = sub2(u0.im, l1.re);
      h1.re = add2(u1.re, l0.im), h1.im = sub2(u1.im, l0.re);
    } else {
      h0.re = sub2(u0.re, l1.im), h0.im = add2(u0.im, l1.re);
      h1.re = sub2(u1.re, l0.im), h1.im = add2(u1.im, l0.re);
    }
  }
}

// Reconstruction for colour c: the upper pair gets sg g, the lower pair
// T sg (B_mu^H g) with B^H: T: (g0, g1); Z (i sigma_3): (i g0, -i g1);
// Y (i sigma_2): (g1, -g0); X (i sigma_1): (i g1, i g0).
template <int MU, int T>
__device__ __forceinline__ void recon2(cx2 acc[12], int c, cx2 g0, cx2 g1, float2 sg) {
  acc[c].re = fma2(sg, g0.re, acc[c].re);
  acc[c].im = fma2(sg, g0.im, acc[c].im);
  acc[3 + c].re = fma2(sg, g1.re, acc[3 + c].re);
  acc[3 + c].im = fma2(sg, g1.im, acc[3 + c].im);
  const float2 sb = T > 0 ? sg : neg2(sg);
  const float2 nb = neg2(sb);
  if constexpr (MU == 0) {
    acc[6 + c].re = fma2(sb, g0.re, acc[6 + c].re);
    acc[6 + c].im = fma2(sb, g0.im, acc[6 + c].im);
    acc[9 + c].re = fma2(sb, g1.re, acc[9 + c].re);
    acc[9 + c].im = fma2(sb, g1.im, acc[9 + c].im);
  } else if constexpr (MU == 1) {
    acc[6 + c].re = fma2(nb, g0.im, acc[6 + c].re);
    acc[6 + c].im = fma2(sb, g0.re, acc[6 + c].im);
    acc[9 + c].re = fma2(sb, g1.im, acc[9 + c].re);
    acc[9 + c].im = fma2(nb, g1.re, acc[9 + c].im);
  } else if constexpr (MU == 2) {
    acc[6 + c].re = fma2(sb, g1.re, acc[6 + c].re);
    acc[6 + c].im = fma2(sb, g1.im, acc[6 + c].im);
    acc[9 + c].re = fma2(nb, g0.re, acc[9 + c].re);
    acc[9 + c].im = fma2(nb, g0.im, acc[9 + c].im);
  } else {
    acc[6 + c].re = fma2(nb, g1.im, acc[6 + c].re);
    acc[6 + c].im = fma2(sb, g1.re, acc[6 + c].im);
    acc[9 + c].re = fma2(nb, g0.im, acc[9 + c].re);
    acc[9 + c].im = fma2(sb, g0.re, acc[9 + c].im);
  }
}

// acc += sg (I + T gamma_mu) (x) W psi for a pair of RHS, W = U (ADJ = false)
// or U^H (ADJ = true): projection, the two colour mat-vecs (complex products
// in the order of cfma / cfmac), reconstruction.
template <int MU, int T, bool ADJ>
__device__ __forceinline__ void hop_pair(cx2 acc[12], const cx2 psi[12], const cx<float> u[9], float2 sg) {
  cx2 h0[3], h1[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) proj2<MU, T>(psi[c], psi[3 + c], psi[6 + c], psi[9 + c], h0[c], h1[c]);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    cx2 g0, g1;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const cx<float> w = ADJ ? u[3 * b + a] : u[3 * a + b];
      const float2 wr = bc2(w.re);
      // U:   re += w.re h.re - w.im h.im,  im += w.re h.im + w.im h.re
      // U^H: re += w.re h.re + w.im h.im,  im += w.re h.im - w.im h.re
      const float2 wi_im = bc2(ADJ ? w.im : -w.im);  // factor of h.im in re
      const float2 wi_re = bc2(ADJ ? -w.im : w.im);  // factor of h.re in im
      if (b == 0) {
        g0.re = mul2(wr, h0[b].re);
        g1.re = mul2(wr, h1[b].re);
      } else {
        g0.re = fma2(wr, h0[b].re, g0.re);
        g1.re = fma2(wr, h1[b].re, g1.re);
      }
      g0.re = fma2(wi_im, h0[b].im, g0.re);
      g1.re = fma2(wi_im, h1[b].im, g1.re);
      if (b == 0) {
        g0.im = mul2(wr, h0[b].im);
        g1.im = mul2(wr, h1[b].im);
      } else {
        g0.im = fma2(wr, h0[b].im, g0.im);
        g1.im = fma2(wr, h1[b].im, g1.im);
      }
      g0.im = fma2(wi_re, h0[b].re, g0.im);
      g1.im = fma2(wi_re, h1[b].re, g1.im);
    }
    recon2<MU, T>(acc, a, g0, g1, sg);
  }
}

// The same hop for FP16 pairs: projection and colour product in half2
// arithmetic on the stored values (u: the nine FP16 link elements, re in the
// low and im in the high half), reconstruction in FP32 with sg the boundary
// sign times the two site scales.
template <int MU, int T, bool ADJ>
__device__ __forceinline__ void hop_pair_h(cx2 acc[12], const hx2 psi[12], const __half2 u[9], float2 sg) {
  hx2 h0[3], h1[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) proj2<MU, T>(psi[c], psi[3 + c], psi[6 + c], psi[9 + c], h0[c], h1[c]);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    hx2 q0, q1;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const __half2 w = ADJ ? u[3 * b + a] : u[3 * a + b];
      const __half2 wr = __low2half2(w), wi = __high2half2(w);
      // U:   re += w.re h.re - w.im h.im,  im += w.re h.im + w.im h.re
      // U^H: re += w.re h.re + w.im h.im,  im += w.re h.im - w.im h.re
      const __half2 wi_im = ADJ ? wi : __hneg2(wi);
      const __half2 wi_re = ADJ ? __hneg2(wi) : wi;
      if (b == 0) {
        q0.re = __hmul2(wr, h0[b].re);
        q1.re = __hmul2(wr, h1[b].re);
        q0.im = __hmul2(wr, h0[b].im);
        q1.im = __hmul2(wr, h1[b].im);
      } else {
        q0.re = __hfma2(wr, h0[b].re, q0.re);
        q1.re = __hfma2(wr, h1[b].re, q1.re);
        q0.im = __hfma2(wr, h0[b].im, q0.im);
        q1.im = __hfma2(wr, h1[b].im, q1.im);
      }
      q0.re = __hfma2(wi_im, h0[b].im, q0.re);
      q1.re = __hfma2(wi_im, h1[b].im, q1.re);
      q0.im = __hfma2(wi_re, h0[b].re, q0.im);
      q1.im = __hfma2(wi_re, h1[b].re, q1.im);
    }
    cx2 g0, g1;
    g0.re = __half22float2(q0.re);
    g0.im = __half22float2(q0.im);
    g1.re = __half22float2(q1.re);
    g1.im = __half22float2(q1.im);
    recon2<MU, T>(acc, a, g0, g1, sg);
  }
}

// One hop from the stored neighbour pair i of field f with link mu of site ls
// of Ubase: FP16 vectors take the half2 hop above, FP32 vectors widen the
// links to FP32 and use the packed FP32x2 hop.
template <int PG, int PV, int MU, int T, bool ADJ>
__device__ __forceinline__ void pair_hop_from(cx2 acc[12], const HalfField& f, int64_t gstride, int64_t i,
                                              const void* Ubase, int64_t ls, int64_t Vh, float sg) {
  if constexpr (PV == P16) {
    static_assert(PG == P16, "FP16 paired vectors come with FP16 links");
    __half2 u[9];
    load_link_h(Ubase, ls, Vh, MU, u);
    hx2 psi[12];
    const float2 ps = load_pair_h(f, gstride, i, psi);
    hop_pair_h<MU, T, ADJ>(acc, psi, u, mul2(bc2(sg), ps));
  } else {
    cx<float> u[9];
    load_link<PG, float>(Ubase, ls, Vh, MU, u);
    cx2 psi[12];
    load_pair<PV>(f, gstride, i, psi);
    hop_pair<MU, T, ADJ>(acc, psi, u, bc2(sg));
  }
}

// out (+)= M x for the two Hermitian 6x6 blocks of site s (storage as in
// block_apply_g), on a pair; the same operation order as block_apply_g.
template <int PG, bool ADD>
__device__ __forceinline__ void block_apply_pair(const void* M, int64_t s, int64_t Vh, const cx2 x[12], cx2 out[12],
                                                 bool streaming) {
  constexpr int PER = BlockGroups<PG>::PER;
  cx<float> grp[4];
#pragma unroll
  for (int E = 0; E < 36; ++E) {
    if (E % PER == 0) load_block_group<PG, float>(M, s, Vh, E / PER, grp, streaming);
    const cx<float> m = grp[E % PER];
    const int b = E / 18, k = E % 18;
    if (k < 3) {
      const int i0 = 6 * b + 2 * k, i1 = i0 + 1;
      const float2 d0 = bc2(m.re), d1 = bc2(m.im);
      if (ADD) {
        out[i0].re = fma2(d0, x[i0].re, out[i0].re);
        out[i0].im = fma2(d0, x[i0].im, out[i0].im);
        out[i1].re = fma2(d1, x[i1].re, out[i1].re);
        out[i1].im = fma2(d1, x[i1].im, out[i1].im);
      } else {
        out[i0].re = mul2(d0, x[i0].re);
        out[i0].im = mul2(d0, x[i0].im);
        out[i1].re = mul2(d1, x[i1].re);
        out[i1].im = mul2(d1, x[i1].im);
      }
    } else {
      int i, j;
      tri_ij(k - 3, i, j);
      i += 6 * b;
      j += 6 * b;
      const float2 mr = bc2(m.re), mi = bc2(m.im), nmi = bc2(-m.im);
      // out_i += m x_j
      out[i].re = fma2(mr, x[j].re, out[i].re);
      out[i].re = fma2(nmi, x[j].im, out[i].re);
      out[i].im = fma2(mr, x[j].im, out[i].im);
      out[i].im = fma2(mi, x[j].re, out[i].im);
      // out_j += conj(m) x_i
      out[j].re = fma2(mr, x[i].re, out[j].re);
      out[j].re = fma2(mi, x[i].im, out[j].re);
      out[j].im = fma2(mr, x[i].im, out[j].im);
      out[j].im = fma2(nmi, x[i].re, out[j].im);
    }
  }
}

// One thread: output site s (parity p) and RHS pair j.
//   EPI_D:    out = M y + beta acc  (M y first, beta folded into the hop signs)
//   EPI_AINV: out = M (beta acc)
template <int PG, int PV, bool DAG, int EPI>
__device__ __forceinline__ void hop_thread_pair(const HopArgs& a, int64_t tid) {
  const int NP = a.nrhs >> 1;
  int p, s, j;
  SiteCoord sc;
  if (a.npar == 2) {
    const int lex = fdiv((int)tid, a.fblk);
    j = (int)tid - lex * NP;
    sc = traversal_coords(a.g, lex);
    p = (sc.c[0] + sc.c[1] + sc.c[2] + sc.c[3]) & 1;
    s = sc.lex >> 1;
  } else {
    p = a.p0;
    s = fdiv((int)tid, a.fblk);
    j = (int)tid - s * NP;
    sc = site_coords(a.g, s, p);
  }
  const int q = p ^ 1;
  const int64_t Vh = a.g.Vh;
  constexpr int TF = DAG ? +1 : -1;
  constexpr int TB = -TF;
  const float beta = (float)a.beta;
  const int64_t i = (int64_t)s * NP + j;

  cx2 acc[12];
  if constexpr (EPI == EPI_D) {
    cx2 y[12];
    const float2 ys = load_pair<PV>(a.y[p], a.gstride, i, y);
    if constexpr (PV == P16) {
#pragma unroll
      for (int c = 0; c < 12; ++c) y[c].re = mul2(ys, y[c].re), y[c].im = mul2(ys, y[c].im);
    }
    block_apply_pair<PG, false>(a.M[p], s, Vh, y, acc, true);
  } else {
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[c].re = acc[c].im = make_float2(0.f, 0.f);
  }
  const float hop_scale = EPI == EPI_D ? beta : 1.f;

#define DD_PAIR_HOP(MU, FWD)                                                                          \
  {                                                                                                   \
    const int nl = FWD ? nb_fwd(a.g, sc, MU) : nb_bwd(a.g, sc, MU);                                   \
    float sg = hop_scale;                                                                             \
    if (MU == 0 && sc.c[0] == (FWD ? a.g.n[0] - 1 : 0)) sg = sg * a.g.t_bc;                           \
    pair_hop_from<PG, PV, MU, FWD ? TF : TB, !FWD>(acc, a.in[q], a.gstride, (int64_t)(nl >> 1) * NP + j, \
                                                   FWD ? a.U[p] : a.U[q],                             \
                                                   FWD ? (int64_t)s : (int64_t)(nl >> 1), Vh, sg);    \
  }
  DD_PAIR_HOP(0, true)
  DD_PAIR_HOP(0, false)
  DD_PAIR_HOP(1, true)
  DD_PAIR_HOP(1, false)
  DD_PAIR_HOP(2, true)
  DD_PAIR_HOP(2, false)
  DD_PAIR_HOP(3, true)
  DD_PAIR_HOP(3, false)
#undef DD_PAIR_HOP

  if constexpr (EPI == EPI_AINV) {
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[c].re = mul2(bc2(beta), acc[c].re), acc[c].im = mul2(bc2(beta), acc[c].im);
    cx2 out[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) out[c].re = out[c].im = make_float2(0.f, 0.f);
    block_apply_pair<PG, true>(a.M[p], s, Vh, acc, out, false);
    store_pair<PV>(a.out[p], a.gstride, i, out);
  } else {
    store_pair<PV>(a.out[p], a.gstride, i, acc);
  }
}

// 128 threads with at least 4 resident CTAs (at most 128 registers): the
// fastest of 3, 4 and 5 resident CTAs on the 32^4 lattice with 12 RHS and
// the 48^3 x 96 lattice with 2 RHS (5 spills).
template <int PG, int PV, bool DAG, int EPI>
__global__ void __launch_bounds__(128, 4) k_hop_pair(const HopArgs a) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= launch_sites(a.g, a.npar) * (a.nrhs >> 1)) return;
  hop_thread_pair<PG, PV, DAG, EPI>(a, tid);
}

// Host launcher: EPI_D or EPI_AINV on paired fields (nrhs even, FP32 or
// FP16 vectors); `a.gstride` is set here to Vh * nrhs / 2.
template <int PG, int PV>
cudaError_t launch_hop_pair(const HopArgs& args, bool dagger, int epi, cudaStream_t st) {
  if (args.nrhs < 2 || args.nrhs % 2 != 0 || (epi != EPI_D && epi != EPI_AINV)) return cudaErrorInvalidValue;
  HopArgs a = args;
  prepare_divs(a.g);
  const int NP = a.nrhs / 2;
  a.fblk = make_fastdiv((uint32_t)NP);
  a.gstride = (int64_t)a.g.Vh * NP;
  const int64_t n = launch_sites(a.g, a.npar) * NP;
  if (n == 0) return cudaSuccess;
  if (n >= (int64_t)1 << 31) return cudaErrorInvalidValue;  // thread indices are 32-bit
  const unsigned blocks = (unsigned)((n + 127) / 128);
  const int key = (epi == EPI_D ? 0 : 2) + (dagger ? 1 : 0);
  switch (key) {
    case 0: k_hop_pair<PG, PV, false, EPI_D><<<blocks, 128, 0, st>>>(a); break;
    case 1: k_hop_pair<PG, PV, true, EPI_D><<<blocks, 128, 0, st>>>(a); break;
    case 2: k_hop_pair<PG, PV, false, EPI_AINV><<<blocks, 128, 0, st>>>(a); break;
    default: k_hop_pair<PG, PV, true, EPI_AINV><<<blocks, 128, 0, st>>>(a); break;
  }
  return cudaGetLastError();
}

#define DD_INSTANTIATE_HOP_PAIR(PG, PV) \
  template cudaError_t launch_hop_pair<PG, PV>(const HopArgs&, bool, int, cudaStream_t);

}  // namespace dd
