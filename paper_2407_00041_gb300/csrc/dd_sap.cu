// Schwarz alternating procedure (SAP) on the GPU: the block smoother that
// the thesis names for DDalphaAMG (Section 1.3), used as a flexible
// preconditioner M_j of Algorithm 2.
//
// Method (red-black multiplicative Schwarz, non-overlapping blocks):
//   * the lattice is cut into blocks of b_T x b_Z x b_Y x b_X sites aligned
//     with the origin, every extent holding an even number of blocks; the
//     colour of a block is the parity of the sum of its block coordinates, so
//     two blocks of one colour never share a face;
//   * D_B is D restricted to block B with every hop that leaves the block
//     dropped (Dirichlet boundary); since every extent holds at least two
//     blocks, no hop inside a block crosses the time boundary;
//   * one cycle on D z = v with r = v - D z: for the blocks of colour 0, then
//     of colour 1, e_B = k minimal-residual steps on D_B e = r_B from e = 0
//     (q = D_B rho, alpha = q^H rho / q^H q, e += alpha rho, rho -= alpha q),
//     z += e on every block of the colour, then r = v - D z;
//   * M^{-1} v is z after n cycles from z = 0.
//
// GPU form: one CTA per (block of the colour, right-hand side), one thread per
// site of the block.  The block residual rho and the correction e live in
// shared memory ([12 components][block sites] each; rho also in registers
// for the own site); each MR step runs the block stencil from it (the fused
// hop of dd_hop.cuh with the factor -1/2 in its sign, hops leaving the block
// skipped, the self coupling first), reduces q^H rho and q^H q over the CTA
// (warp shuffles, then the warps in a fixed order, in the working precision),
// and updates e and rho.  The residual between the colours is the full-lattice
// r = v - D z stencil (EPI_RESID).  FP64, FP32, and FP16 links / blocks with
// FP32 vectors.
#include <cstdio>

#include "dd_hop.cuh"
#include "dd_internal.h"
#include "dd_ops.h"
#include "dd_sap.h"

namespace dd {

namespace {

struct SapArgs {
  Geom g;            // lattice geometry (n, strides, Vh)
  int b[4];          // block extents (T, Z, Y, X)
  int nb[4];         // blocks per direction
  int bstride[4];    // local lexicographic strides inside a block
  int colour;        // colour of the blocks of this launch
  int nrhs;
  int mr_steps;
  int64_t gstride;   // component-group stride of a half field (Vh * nrhs)
  HalfField r[2];    // residual r (read)
  HalfField z[2];    // iterate z (z += e)
  const void* U[2];  // links by parity
  const void* M[2];  // self-coupling blocks by parity
};

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// One MR block solve per CTA.  blockIdx.x: block of this colour; blockIdx.y:
// right-hand side; thread t < bsites: site t of the block (local
// lexicographic order, X fastest); the threads of a last partial warp only
// take part in the reductions.  Shared memory: rho and e as [12][bsites]
// complex, then the reduction slots.
template <int PG, int PV>
__global__ void __launch_bounds__(kSapMaxSites, PG == P64 ? 1 : 2) k_sap_block(const SapArgs a) {
  using R = typename Store<PG>::real;
  extern __shared__ __align__(16) unsigned char sap_smem[];
  const int bsites = a.b[0] * a.b[1] * a.b[2] * a.b[3];
  cx<R>* rho_s = reinterpret_cast<cx<R>*>(sap_smem);  // [12][bsites]
  cx<R>* e_s = rho_s + (size_t)12 * bsites;           // [12][bsites]
  R* red = reinterpret_cast<R*>(e_s + (size_t)12 * bsites);  // [warps][3], then alpha at [96], [97]
  const int t = threadIdx.x;
  const bool act = t < bsites;
  const int tt = act ? t : 0;  // inactive threads decode site 0 and touch nothing
  const int r = blockIdx.y;
  // block coordinates of the k-th block of this colour: every row of blocks
  // along X holds nb_X / 2 blocks of each colour (nb_X is even)
  int k = blockIdx.x;
  const int hx = a.nb[3] >> 1;
  const int bxh = k % hx;
  k /= hx;
  const int BY = k % a.nb[2];
  k /= a.nb[2];
  const int BZ = k % a.nb[1];
  const int BT = k / a.nb[1];
  const int B[4] = {BT, BZ, BY, 2 * bxh + ((a.colour + BT + BZ + BY) & 1)};
  int lc[4];
  {
    int u = tt;
    lc[3] = u % a.b[3];
    u /= a.b[3];
    lc[2] = u % a.b[2];
    u /= a.b[2];
    lc[1] = u % a.b[1];
    lc[0] = u / a.b[1];
  }
  int c[4], lex = 0;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    c[mu] = B[mu] * a.b[mu] + lc[mu];
    lex += c[mu] * a.g.stride[mu];
  }
  const int p = (c[0] + c[1] + c[2] + c[3]) & 1;
  const int q = p ^ 1;
  const int64_t s = lex >> 1;
  const int64_t Vh = a.g.Vh;
  const int64_t i = s * a.nrhs + r;

  cx<R> rho[12];
  if (act) {
    load_spinor<PV, R>(a.r[p], a.gstride, i, rho);
#pragma unroll
    for (int cc = 0; cc < 12; ++cc) {
      rho_s[cc * bsites + t] = rho[cc];
      e_s[cc * bsites + t] = zero<R>();
    }
  } else {
#pragma unroll
    for (int cc = 0; cc < 12; ++cc) rho[cc] = zero<R>();
  }
  __syncthreads();
  const int lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
  for (int step = 0; step < a.mr_steps; ++step) {
    // q = D_B rho = A rho - 1/2 (hops that stay inside the block)
    cx<R> qv[12];
    if (act) {
      block_apply_g<PG, false, R>(a.M[p], s, Vh, rho, qv, false);
#define DD_SAP_HOP(MU)                                                                           \
      if (lc[MU] < a.b[MU] - 1) {                                                                \
        cx<R> nbv[12], u[9];                                                                     \
        const int tn = t + a.bstride[MU];                                                        \
        _Pragma("unroll") for (int cc = 0; cc < 12; ++cc) nbv[cc] = rho_s[cc * bsites + tn];     \
        load_link<PG, R>(a.U[p], s, Vh, MU, u);                                                  \
        hop_regs<MU, -1, false, R>(qv, nbv, u, (R)-0.5);                                         \
      }                                                                                          \
      if (lc[MU] > 0) {                                                                          \
        cx<R> nbv[12], u[9];                                                                     \
        const int tn = t - a.bstride[MU];                                                        \
        _Pragma("unroll") for (int cc = 0; cc < 12; ++cc) nbv[cc] = rho_s[cc * bsites + tn];     \
        load_link<PG, R>(a.U[q], (int64_t)((lex - a.g.stride[MU]) >> 1), Vh, MU, u);             \
        hop_regs<MU, +1, true, R>(qv, nbv, u, (R)-0.5);                                          \
      }
      DD_SAP_HOP(0)
      DD_SAP_HOP(1)
      DD_SAP_HOP(2)
      DD_SAP_HOP(3)
#undef DD_SAP_HOP
    } else {
#pragma unroll
      for (int cc = 0; cc < 12; ++cc) qv[cc] = zero<R>();
    }
    // q^H rho and q^H q over the block
    R qr_re = 0, qr_im = 0, qq = 0;
#pragma unroll
    for (int cc = 0; cc < 12; ++cc) {
      qr_re = ffma(qv[cc].re, rho[cc].re, qr_re);
      qr_re = ffma(qv[cc].im, rho[cc].im, qr_re);
      qr_im = ffma(qv[cc].re, rho[cc].im, qr_im);
      qr_im = ffma(-qv[cc].im, rho[cc].re, qr_im);
      qq = ffma(qv[cc].re, qv[cc].re, qq);
      qq = ffma(qv[cc].im, qv[cc].im, qq);
    }
    qr_re = warp_sum(qr_re);
    qr_im = warp_sum(qr_im);
    qq = warp_sum(qq);
    if (lane == 0) {
      red[3 * warp] = qr_re;
      red[3 * warp + 1] = qr_im;
      red[3 * warp + 2] = qq;
    }
    __syncthreads();  // also: every read of rho_s for this step is done
    if (t == 0) {
      R sr = 0, si = 0, sq = 0;
      for (int w = 0; w < nw; ++w) sr += red[3 * w], si += red[3 * w + 1], sq += red[3 * w + 2];
      const R inv = sq > (R)0 ? (R)1 / sq : (R)0;
      red[96] = sr * inv;
      red[97] = si * inv;
    }
    __syncthreads();
    const cx<R> alpha = mk(red[96], red[97]);
    const cx<R> nalpha = mk(-alpha.re, -alpha.im);
    if (act) {
#pragma unroll
      for (int cc = 0; cc < 12; ++cc) {
        e_s[cc * bsites + t] = cfma(alpha, rho[cc], e_s[cc * bsites + t]);
        rho[cc] = cfma(nalpha, qv[cc], rho[cc]);
        rho_s[cc * bsites + t] = rho[cc];
      }
    }
    __syncthreads();
  }
  if (!act) return;
  // z += e on the block
  cx<R> zv[12];
  load_spinor<PV, R>(a.z[p], a.gstride, i, zv);
#pragma unroll
  for (int cc = 0; cc < 12; ++cc) zv[cc] = zv[cc] + e_s[cc * bsites + t];
  store_spinor<PV, R>(a.z[p], a.gstride, i, zv);
}

template <int PG, int PV>
size_t sap_smem_bytes(int bsites) {
  using R = typename Store<PG>::real;
  return (size_t)24 * bsites * sizeof(cx<R>) + 100 * sizeof(R);
}

template <int PG, int PV>
cudaError_t launch_sap_block(const SapArgs& a, cudaStream_t st) {
  const int bsites = a.b[0] * a.b[1] * a.b[2] * a.b[3];
  const size_t smem = sap_smem_bytes<PG, PV>(bsites);
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_sap_block<PG, PV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sap_smem_bytes<P64, P64>(kSapMaxSites));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int nblocks = a.nb[0] * a.nb[1] * a.nb[2] * a.nb[3] / 2;
  const unsigned threads = (unsigned)((bsites + 31) / 32 * 32);
  k_sap_block<PG, PV><<<dim3((unsigned)nblocks, (unsigned)a.nrhs), threads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

int sap_check_blocks(const dd_lattice* lat, const int block[4], int pv) {
  int bs = 1;
  for (int mu = 0; mu < 4; ++mu) {
    const int n = lat->dims[mu], b = block[mu];
    if (b < 1 || n % b != 0 || (n / b) % 2 != 0)
      return fail(DD_ERR_ARG, "SAP: every extent must hold an even number of blocks");
    bs *= b;
  }
  if (bs > kSapMaxSites) return fail(DD_ERR_ARG, "SAP: a block holds at most 256 sites");
  return DD_OK;
}

int sap_apply(const dd_clover* op, int pg, int pv, const int block[4], int cycles, int mr_steps, const Field& v,
              const Field& z, const Field& r, cudaStream_t st) {
  const dd_lattice* lat = op->lat;
  DD_TRY(sap_check_blocks(lat, block, pv));
  if (cycles < 1 || mr_steps < 1) return fail(DD_ERR_ARG, "SAP: cycles and MR steps must be >= 1");
  if (!((pg == P64 && pv == P64) || (pg == P32 && pv == P32) || (pg == P16 && pv == P32)))
    return fail(DD_ERR_UNSUPPORTED, "SAP: FP64, FP32, or FP16 links / blocks with FP32 vectors");
  const int pi = prec_index(pg);
  if (!op->gauge->links[pi].ptr || !op->clov[pi].ptr)
    return fail(DD_ERR_UNSUPPORTED, "precision not created in the gauge/operator handles");
  const int N = v.nrhs;
  SapArgs a;
  a.g = lat->geom();
  a.nrhs = N;
  a.mr_steps = mr_steps;
  a.gstride = lat->Vh * N;
  int bst = 1;
  for (int mu = 3; mu >= 0; --mu) {
    a.b[mu] = block[mu];
    a.nb[mu] = lat->dims[mu] / block[mu];
    a.bstride[mu] = bst;
    bst *= block[mu];
  }
  for (int p = 0; p < 2; ++p) {
    a.r[p] = r.h[p];
    a.z[p] = z.h[p];
    a.U[p] = op->gauge->U(pi, p);
    a.M[p] = op->M(pi, p);
  }
  // z = 0, r = v
  const size_t fb = field_bytes(lat, pv, 0, N);
  DD_CUDA(cudaMemsetAsync(z.h[0].base, 0, fb, st));
  DD_CUDA(cudaMemcpyAsync(r.h[0].base, v.h[0].base, fb, cudaMemcpyDeviceToDevice, st));
  for (int cyc = 0; cyc < cycles; ++cyc) {
    for (int colour = 0; colour < 2; ++colour) {
      a.colour = colour;
      cudaError_t e;
      if (pg == P64)
        e = launch_sap_block<P64, P64>(a, st);
      else if (pg == P32)
        e = launch_sap_block<P32, P32>(a, st);
      else
        e = launch_sap_block<P16, P32>(a, st);
      if (e != cudaSuccess) return cuda_fail(e, "SAP block solve launch");
      if (cyc + 1 < cycles || colour == 0) DD_TRY(op_residual(op, pg, pv, v, z, r, st));  // r = v - D z
    }
  }
  return DD_OK;
}

}  // namespace dd
