// FGMRES (Algorithm 2 of the thesis) inside an FP64 iterative-refinement
// loop, for several right-hand sides at once.
//
// Outer loop (FP64): r = b - D x with the full FP64 operator; stop when
// ||r_k|| < tol ||b_k|| for every right-hand side k.  Otherwise solve
// D e = r approximately (inner solve) and update x += e in FP64.
//
// Inner solve: FGMRES(m) with M_j = I (so z_j = v_j) on the even-odd Schur
// operator Dhat (odd sites) or on D, in the inner precision.  Each Arnoldi
// step applies the operator once (Algorithm 2) and orthogonalises with
// classical Gram-Schmidt (one pass, or two with gs_passes = 2) in place of the
// algorithm's modified Gram-Schmidt: it reads every basis vector once per
// pass; inner products accumulated in FP64.  The small least-squares problem is
// solved on the host with complex Givens rotations, whose
// residual estimate is checked after every step; a cycle also ends when
// |h_{j+1,j}| falls below tol / 10 of ||f|| (the breakdown rule after
// Algorithm 1).  Right-hand sides that have converged are masked out (their
// new basis vectors are scaled by zero).
//
// Preconditioners M_j (Algorithm 2):
//   none    z_j = v_j
//   normal  the fixed right preconditioner M^{-1} = A^H: A M^{-1} = A A^H is
//           Hermitian positive definite, so restarted FGMRES cannot stagnate
//   cgnr    the flexible preconditioner z_j = k steps of the conjugate-gradient
//           method on the normal equations A^H A z = A^H v_j (from z = 0), run
//           on the device with step sizes kept in device memory; Z_m is stored
//           and x += Z_m y.
//   cgnr16  the same CG with its vectors r, A^H r, p and A p stored in FP16
//           (per-site scales) and read by the stencil with FP16 vectors and
//           the inner precision's links and blocks (FP16 for inner_prec F16,
//           FP32 for F32); z accumulates in FP32
//   amg     the flexible two-level preconditioner of dd_amg.cu (coarse-grid
//           correction and SAP post-smoothing), for the even-odd system
//           applied to (0, v_j) like sap;
//   sap     the flexible preconditioner z_j = n red-black Schwarz cycles on
//           D z = v_j (dd_sap.cu); for the even-odd system (A = Dhat, whose
//           inverse is the odd-odd block of D^{-1}) z_j is the odd half of the
//           cycles applied to the full field (0 on even sites, v_j on odd).
#include <algorithm>
#include <new>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <functional>
#include <vector>

#include "dd_blas.h"
#include "dd_internal.h"
#include "dd_ops.h"
#include "dd_sap.h"
#include "dd_krylov.h"
#include "dd_amg.h"

namespace dd {

namespace {

using cd = std::complex<double>;

struct Pinned {
  void* p = nullptr;
  ~Pinned() {
    if (p) cudaFreeHost(p);
  }
  int alloc(size_t n) {
    if (cudaMallocHost(&p, n) != cudaSuccess) {
      p = nullptr;
      (void)cudaGetLastError();
      return fail(DD_ERR_OOM, "pinned host allocation failed");
    }
    return DD_OK;
  }
};

struct Inner {
  const dd_clover* op;
  int pg, pv;
  bool eo;
  int N, m;
  int64_t L;     // 16-byte groups per vector
  size_t vbytes;
  int mode = 0;         // DD_PRECOND_NONE / _NORMAL / _CGNR / _SAP
  int cg_iters = 32;    // CG steps per application of the cgnr preconditioner
  bool normal = false;  // mode == DD_PRECOND_NORMAL
  int verbose = 0;
  int gs_passes = 1;    // classical Gram-Schmidt passes per Arnoldi step
  DevBuf basis, w, rvec, tmp, red, partials, coef, zt, ut, zbasis, cr, cz, cp, cgs;
  // cgnr16: the CG vectors in FP16 (r, A^H r, p, A p) and Dhat's intermediate
  DevBuf cr16, cz16, cp16, cw16, tmp16;
  size_t vbytes16 = 0;
  // sap: block extents, cycles and MR steps per block solve; full fields v, z, r
  int sap_block[4] = {4, 4, 4, 4};
  int sap_cycles = 1, sap_mr = 4;
  DevBuf sv, sz, sr;
  dd_amg* amg = nullptr;  // DD_PRECOND_AMG
  // CG norms formed by the second stencil launch of Dhat (one RHS; FP32
  // vectors, or the FP16 CG vectors of cgnr16; DD_FUSED_NORM=0 turns it
  // off): per-block partial sums
  bool fuse_norm = false;
  DevBuf npart;
  int64_t npart_len = 0;
  Pinned hred, hcoef;
  // counters
  int applies = 0, steps = 0, cycles = 0;
  // a custom operator (the AMG coarse system): vectors of L double2 groups
  // (N right-hand sides innermost), FP64, no preconditioner
  std::function<int(const void*, void*, cudaStream_t)> custom;

  int init_custom(int64_t L_, int N_, int m_) {
    mode = DD_PRECOND_NONE;
    normal = false;
    op = nullptr;
    pg = pv = P64;
    eo = false;
    N = N_;
    m = m_;
    L = L_;
    vbytes = (size_t)L_ * 16;
    DD_TRY(basis.ensure(vbytes * (m + 1)));
    DD_TRY(w.ensure(vbytes));
    DD_TRY(rvec.ensure(vbytes));
    const size_t nred = (size_t)(2 * (m + 1) + 1) * N;
    DD_TRY(red.ensure(nred * sizeof(double2)));
    DD_TRY(partials.ensure((size_t)blas_partials_len(N) * sizeof(double2)));
    DD_TRY(coef.ensure((size_t)(m + 1) * N * sizeof(double2)));
    if (!hred.p) DD_TRY(hred.alloc(nred * sizeof(double2)));
    if (!hcoef.p) DD_TRY(hcoef.alloc((size_t)(m + 1) * N * sizeof(double2)));
    return DD_OK;
  }

  int init(const dd_clover* op_, int pg_, int pv_, bool eo_, int N_, int m_, int mode_) {
    mode = mode_;
    normal = mode == DD_PRECOND_NORMAL;
    fuse_norm = false;
    op = op_;
    pg = pg_;
    pv = pv_;
    eo = eo_;
    N = N_;
    m = m_;
    const dd_lattice* lat = op->lat;
    vbytes = field_bytes(lat, pv, eo ? 1 : 0, N);
    L = (int64_t)(vbytes / 16);
    DD_TRY(basis.ensure(vbytes * (m + 1)));
    DD_TRY(w.ensure(vbytes));
    DD_TRY(rvec.ensure(vbytes));
    if (normal) {
      DD_TRY(zt.ensure(vbytes));
      DD_TRY(ut.ensure(vbytes));
    }
    if (mode == DD_PRECOND_SAP || mode == DD_PRECOND_AMG) {
      DD_TRY(zbasis.ensure(vbytes * m));
      const size_t fb = field_bytes(lat, pv, 0, N);
      DD_TRY(sv.ensure(fb));
      DD_TRY(sz.ensure(fb));
      DD_TRY(sr.ensure(fb));
    }
    if (mode == DD_PRECOND_CGNR) {
      DD_TRY(zbasis.ensure(vbytes * m));
      DD_TRY(cr.ensure(vbytes));
      DD_TRY(cz.ensure(vbytes));
      DD_TRY(cp.ensure(vbytes));
      DD_TRY(cgs.ensure((size_t)3 * N * sizeof(double2)));
      const char* fe = getenv("DD_FUSED_NORM");
      fuse_norm = eo && dhat_norm_fused(pg, pv, N) && !(fe && atoi(fe) == 0);
      if (fuse_norm) {
        const int64_t nb = hop_norm_blocks(lat->Vh);
        npart_len = nb + blas_reduce_scratch((int)std::min<int64_t>(nb, INT32_MAX), 1);
        DD_TRY(npart.ensure((size_t)npart_len * sizeof(double2)));
      }
    }
    if (mode == DD_PRECOND_CGNR16) {
      DD_TRY(zbasis.ensure(vbytes * m));
      DD_TRY(cgs.ensure((size_t)3 * N * sizeof(double2)));
      vbytes16 = field_bytes(lat, P16, eo ? 1 : 0, N);
      DD_TRY(cr16.ensure(vbytes16));
      DD_TRY(cz16.ensure(vbytes16));
      DD_TRY(cp16.ensure(vbytes16));
      DD_TRY(cw16.ensure(vbytes16));
      if (eo) DD_TRY(tmp16.ensure(field_bytes(lat, P16, 2, N)));
      const char* fe = getenv("DD_FUSED_NORM");
      fuse_norm = eo && dhat_norm_fused(pg, P16, N) && !(fe && atoi(fe) == 0);
      if (fuse_norm) {
        const int64_t nb = hop_norm_blocks(lat->Vh);
        npart_len = nb + blas_reduce_scratch((int)std::min<int64_t>(nb, INT32_MAX), 1);
        DD_TRY(npart.ensure((size_t)npart_len * sizeof(double2)));
      }
    }
    if (eo) DD_TRY(tmp.ensure(field_bytes(lat, pv, 2, N)));
    const size_t nred = (size_t)(2 * (m + 1) + 1) * N;
    DD_TRY(red.ensure(nred * sizeof(double2)));
    DD_TRY(partials.ensure((size_t)blas_partials_len(N) * sizeof(double2)));
    DD_TRY(coef.ensure((size_t)(m + 1) * N * sizeof(double2)));
    if (!hred.p) DD_TRY(hred.alloc(nred * sizeof(double2)));
    if (!hcoef.p) DD_TRY(hcoef.alloc((size_t)(m + 1) * N * sizeof(double2)));
    return DD_OK;
  }

  void set_sap(const dd_solve_params* prm) {
    for (int mu = 0; mu < 4; ++mu) sap_block[mu] = prm->sap_block[mu];
    sap_cycles = prm->sap_cycles;
    sap_mr = prm->sap_mr_steps;
    amg = prm->amg;
  }

  void* V(int j) { return reinterpret_cast<char*>(basis.ptr) + vbytes * j; }
  void* Zb(int j) { return reinterpret_cast<char*>(zbasis.ptr) + vbytes * j; }
  Field fv(void* p) { return field_view(op->lat, pv, eo ? 1 : 0, p, N); }

  // the operator A of the inner system (Dhat or D)
  int apply_op(const void* in, void* out, bool dagger, cudaStream_t st) {
    ++applies;
    if (custom) return custom(in, out, st);
    void* i = const_cast<void*>(in);
    if (eo) return op_Dhat(op, pg, pv, dagger, fv(i), fv(out), field_view(op->lat, pv, 2, tmp.ptr, N), st);
    return op_D(op, pg, pv, dagger, fv(i), fv(out), st);
  }
  // out = A in and nrm[0] = (|out|^2, 0): fused into the stencil where
  // supported, else a separate reduction
  int apply_op_norm(const void* in, void* out, bool dagger, double2* nrm, cudaStream_t st) {
    if (!fuse_norm) {
      DD_TRY(apply_op(in, out, dagger, st));
      VecList one;
      one.p[0] = out;
      return dots(one, 1, out, nrm, 0, st);
    }
    ++applies;
    void* i = const_cast<void*>(in);
    return op_Dhat_norm(op, pg, pv, dagger, fv(i), fv(out), field_view(op->lat, pv, 2, tmp.ptr, N), nrm,
                        (double2*)npart.ptr, npart_len, st);
  }
  // w = A M^{-1} v (Algorithm 2)
  int apply(const void* v, void* out, cudaStream_t st) {
    if (!normal) return apply_op(v, out, false, st);
    DD_TRY(apply_op(v, zt.ptr, true, st));
    return apply_op(zt.ptr, out, false, st);
  }

  // z = SAP cycles on D z = v (full lattice), or for the even-odd system the
  // odd half of the cycles applied to (0, v)
  int sap(const void* v, void* z, cudaStream_t st) {
    const dd_lattice* lat = op->lat;
    Field V = field_view(lat, pv, 0, sv.ptr, N), Z = field_view(lat, pv, 0, sz.ptr, N),
          R = field_view(lat, pv, 0, sr.ptr, N);
    if (!eo) {
      Field Vin = field_view(lat, pv, 0, const_cast<void*>(v), N), Zout = field_view(lat, pv, 0, z, N);
      return sap_apply(op, pg, pv, sap_block, sap_cycles, sap_mr, Vin, Zout, R, st);
    }
    const size_t hb = field_bytes(lat, pv, 1, N);
    DD_CUDA(cudaMemsetAsync(V.h[0].base, 0, hb, st));
    DD_CUDA(cudaMemcpyAsync(V.h[1].base, v, hb, cudaMemcpyDeviceToDevice, st));
    DD_TRY(sap_apply(op, pg, pv, sap_block, sap_cycles, sap_mr, V, Z, R, st));
    DD_CUDA(cudaMemcpyAsync(z, Z.h[1].base, hb, cudaMemcpyDeviceToDevice, st));
    return DD_OK;
  }

  // z = M^{-1} v of the AMG handle (full lattice), or for the even-odd
  // system the odd half of M^{-1} (0, v)
  int amgp(const void* v, void* z, cudaStream_t st) {
    const dd_lattice* lat = op->lat;
    if (!eo) {
      Field Vin = field_view(lat, pv, 0, const_cast<void*>(v), N), Zout = field_view(lat, pv, 0, z, N);
      return amg_apply(amg, Vin, Zout, st);
    }
    Field V = field_view(lat, pv, 0, sv.ptr, N), Z = field_view(lat, pv, 0, sz.ptr, N);
    const size_t hb = field_bytes(lat, pv, 1, N);
    DD_CUDA(cudaMemsetAsync(V.h[0].base, 0, hb, st));
    DD_CUDA(cudaMemcpyAsync(V.h[1].base, v, hb, cudaMemcpyDeviceToDevice, st));
    DD_TRY(amg_apply(amg, V, Z, st));
    DD_CUDA(cudaMemcpyAsync(z, Z.h[1].base, hb, cudaMemcpyDeviceToDevice, st));
    return DD_OK;
  }

  // the cgnr16 preconditioner: the same CG with r, A^H r, p and A p stored in
  // FP16 (dd_cg16.cu), z accumulated in FP32
  Field fv16(void* p) { return field_view(op->lat, P16, eo ? 1 : 0, p, N); }
  int apply16(void* in, void* out, bool dagger, cudaStream_t st) {
    ++applies;
    if (eo) return op_Dhat(op, pg, P16, dagger, fv16(in), fv16(out), field_view(op->lat, P16, 2, tmp16.ptr, N), st);
    return op_D(op, pg, P16, dagger, fv16(in), fv16(out), st);
  }
  int norm16(void* x, double2* out, cudaStream_t st) {
    return cg16_norm(fv16(x), op->lat->Vh, eo ? 1 : 2, (double2*)partials.ptr, out, st);
  }
  // out = A in and nrm[0] = (|out|^2, 0): the norm formed by the stencil
  // launch (of the FP32 result before its rounding to FP16) where supported,
  // else a pass over the stored FP16 vector
  int apply16_norm(void* in, void* out, bool dagger, double2* nrm, cudaStream_t st) {
    if (!fuse_norm) {
      DD_TRY(apply16(in, out, dagger, st));
      return norm16(out, nrm, st);
    }
    ++applies;
    return op_Dhat_norm(op, pg, P16, dagger, fv16(in), fv16(out), field_view(op->lat, P16, 2, tmp16.ptr, N), nrm,
                        (double2*)npart.ptr, npart_len, st);
  }
  int cgnr16(const void* v, void* z, cudaStream_t st) {
    double2* g0 = reinterpret_cast<double2*>(cgs.ptr);
    double2* g1 = g0 + N;
    double2* nw = g0 + 2 * N;
    double2* g[2] = {g0, g1};
    const int npar = eo ? 1 : 2;
    const int64_t Vh = op->lat->Vh;
    DD_CUDA(cudaMemsetAsync(z, 0, vbytes, st));
    DD_TRY(cg16_convert(fv(const_cast<void*>(v)), fv16(cr16.ptr), Vh, npar, st));
    DD_TRY(apply16_norm(cr16.ptr, cz16.ptr, true, g[0], st));  // A^H r
    DD_CUDA(cudaMemcpyAsync(cp16.ptr, cz16.ptr, vbytes16, cudaMemcpyDeviceToDevice, st));
    const Field Z = fv(z), P = fv16(cp16.ptr), W = fv16(cw16.ptr), Rr = fv16(cr16.ptr), Zz = fv16(cz16.ptr);
    for (int i = 0; i < cg_iters; ++i) {
      DD_TRY(apply16_norm(cp16.ptr, cw16.ptr, false, nw, st));  // w = A p
      if (i + 1 == cg_iters) {
        DD_TRY(cg16_xp(Z, P, nullptr, Vh, npar, g[i & 1], nw, nullptr, st));
        break;
      }
      DD_TRY(cg16_r(Rr, W, Vh, npar, g[i & 1], nw, st));
      DD_TRY(apply16_norm(cr16.ptr, cz16.ptr, true, g[(i + 1) & 1], st));  // z' = A^H r
      DD_TRY(cg16_xp(Z, P, &Zz, Vh, npar, g[i & 1], nw, g[(i + 1) & 1], st));
    }
    return DD_OK;
  }

  // z = k steps of CG on A^H A z = A^H v from z = 0 (the cgnr preconditioner)
  int cgnr(const void* v, void* z, cudaStream_t st) {
    double2* g0 = reinterpret_cast<double2*>(cgs.ptr);
    double2* g1 = g0 + N;
    double2* nw = g0 + 2 * N;
    double2* g[2] = {g0, g1};
    DD_CUDA(cudaMemsetAsync(z, 0, vbytes, st));
    DD_CUDA(cudaMemcpyAsync(cr.ptr, v, vbytes, cudaMemcpyDeviceToDevice, st));
    DD_TRY(apply_op_norm(cr.ptr, cz.ptr, true, g[0], st));  // A^H r and its norm
    DD_CUDA(cudaMemcpyAsync(cp.ptr, cz.ptr, vbytes, cudaMemcpyDeviceToDevice, st));
    // step i: alpha = g_i / |A p|^2, x += alpha p, r -= alpha A p,
    // z' = A^H r, beta = g_{i+1} / g_i, p = z' + beta p; the x update is
    // deferred into the direction update (one pass over p), and the last
    // step updates x only (r is not needed after it)
    for (int i = 0; i < cg_iters; ++i) {
      DD_TRY(apply_op_norm(cp.ptr, w.ptr, false, nw, st));  // w = A p, |w|^2
      if (i + 1 == cg_iters) {
        if (pv == P64)
          DD_TRY(blas_cg_x<P64>(z, cp.ptr, g[i & 1], nw, L, N, st));
        else
          DD_TRY(blas_cg_x<P32>(z, cp.ptr, g[i & 1], nw, L, N, st));
        break;
      }
      if (pv == P64)
        DD_TRY(blas_cg_r<P64>(cr.ptr, w.ptr, g[i & 1], nw, L, N, st));
      else
        DD_TRY(blas_cg_r<P32>(cr.ptr, w.ptr, g[i & 1], nw, L, N, st));
      DD_TRY(apply_op_norm(cr.ptr, cz.ptr, true, g[(i + 1) & 1], st));  // z' = A^H r, |z'|^2
      if (pv == P64)
        DD_TRY(blas_cg_xp<P64>(z, cp.ptr, cz.ptr, g[i & 1], nw, g[(i + 1) & 1], L, N, st));
      else
        DD_TRY(blas_cg_xp<P32>(z, cp.ptr, cz.ptr, g[i & 1], nw, g[(i + 1) & 1], L, N, st));
    }
    return DD_OK;
  }

  int dots(const VecList& vs, int J, const void* x, double2* out, int add, cudaStream_t st) {
    if (pv == P64) return blas_multidot<P64>(vs, J, x, L, N, out, add, (double2*)partials.ptr, st);
    return blas_multidot<P32>(vs, J, x, L, N, out, add, (double2*)partials.ptr, st);
  }
  int axpys(const VecList& vs, int J, const double2* c, double sgn, void* x, cudaStream_t st,
            double2* norm_out = nullptr) {
    double2* pp = (double2*)partials.ptr;
    if (pv == P64) return blas_multiaxpy<P64>(vs, J, c, sgn, x, L, N, st, norm_out, pp);
    return blas_multiaxpy<P32>(vs, J, c, sgn, x, L, N, st, norm_out, pp);
  }
  int scale(const double2* c, const void* in, void* out, cudaStream_t st) {
    if (pv == P64) return blas_scale<P64>(c, in, out, L, N, st);
    return blas_scale<P32>(c, in, out, L, N, st);
  }
  int norms(const void* x, std::vector<double>& out, cudaStream_t st) {
    VecList vs;
    vs.p[0] = x;
    double2* d = reinterpret_cast<double2*>(red.ptr);
    DD_TRY(dots(vs, 1, x, d, 0, st));
    DD_CUDA(cudaMemcpyAsync(hred.p, d, N * sizeof(double2), cudaMemcpyDeviceToHost, st));
    DD_CUDA(cudaStreamSynchronize(st));
    const double2* h = reinterpret_cast<const double2*>(hred.p);
    out.resize(N);
    for (int r = 0; r < N; ++r) out[r] = std::sqrt(std::max(h[r].x, 0.0));
    return DD_OK;
  }

  // Solve A e = f; e (a vector of this solver's shape) must be zero on entry.
  // tol_rel[r]: requested reduction of ||f_r - A e_r|| / ||f_r||.
  int solve(const void* f, void* e, const std::vector<double>& tol_rel, int max_restarts, cudaStream_t st,
            std::vector<double>* est_out) {
    std::vector<double> fnorm;
    DD_TRY(norms(f, fnorm, st));
    std::vector<cd> H((size_t)N * (m + 1) * m), g((size_t)N * (m + 1)), sn((size_t)N * m);
    std::vector<double> cs((size_t)N * m), est(N), beta(N);
    std::vector<int> k(N), live(N);
    double2* dd = reinterpret_cast<double2*>(red.ptr);
    double2* dots1 = dd;
    double2* dots2 = dd + (size_t)(m + 1) * N;
    double2* nrm = dd + (size_t)2 * (m + 1) * N;
    const double2* h1 = reinterpret_cast<const double2*>(hred.p);
    const double2* h2 = h1 + (size_t)(m + 1) * N;
    const double2* hn = h1 + (size_t)2 * (m + 1) * N;
    double2* hc = reinterpret_cast<double2*>(hcoef.p);
    double2* dcoef = reinterpret_cast<double2*>(coef.ptr);
    bool done = false;
    for (int cyc = 0; cyc < max_restarts && !done; ++cyc) {
      ++cycles;
      // residual of this cycle (Algorithm 2); x0 = 0 on the first
      if (cyc == 0) {
        DD_CUDA(cudaMemcpyAsync(rvec.ptr, f, vbytes, cudaMemcpyDeviceToDevice, st));
      } else {
        DD_TRY(apply_op(e, w.ptr, false, st));
        DD_CUDA(cudaMemcpyAsync(rvec.ptr, f, vbytes, cudaMemcpyDeviceToDevice, st));
        VecList vw;
        vw.p[0] = w.ptr;
        for (int r = 0; r < N; ++r) hc[r] = make_double2(1.0, 0.0);
        DD_CUDA(cudaMemcpyAsync(dcoef, hc, N * sizeof(double2), cudaMemcpyHostToDevice, st));
        DD_TRY(axpys(vw, 1, dcoef, -1.0, rvec.ptr, st));
      }
      DD_TRY(norms(rvec.ptr, beta, st));  // beta = ||r||
      int nlive = 0;
      for (int r = 0; r < N; ++r) {
        live[r] = beta[r] > tol_rel[r] * fnorm[r] && fnorm[r] > 0.0;
        est[r] = fnorm[r] > 0.0 ? beta[r] / fnorm[r] : 0.0;
        nlive += live[r];
        k[r] = 0;
        for (int i = 0; i <= m; ++i) g[(size_t)r * (m + 1) + i] = 0.0;
        g[(size_t)r * (m + 1)] = beta[r];
      }
      if (!nlive) break;
      for (int r = 0; r < N; ++r) hc[r] = make_double2(live[r] ? 1.0 / beta[r] : 0.0, 0.0);
      DD_CUDA(cudaMemcpyAsync(dcoef, hc, N * sizeof(double2), cudaMemcpyHostToDevice, st));
      DD_TRY(scale(dcoef, rvec.ptr, V(0), st));  // v_1 = r / beta
      int jmax = 0;
      for (int j = 0; j < m; ++j) {
        ++steps;
        if (mode == DD_PRECOND_CGNR || mode == DD_PRECOND_CGNR16 || mode == DD_PRECOND_SAP ||
            mode == DD_PRECOND_AMG) {
          if (mode == DD_PRECOND_CGNR)
            DD_TRY(cgnr(V(j), Zb(j), st));  // z_j = M_j^{-1} v_j
          else if (mode == DD_PRECOND_CGNR16)
            DD_TRY(cgnr16(V(j), Zb(j), st));
          else if (mode == DD_PRECOND_SAP)
            DD_TRY(sap(V(j), Zb(j), st));
          else
            DD_TRY(amgp(V(j), Zb(j), st));
          DD_TRY(apply_op(Zb(j), w.ptr, false, st));  // w = A z_j
        } else {
          DD_TRY(apply(V(j), w.ptr, st));  // w = A z_j (z_j = v_j, or A^H v_j for the fixed preconditioner)
        }
        VecList vs;
        for (int i = 0; i <= j; ++i) vs.p[i] = V(i);
        // classical Gram-Schmidt (one pass, or two when
        // gs_passes = 2); the norm h_{j+1,j} is fused into the last update
        DD_TRY(dots(vs, j + 1, w.ptr, dots1, 0, st));
        if (gs_passes > 1) {
          DD_TRY(axpys(vs, j + 1, dots1, -1.0, w.ptr, st));
          DD_TRY(dots(vs, j + 1, w.ptr, dots2, 0, st));
          DD_TRY(axpys(vs, j + 1, dots2, -1.0, w.ptr, st, nrm));
        } else {
          DD_CUDA(cudaMemsetAsync(dots2, 0, (size_t)(j + 1) * N * sizeof(double2), st));
          DD_TRY(axpys(vs, j + 1, dots1, -1.0, w.ptr, st, nrm));
        }
        DD_CUDA(cudaMemcpyAsync(hred.p, dd, (size_t)(2 * (m + 1) + 1) * N * sizeof(double2), cudaMemcpyDeviceToHost,
                                st));
        DD_CUDA(cudaStreamSynchronize(st));
        int still = 0;
        for (int r = 0; r < N; ++r) {
          hc[r] = make_double2(0.0, 0.0);
          if (!live[r]) continue;
          cd* h = &H[((size_t)r * m + j) * (m + 1)];
          for (int i = 0; i <= j; ++i) {
            const double2 a = h1[(size_t)i * N + r], b = h2[(size_t)i * N + r];
            h[i] = cd(a.x + b.x, a.y + b.y);
          }
          const double hn1 = std::sqrt(std::max(hn[r].x, 0.0));
          h[j + 1] = hn1;
          // apply the previous rotations to the new column
          for (int i = 0; i < j; ++i) {
            const double c = cs[(size_t)r * m + i];
            const cd s = sn[(size_t)r * m + i];
            const cd t = c * h[i] + s * h[i + 1];
            h[i + 1] = -std::conj(s) * h[i] + c * h[i + 1];
            h[i] = t;
          }
          // new rotation zeroing h[j+1]
          const double aa = std::abs(h[j]), bb = std::abs(h[j + 1]);
          const double rho = std::sqrt(aa * aa + bb * bb);
          double c;
          cd s;
          if (aa == 0.0) {
            c = 0.0;
            s = 1.0;
            h[j] = rho;
          } else {
            c = aa / rho;
            s = (h[j] / aa) * std::conj(h[j + 1]) / rho;
            h[j] = (h[j] / aa) * rho;
          }
          h[j + 1] = 0.0;
          cs[(size_t)r * m + j] = c;
          sn[(size_t)r * m + j] = s;
          cd* gr = &g[(size_t)r * (m + 1)];
          gr[j + 1] = -std::conj(s) * gr[j];
          gr[j] = c * gr[j];
          k[r] = j + 1;
          est[r] = std::abs(gr[j + 1]) / fnorm[r];
          const bool conv = std::abs(gr[j + 1]) < tol_rel[r] * fnorm[r];
          const bool brk = hn1 < 0.1 * tol_rel[r] * fnorm[r];
          if (conv || brk || rho == 0.0) {
            live[r] = 0;
          } else {
            hc[r] = make_double2(1.0 / hn1, 0.0);
            ++still;
          }
        }
        jmax = j + 1;
        if (!still) break;
        DD_CUDA(cudaMemcpyAsync(dcoef, hc, N * sizeof(double2), cudaMemcpyHostToDevice, st));
        DD_TRY(scale(dcoef, w.ptr, V(j + 1), st));  // v_{j+1} = w / h_{j+1,j}
      }
      DD_CUDA(cudaStreamSynchronize(st));  // the last coefficient upload has landed before hc is reused
      // back substitution R y = g, then e += Z_m y
      std::vector<cd> y((size_t)N * m);
      for (int r = 0; r < N; ++r) {
        for (int i = k[r] - 1; i >= 0; --i) {
          cd acc = g[(size_t)r * (m + 1) + i];
          for (int l = i + 1; l < k[r]; ++l) acc -= H[((size_t)r * m + l) * (m + 1) + i] * y[(size_t)r * m + l];
          y[(size_t)r * m + i] = acc / H[((size_t)r * m + i) * (m + 1) + i];
        }
      }
      for (int i = 0; i < jmax; ++i)
        for (int r = 0; r < N; ++r) {
          const cd v = i < k[r] ? y[(size_t)r * m + i] : cd(0.0);
          hc[(size_t)i * N + r] = make_double2(v.real(), v.imag());
        }
      DD_CUDA(cudaMemcpyAsync(dcoef, hc, (size_t)jmax * N * sizeof(double2), cudaMemcpyHostToDevice, st));
      VecList vs;
      for (int i = 0; i < jmax; ++i)
        vs.p[i] = (mode == DD_PRECOND_CGNR || mode == DD_PRECOND_CGNR16 || mode == DD_PRECOND_SAP ||
                   mode == DD_PRECOND_AMG)
                      ? Zb(i)
                      : V(i);
      if (!normal) {
        DD_TRY(axpys(vs, jmax, dcoef, 1.0, e, st));  // e += Z_m y (Z_m = V_m without preconditioner)
      } else {
        // fixed preconditioner: e += M^{-1} (V y) (Algorithm 1)
        DD_CUDA(cudaMemsetAsync(ut.ptr, 0, vbytes, st));
        DD_TRY(axpys(vs, jmax, dcoef, 1.0, ut.ptr, st));
        DD_TRY(apply_op(ut.ptr, zt.ptr, true, st));
        VecList vz;
        vz.p[0] = zt.ptr;
        DD_CUDA(cudaStreamSynchronize(st));
        for (int r = 0; r < N; ++r) hc[r] = make_double2(1.0, 0.0);
        DD_CUDA(cudaMemcpyAsync(dcoef, hc, N * sizeof(double2), cudaMemcpyHostToDevice, st));
        DD_TRY(axpys(vz, 1, dcoef, 1.0, e, st));
      }
      DD_CUDA(cudaStreamSynchronize(st));  // hc is reused by the next cycle
      if (verbose) {
        double worst = 0.0;
        for (int r = 0; r < N; ++r) worst = std::max(worst, est[r]);
        fprintf(stderr, "[dd_solve]   cycle %d: %d steps, max residual estimate %.3e\n", cycles, jmax, worst);
      }
      done = true;
      for (int r = 0; r < N; ++r)
        if (est[r] >= tol_rel[r] && fnorm[r] > 0.0) done = false;
    }
    if (est_out) *est_out = est;
    return DD_OK;
  }
};

int dot_norms64(const dd_lattice* lat, const void* x, int N, double2* scratch_red, double2* partials,
                Pinned& hbuf, std::vector<double>& out, cudaStream_t st) {
  VecList vs;
  vs.p[0] = x;
  const int64_t L = (int64_t)(field_bytes(lat, P64, 0, N) / 16);
  DD_TRY(blas_multidot<P64>(vs, 1, x, L, N, scratch_red, 0, partials, st));
  DD_CUDA(cudaMemcpyAsync(hbuf.p, scratch_red, N * sizeof(double2), cudaMemcpyDeviceToHost, st));
  DD_CUDA(cudaStreamSynchronize(st));
  out.resize(N);
  const double2* h = reinterpret_cast<const double2*>(hbuf.p);
  for (int r = 0; r < N; ++r) out[r] = std::sqrt(std::max(h[r].x, 0.0));
  return DD_OK;
}

int half_norms64(const dd_lattice* lat, const void* x, int N, double2* red, double2* partials, Pinned& hbuf,
                 std::vector<double>& out, cudaStream_t st) {
  VecList vs;
  vs.p[0] = x;
  const int64_t L = (int64_t)(field_bytes(lat, P64, 1, N) / 16);
  DD_TRY(blas_multidot<P64>(vs, 1, x, L, N, red, 0, partials, st));
  DD_CUDA(cudaMemcpyAsync(hbuf.p, red, N * sizeof(double2), cudaMemcpyDeviceToHost, st));
  DD_CUDA(cudaStreamSynchronize(st));
  out.resize(N);
  const double2* h = reinterpret_cast<const double2*>(hbuf.p);
  for (int r = 0; r < N; ++r) out[r] = std::max(h[r].x, 0.0);  // squared norms
  return DD_OK;
}

// One batch of nb right-hand sides of the even-odd solve.  FP64 refinement
// runs on the odd-site Schur system Dhat x_o = bhat_o; x_e is reconstructed
// and the full-system FP64 residual ||b - D x|| is verified at the end (and
// refinement resumes with a tighter target if it is not met).  Only six FP64
// half fields are kept, which lets large lattices fit.
int schur_batch(dd_clover* op, const dd_solve_params* prm, const double* b_in, double* x_io, int nb, bool host,
                Inner& inner, cudaStream_t st, dd_stats& s, double& worst_out, bool& ok_out) {
  const dd_lattice* lat = op->lat;
  const int pin = prm->inner_prec;
  const int pv = (pin == P64 || pin == PDF) ? P64 : P32;  // FP32 pairs work on FP64 vectors
  // the refinement's operator on the FP64 vectors: FP64 or FP32-pair arithmetic
  const int rp = prm->refine_prec == DD_PREC_DF64 ? PDF : P64;
  const size_t h64 = field_bytes(lat, P64, 1, nb);
  const size_t canon = (size_t)lat->V * 12 * 16 * nb;
  DevBuf be, bo, bh, xo, ro, te, stage, red, partials, fv, ev;
  Pinned hbuf;
  DD_TRY(hbuf.alloc((size_t)nb * sizeof(double2)));
  DD_TRY(red.alloc((size_t)nb * sizeof(double2)));
  DD_TRY(partials.alloc((size_t)blas_partials_len(nb) * sizeof(double2)));
  for (DevBuf* d : {&be, &bo, &bh, &xo, &ro, &te}) DD_TRY(d->alloc(h64));
  const double* bsrc = b_in;
  double* xdst = x_io;
  if (host) {
    DD_TRY(stage.alloc(canon));
    DD_CUDA(cudaMemcpyAsync(stage.ptr, b_in, canon, cudaMemcpyHostToDevice, st));
    bsrc = reinterpret_cast<const double*>(stage.ptr);
  }
  Field BE = field_view(lat, P64, 2, be.ptr, nb), BO = field_view(lat, P64, 1, bo.ptr, nb);
  Field BH = field_view(lat, P64, 1, bh.ptr, nb), XO = field_view(lat, P64, 1, xo.ptr, nb);
  Field RO = field_view(lat, P64, 1, ro.ptr, nb), TE = field_view(lat, P64, 2, te.ptr, nb);
  DD_TRY(pack(lat, P64, 3, bsrc, BE, st));
  DD_TRY(pack(lat, P64, 4, bsrc, BO, st));
  if (host) {
    DD_CUDA(cudaMemcpyAsync(stage.ptr, x_io, canon, cudaMemcpyHostToDevice, st));
    DD_TRY(pack(lat, P64, 4, reinterpret_cast<const double*>(stage.ptr), XO, st));
  } else {
    DD_TRY(pack(lat, P64, 4, x_io, XO, st));
  }
  Field B;  // the full right-hand side as two half fields
  B.prec = P64;
  B.nrhs = nb;
  B.h[0] = BE.h[0];
  B.h[1] = BO.h[1];
  std::vector<double> n_e, n_o, bnorm(nb), rn;
  DD_TRY(half_norms64(lat, be.ptr, nb, (double2*)red.ptr, (double2*)partials.ptr, hbuf, n_e, st));
  DD_TRY(half_norms64(lat, bo.ptr, nb, (double2*)red.ptr, (double2*)partials.ptr, hbuf, n_o, st));
  for (int r = 0; r < nb; ++r) {
    bnorm[r] = std::sqrt(n_e[r] + n_o[r]);
    if (!std::isfinite(bnorm[r])) return fail(DD_ERR_ARG, "right-hand side contains NaN or Inf");
  }
  DD_TRY(op_prepare(op, rp, P64, B, BH, TE, st));
  if (pv == P32) {
    DD_TRY(fv.alloc(field_bytes(lat, P32, 1, nb)));
    DD_TRY(ev.alloc(field_bytes(lat, P32, 1, nb)));
  } else {
    DD_TRY(ev.alloc(h64));
  }
  double target = 0.5;  // refine the Schur residual to target * tol, then verify
  bool ok = false;
  double worst = 0.0;
  for (int outer = 0;; ++outer) {
    DD_TRY(op_dhat_residual(op, rp, P64, BH, XO, RO, TE, st));
    ++s.applies_fp64;
    DD_TRY(half_norms64(lat, ro.ptr, nb, (double2*)red.ptr, (double2*)partials.ptr, hbuf, rn, st));
    bool reached = true;
    for (int r = 0; r < nb; ++r)
      if (bnorm[r] > 0 && !(std::sqrt(rn[r]) < target * prm->tol * bnorm[r])) reached = false;
    if (reached || outer >= prm->max_outer) {
      // x_e = A_ee^{-1} (b_e - D_eo x_o); full residual r = b - D x in FP64
      Field X;
      X.prec = P64;
      X.nrhs = nb;
      X.h[0] = TE.h[0];
      X.h[1] = XO.h[1];
      DD_TRY(op_reconstruct(op, rp, P64, B, X, st));
      Field R;
      R.prec = P64;
      R.nrhs = nb;
      R.h[0] = field_view(lat, P64, 2, bh.ptr, nb).h[0];
      R.h[1] = RO.h[1];
      DD_TRY(op_residual(op, rp, P64, B, X, R, st));
      ++s.applies_fp64;
      DD_TRY(half_norms64(lat, bh.ptr, nb, (double2*)red.ptr, (double2*)partials.ptr, hbuf, n_e, st));
      DD_TRY(half_norms64(lat, ro.ptr, nb, (double2*)red.ptr, (double2*)partials.ptr, hbuf, n_o, st));
      ok = true;
      worst = 0.0;
      for (int r = 0; r < nb; ++r) {
        const double rel = bnorm[r] > 0 ? std::sqrt(n_e[r] + n_o[r]) / bnorm[r] : 0.0;
        worst = std::max(worst, rel);
        if (!(rel < prm->tol) && bnorm[r] > 0) ok = false;
      }
      if (prm->verbose)
        fprintf(stderr, "[dd_solve] outer %d  full FP64 residual max %.3e  inner steps so far %d\n", outer, worst,
                inner.steps);
      if (ok || outer >= prm->max_outer) {
        s.outer_iterations += outer;
        // write x back (both parities)
        double* xc = host ? reinterpret_cast<double*>(stage.ptr) : xdst;
        DD_TRY(unpack(lat, P64, 3, X, xc, st));
        DD_TRY(unpack(lat, P64, 4, X, xc, st));
        if (host) DD_CUDA(cudaMemcpyAsync(x_io, stage.ptr, canon, cudaMemcpyDeviceToHost, st));
        DD_CUDA(cudaStreamSynchronize(st));
        break;
      }
      target *= 0.1;  // the Schur residual understated the full one: tighten and go on
      DD_TRY(op_prepare(op, rp, P64, B, BH, TE, st));  // bh held r_e
      continue;
    }
    if (prm->verbose) {
      double w = 0.0;
      for (int r = 0; r < nb; ++r) w = std::max(w, bnorm[r] > 0 ? std::sqrt(rn[r]) / bnorm[r] : 0.0);
      fprintf(stderr, "[dd_solve] outer %d  Schur FP64 residual max %.3e  inner steps so far %d\n", outer, w,
              inner.steps);
    }
    // inner solve of Dhat e = r in the inner precision
    const void* f = ro.ptr;
    if (pv == P32) {
      DD_TRY(blas_demote(ro.ptr, fv.ptr, 1, lat->Vh * nb, st));
      f = fv.ptr;
    }
    DD_CUDA(cudaMemsetAsync(ev.ptr, 0, pv == P32 ? field_bytes(lat, P32, 1, nb) : h64, st));
    std::vector<double> fn;
    DD_TRY(inner.norms(f, fn, st));
    std::vector<double> tol_rel(nb);
    for (int r = 0; r < nb; ++r) {
      const double need = fn[r] > 0 ? 0.3 * target * prm->tol * bnorm[r] / fn[r] : 1.0;
      tol_rel[r] = pv == P64 ? need : std::max(prm->inner_tol, need);
    }
    DD_TRY(inner.solve(f, ev.ptr, tol_rel, prm->max_restarts, st, nullptr));
    if (pv == P32)
      DD_TRY(blas_promote_add(ev.ptr, xo.ptr, 1, lat->Vh * nb, st));
    else
      DD_TRY(blas_add64(ev.ptr, xo.ptr, (int64_t)(h64 / 16), st));
  }
  worst_out = worst;
  ok_out = ok;
  return DD_OK;
}

}  // namespace

// Even-odd solve: the right-hand sides in batches of prm->rhs_batch.
int solve_schur(dd_clover* op, const dd_solve_params* prm, const double* b, double* x, int N, bool host,
                cudaStream_t st, dd_stats* stats) {
  const auto t0 = std::chrono::steady_clock::now();
  const dd_lattice* lat = op->lat;
  const int pin = prm->inner_prec;
  const int pv = (pin == P64 || pin == PDF) ? P64 : P32;  // FP32 pairs work on FP64 vectors
  if (prec_index(pin) < 0) return fail(DD_ERR_ARG, "bad inner precision");
  if (!op->clov[prec_index(pin)].ptr || !op->gauge->links[prec_index(pin)].ptr)
    return fail(DD_ERR_UNSUPPORTED, "inner precision not created in the handles");
  if (prm->restart < 1 || prm->restart > 32) return fail(DD_ERR_ARG, "restart must be in 1..32");
  if (prm->gs_passes < 1 || prm->gs_passes > 2) return fail(DD_ERR_ARG, "gs_passes must be 1 or 2");
  const int nbmax = prm->rhs_batch > 0 ? std::min(prm->rhs_batch, N) : N;
  dd_stats s{};
  Inner inner;
  bool all_ok = true;
  double worst = 0.0;
  for (int r0 = 0; r0 < N; r0 += nbmax) {
    const int nb = std::min(nbmax, N - r0);
    DD_TRY(inner.init(op, pin, pv, true, nb, prm->restart, prm->precond));
    inner.cg_iters = prm->precond_iters;
    inner.set_sap(prm);
    inner.verbose = prm->verbose;
    inner.gs_passes = prm->gs_passes;
    const size_t off = (size_t)r0 * lat->V * 24;  // doubles per RHS: V sites x 12 complex
    double w = 0.0;
    bool ok = false;
    DD_TRY(schur_batch(op, prm, b + off, x + off, nb, host, inner, st, s, w, ok));
    worst = std::max(worst, w);
    all_ok = all_ok && ok;
  }
  s.converged = all_ok;
  s.true_residual = worst;
  s.inner_iterations = inner.steps;
  s.restarts = inner.cycles;
  s.applies_inner = inner.applies;
  s.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = s;
  if (!all_ok) return fail(DD_ERR_NOT_CONVERGED, "solver reached its iteration limits");
  return DD_OK;
}

int solve(dd_clover* op, const dd_solve_params* prm, const double* b_canon, double* x_canon, int N, cudaStream_t st,
          dd_stats* stats) {
  const auto t0 = std::chrono::steady_clock::now();
  const dd_lattice* lat = op->lat;
  const int pin = prm->inner_prec;
  const int pv = (pin == P64 || pin == PDF) ? P64 : P32;  // FP32 pairs work on FP64 vectors
  const int pg = pin;
  const int rp = prm->refine_prec == DD_PREC_DF64 ? PDF : P64;  // the refinement operator
  if (prec_index(pin) < 0) return fail(DD_ERR_ARG, "bad inner precision");
  if (!op->clov[prec_index(pg)].ptr || !op->gauge->links[prec_index(pg)].ptr)
    return fail(DD_ERR_UNSUPPORTED, "inner precision not created in the handles");
  if (prm->restart < 1 || prm->restart > 32) return fail(DD_ERR_ARG, "restart must be in 1..32");
  if (prm->gs_passes < 1 || prm->gs_passes > 2) return fail(DD_ERR_ARG, "gs_passes must be 1 or 2");
  const bool eo = prm->even_odd != 0;
  const size_t f64 = field_bytes(lat, P64, 0, N);
  DevBuf b64, x64, r64, r32, fvec, evec, tmp, red, partials;
  Pinned hbuf;
  DD_TRY(hbuf.alloc((size_t)N * sizeof(double2)));
  DD_TRY(b64.alloc(f64));
  DD_TRY(x64.alloc(f64));
  DD_TRY(r64.alloc(f64));
  DD_TRY(red.alloc((size_t)N * sizeof(double2)));
  DD_TRY(partials.alloc((size_t)blas_partials_len(N) * sizeof(double2)));
  if (pv == P32) DD_TRY(r32.alloc(field_bytes(lat, P32, 0, N)));
  DD_TRY(evec.alloc(field_bytes(lat, pv, 0, N)));
  if (eo) {
    DD_TRY(fvec.alloc(field_bytes(lat, pv, 1, N)));
    DD_TRY(tmp.alloc(field_bytes(lat, pv, 2, N)));
  }
  Field B = field_view(lat, P64, 0, b64.ptr, N), X = field_view(lat, P64, 0, x64.ptr, N),
        Rr = field_view(lat, P64, 0, r64.ptr, N);
  DD_TRY(pack(lat, P64, 0, b_canon, B, st));
  DD_TRY(pack(lat, P64, 0, x_canon, X, st));
  std::vector<double> bnorm, rnorm;
  DD_TRY(dot_norms64(lat, b64.ptr, N, (double2*)red.ptr, (double2*)partials.ptr, hbuf, bnorm, st));

  for (int r = 0; r < N; ++r)
    if (!std::isfinite(bnorm[r])) return fail(DD_ERR_ARG, "right-hand side contains NaN or Inf");
  Inner inner;
  DD_TRY(inner.init(op, pg, pv, eo, N, prm->restart, prm->precond));
  inner.cg_iters = prm->precond_iters;
  inner.set_sap(prm);
  inner.verbose = prm->verbose;
  inner.gs_passes = prm->gs_passes;
  dd_stats s{};
  int status = DD_ERR_NOT_CONVERGED;
  for (int outer = 0;; ++outer) {
    DD_TRY(op_residual(op, rp, P64, B, X, Rr, st));  // r = b - D x in FP64
    ++s.applies_fp64;
    DD_TRY(dot_norms64(lat, r64.ptr, N, (double2*)red.ptr, (double2*)partials.ptr, hbuf, rnorm, st));
    double worst = 0.0;
    bool all = true;
    for (int r = 0; r < N; ++r) {
      const double rel = bnorm[r] > 0 ? rnorm[r] / bnorm[r] : 0.0;
      worst = std::max(worst, rel);
      if (!(rel < prm->tol) && bnorm[r] > 0) all = false;
    }
    s.true_residual = worst;
    s.outer_iterations = outer;
    if (prm->verbose)
      fprintf(stderr, "[dd_solve] outer %d  max ||b-Dx||/||b|| = %.3e  inner steps so far %d\n", outer, worst,
              inner.steps);
    if (all) {
      status = DD_OK;
      break;
    }
    if (outer >= prm->max_outer) break;
    // inner right-hand side in the inner precision
    const void* rin = r64.ptr;
    if (pv == P32) {
      DD_TRY(blas_demote(r64.ptr, r32.ptr, 2, lat->Vh * N, st));
      rin = r32.ptr;
    }
    Field Rin = field_view(lat, pv, 0, const_cast<void*>(rin), N);
    Field E = field_view(lat, pv, 0, evec.ptr, N);
    DD_CUDA(cudaMemsetAsync(evec.ptr, 0, field_bytes(lat, pv, 0, N), st));
    const void* f = rin;
    void* e = evec.ptr;
    if (eo) {
      DD_TRY(op_prepare(op, pg, pv, Rin, field_view(lat, pv, 1, fvec.ptr, N), field_view(lat, pv, 2, tmp.ptr, N),
                        st));
      f = fvec.ptr;
      e = E.h[1].base;
    }
    std::vector<double> fn;
    DD_TRY(inner.norms(f, fn, st));
    std::vector<double> tol_rel(N);
    for (int r = 0; r < N; ++r) {
      const double need = fn[r] > 0 ? 0.3 * prm->tol * bnorm[r] / fn[r] : 1.0;
      tol_rel[r] = std::max(prm->inner_tol, need);
      if (pv == P64) tol_rel[r] = need;  // FP64 inner: one inner solve reaches the target
    }
    DD_TRY(inner.solve(f, e, tol_rel, prm->max_restarts, st, nullptr));
    if (eo) DD_TRY(op_reconstruct(op, pg, pv, Rin, E, st));
    if (pv == P32)
      DD_TRY(blas_promote_add(evec.ptr, x64.ptr, 2, lat->Vh * N, st));
    else
      DD_TRY(blas_add64(evec.ptr, x64.ptr, (int64_t)(f64 / 16), st));
  }
  DD_TRY(unpack(lat, P64, 0, X, x_canon, st));
  DD_CUDA(cudaStreamSynchronize(st));
  s.converged = status == DD_OK;
  s.inner_iterations = inner.steps;
  s.restarts = inner.cycles;
  s.applies_inner = inner.applies;
  s.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = s;
  if (status != DD_OK) set_error("solver reached its iteration limits");
  return status;
}

// ---- GMRES on a custom FP64 operator (the AMG coarse system) ----
struct CoarseKrylov {
  Inner inner;
};

CoarseKrylov* coarse_krylov_create(int64_t L, int N, int m, std::function<int(const void*, void*, cudaStream_t)> op) {
  CoarseKrylov* k = new (std::nothrow) CoarseKrylov();
  if (!k) return nullptr;
  if (k->inner.init_custom(L, N, m) != DD_OK) {
    delete k;
    return nullptr;
  }
  k->inner.custom = std::move(op);
  return k;
}

void coarse_krylov_destroy(CoarseKrylov* k) { delete k; }

int coarse_krylov_solve(CoarseKrylov* k, const void* f, void* e, double tol_rel, int max_restarts, cudaStream_t st,
                        int* steps) {
  const int before = k->inner.steps;
  std::vector<double> tol((size_t)k->inner.N, tol_rel);
  DD_CUDA(cudaMemsetAsync(e, 0, k->inner.vbytes, st));
  DD_TRY(k->inner.solve(f, e, tol, max_restarts, st, nullptr));
  if (steps) *steps = k->inner.steps - before;
  return DD_OK;
}

}  // namespace dd
