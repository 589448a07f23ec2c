// Operator layer: D, D^H, D_sc and the even-odd pieces built from the fused
// stencil kernel, plus handle helpers and error reporting.
#include <cstdio>
#include <mutex>
#include <string>

#include "dd_internal.h"
#include "dd_ops.h"

namespace dd {

// ---------------------------------------------------------------- errors
namespace {
thread_local std::string g_last_error = "no error";
}

void set_error(const std::string& msg) { g_last_error = msg; }
const char* last_error() { return g_last_error.c_str(); }

int fail(int status, const std::string& msg) {
  set_error(msg);
  return status;
}

int cuda_fail(cudaError_t e, const char* where) {
  set_error(std::string(where) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? DD_ERR_OOM : DD_ERR_CUDA;
}

// ---------------------------------------------------------------- buffers
int DevBuf::alloc(size_t n) {
  release();
  if (n == 0) return DD_OK;
  cudaError_t e = cudaMalloc(&ptr, n);
  if (e != cudaSuccess) {
    ptr = nullptr;
    (void)cudaGetLastError();
    return fail(DD_ERR_OOM, "cudaMalloc of " + std::to_string(n) + " bytes failed");
  }
  bytes = n;
  return DD_OK;
}

int DevBuf::ensure(size_t n) {
  if (n <= bytes) return DD_OK;
  return alloc(n);
}

void DevBuf::release() {
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
  bytes = 0;
}

// ---------------------------------------------------------------- fields
size_t field_bytes(const dd_lattice* lat, int prec, int subset, int nrhs) {
  size_t h = (prec == P64 || prec == PDF) ? half_field_bytes<P64>(lat->Vh, nrhs)
             : prec == P32 ? half_field_bytes<P32>(lat->Vh, nrhs)
                           : half_field_bytes<P16>(lat->Vh, nrhs);
  return subset == 0 ? 2 * h : h;
}

static HalfField half_view(const dd_lattice* lat, int prec, char* base, int nrhs) {
  HalfField h;
  h.base = base;
  h.scale = nullptr;
  if (prec == P16) h.scale = reinterpret_cast<float*>(base + (size_t)lat->Vh * nrhs * 3 * 16);
  return h;
}

Field field_view(const dd_lattice* lat, int prec, int subset, void* base, int nrhs, int paired) {
  Field f;
  f.prec = prec;
  f.nrhs = nrhs;
  f.paired = paired;
  char* b = reinterpret_cast<char*>(base);
  const size_t hb = field_bytes(lat, prec, 1, nrhs);
  f.h[0] = HalfField{nullptr, nullptr};
  f.h[1] = HalfField{nullptr, nullptr};
  if (subset == 0) {
    f.h[0] = half_view(lat, prec, b, nrhs);
    f.h[1] = half_view(lat, prec, b + hb, nrhs);
  } else if (subset == 1) {
    f.h[1] = half_view(lat, prec, b, nrhs);
  } else {
    f.h[0] = half_view(lat, prec, b, nrhs);
  }
  return f;
}

int64_t stencil_bytes_per_site(int pg, int nrhs) {
  return (pg == P64 || pg == PDF) ? 1152 + 384 * nrhs : pg == P32 ? 576 + 192 * nrhs : 288 + 104 * nrhs;
}

// Depth of the Z-slabs of the full-lattice traversal: the largest divisor of
// nZ whose slab-slice (depth * nY * nX sites) moves at most ~30 MB through the
// stencil (bytes_per_site per site), well inside L2; DD_ZBLOCK overrides
// (0 = no slabs).  Measured at 48^3 x 96: 16 for FP32 with one RHS (+4%);
// at 32^4 with 12 RHS: 8 (+13%).
int* device_error_flag() {
  static int* flag = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    if (cudaMalloc(&p, sizeof(int)) == cudaSuccess && cudaMemset(p, 0, sizeof(int)) == cudaSuccess)
      flag = static_cast<int*>(p);
  });
  return flag;
}

int zblock_for(const int dims[4], int64_t bytes_per_site) {
  static int forced = -2;
  if (forced == -2) {
    const char* e = getenv("DD_ZBLOCK");
    forced = e ? atoi(e) : -1;
  }
  const int nZ = dims[1];
  const int64_t plane = (int64_t)dims[2] * dims[3];
  if (forced == 0) return nZ;
  if (forced > 0 && nZ % forced == 0) return forced;
  const int64_t budget = 30000000;
  int best = 1;
  for (int b = 1; b <= nZ; ++b)
    if (nZ % b == 0 && b * plane * bytes_per_site <= budget) best = b;
  return best;
}

// ---------------------------------------------------------------- dispatch
namespace {



int run_hop(int pg, int pv, const HopArgs& a, bool dag, int epi, cudaStream_t st) {
  cudaError_t e;
  if (a.paired) {
    if (a.nrhs % 2 != 0 || (epi != EPI_D && epi != EPI_AINV))
      return fail(DD_ERR_UNSUPPORTED, "paired layout: an even RHS count and the D / Dhat stencils only");
    if (pg == P32 && pv == P32)
      e = launch_hop_pair<P32, P32>(a, dag, epi, st);
    else if (pg == P16 && pv == P16)
      e = launch_hop_pair<P16, P16>(a, dag, epi, st);
    else if (pg == P16 && pv == P32)
      e = launch_hop_pair<P16, P32>(a, dag, epi, st);
    else
      return fail(DD_ERR_UNSUPPORTED, "paired layout: FP32 or FP16 only");
    if (e != cudaSuccess) return cuda_fail(e, "paired stencil launch");
    return DD_OK;
  }
  if (pg == P64 && pv == P64)
    e = launch_hop<P64, P64, P64>(a, dag, epi, st);
  else if (pg == PDF && pv == PDF)
    e = launch_hop<PDF, PDF, PDF>(a, dag, epi, st);
  else if (pg == PDF && pv == P64)
    e = launch_hop<PDF, P64, P64>(a, dag, epi, st);
  else if (pg == P32 && pv == P32)
    e = launch_hop<P32, P32, P32>(a, dag, epi, st);
  else if (pg == P16 && pv == P16)
    e = launch_hop<P16, P16, P16>(a, dag, epi, st);
  else if (pg == P16 && pv == P32)
    e = launch_hop<P16, P32, P32>(a, dag, epi, st);
  else if (pg == P32 && pv == P16)
    e = launch_hop<P32, P16, P16>(a, dag, epi, st);
  else
    return fail(DD_ERR_UNSUPPORTED, "unsupported precision pair");
  if (e != cudaSuccess) return cuda_fail(e, "stencil launch");
  return DD_OK;
}

int check_prec(const dd_clover* op, int pg) {
  int pi = prec_index(pg);
  if (pi < 0) return fail(DD_ERR_ARG, "bad precision");
  if (!op->gauge->links[pi].ptr || !op->clov[pi].ptr)
    return fail(DD_ERR_UNSUPPORTED, "precision not created in the gauge/operator handles");
  return DD_OK;
}

HopArgs base_args(const dd_clover* op, int pg, int nrhs) {
  HopArgs a;
  a.g = op->lat->geom();
  a.g.zblock = zblock_for(op->lat->dims, stencil_bytes_per_site(pg, nrhs));
  a.nrhs = nrhs;
  a.p0 = 0;
  a.npar = 2;
  a.gstride = op->lat->Vh * nrhs;
  const int pi = prec_index(pg);
  a.U[0] = op->gauge->U(pi, 0);
  a.U[1] = op->gauge->U(pi, 1);
  a.M[0] = op->M(pi, 0);
  a.M[1] = op->M(pi, 1);
  for (int p = 0; p < 2; ++p) {
    a.in[p] = a.out[p] = a.y[p] = a.z[p] = HalfField{nullptr, nullptr};
  }
  a.beta = -0.5;
  a.rhs_block = 1;
  a.paired = 0;
  // single right-hand side: the compressed FP32 links (fewer bytes; the
  // RHS-blocked kernels of several RHS are faster with three rows)
  a.recon = pg == P32 && nrhs == 1 ? op->gauge->recon32 : pg == P16 && nrhs == 1 && op->gauge->recon16 ? 12 : 0;
  if (a.recon) {
    a.U[0] = pg == P32 ? op->gauge->U2(0) : op->gauge->U2h(0);
    a.U[1] = pg == P32 ? op->gauge->U2(1) : op->gauge->U2h(1);
  }
  return a;
}

}  // namespace

// D (or D^H) on the full lattice: out_p = A_pp in_p - 1/2 H_{p,1-p} in_{1-p}
int op_D(const dd_clover* op, int pg, int pv, bool dagger, const Field& in, const Field& out, cudaStream_t st) {
  DD_TRY(check_prec(op, pg));
  if (in.paired != out.paired) return fail(DD_ERR_ARG, "input and output layouts differ");
  HopArgs a = base_args(op, pg, in.nrhs);
  a.paired = in.paired;
  for (int p = 0; p < 2; ++p) {
    a.in[p] = in.h[p];
    a.y[p] = in.h[p];
    a.out[p] = out.h[p];
  }
  return run_hop(pg, pv, a, dagger, EPI_D, st);
}

int op_D_slices(const dd_clover* op, int pg, int pv, bool dagger, const Field& in, const Field& out, int t0, int nt,
                cudaStream_t st) {
  DD_TRY(check_prec(op, pg));
  if (t0 < 0 || nt < 1 || t0 + nt > op->lat->dims[0]) return fail(DD_ERR_ARG, "bad time-slice range");
  HopArgs a = base_args(op, pg, in.nrhs);
  a.g.t0 = t0;
  a.g.nt = nt;
  for (int p = 0; p < 2; ++p) {
    a.in[p] = in.h[p];
    a.y[p] = in.h[p];
    a.out[p] = out.h[p];
  }
  return run_hop(pg, pv, a, dagger, EPI_D, st);
}

int run_block(int pg, int pv, const BlockArgs& a, cudaStream_t st) {
  cudaError_t e;
  if (pg == P64 && pv == P64)
    e = launch_block<P64, P64, P64>(a, st);
  else if (pg == PDF && pv == PDF)
    e = launch_block<PDF, PDF, PDF>(a, st);
  else if (pg == PDF && pv == P64)
    e = launch_block<PDF, P64, P64>(a, st);
  else if (pg == P32 && pv == P32)
    e = launch_block<P32, P32, P32>(a, st);
  else if (pg == P16 && pv == P16)
    e = launch_block<P16, P16, P16>(a, st);
  else if (pg == P16 && pv == P32)
    e = launch_block<P16, P32, P32>(a, st);
  else if (pg == P32 && pv == P16)
    e = launch_block<P32, P16, P16>(a, st);
  else
    return fail(DD_ERR_UNSUPPORTED, "unsupported precision pair");
  if (e != cudaSuccess) return cuda_fail(e, "self-coupling launch");
  return DD_OK;
}

int op_SC(const dd_clover* op, int pg, int pv, const Field& in, const Field& out, cudaStream_t st) {
  DD_TRY(check_prec(op, pg));
  BlockArgs a;
  a.Vh = op->lat->Vh;
  a.nrhs = in.nrhs;
  a.p0 = 0;
  a.npar = 2;
  a.gstride = a.Vh * in.nrhs;
  const int pi = prec_index(pg);
  for (int p = 0; p < 2; ++p) {
    a.y[p] = in.h[p];
    a.out[p] = out.h[p];
    a.M[p] = op->M(pi, p);
  }
  return run_block(pg, pv, a, st);
}

// Dhat in_o = A_oo in_o - (1/4) H_oe A_ee^{-1} H_eo in_o (D_eo = -1/2 H_eo):
//   tmp_e = A_ee^{-1} (1/2 H_eo in_o);  out_o = A_oo in_o - 1/2 H_oe tmp_e
// The two launches of Dhat: a) tmp_e = A_ee^{-1} (1/2 H_eo in_o);
// b) out_o = A_oo in_o - 1/2 H_oe tmp_e.
static void dhat_args(const dd_clover* op, int pg, const Field& in, const Field& out, const Field& tmp, HopArgs& a,
                      HopArgs& b) {
  a = base_args(op, pg, in.nrhs);
  a.npar = 1;
  a.p0 = 0;
  a.in[1] = in.h[1];
  a.out[0] = tmp.h[0];
  a.M[0] = op->Ainv(prec_index(pg));
  a.beta = 0.5;
  b = base_args(op, pg, in.nrhs);
  b.npar = 1;
  b.p0 = 1;
  b.in[0] = tmp.h[0];
  b.y[1] = in.h[1];
  b.out[1] = out.h[1];
  b.beta = -0.5;
  a.paired = b.paired = in.paired;
}

int op_Dhat(const dd_clover* op, int pg, int pv, bool dagger, const Field& in, const Field& out, const Field& tmp,
            cudaStream_t st) {
  DD_TRY(check_prec(op, pg));
  if (in.paired != out.paired || in.paired != tmp.paired) return fail(DD_ERR_ARG, "field layouts differ");
  HopArgs a, b;
  dhat_args(op, pg, in, out, tmp, a, b);
  DD_TRY(run_hop(pg, pv, a, dagger, EPI_AINV, st));
  return run_hop(pg, pv, b, dagger, EPI_D, st);
}

bool dhat_norm_fused(int pg, int pv, int nrhs) {
  return nrhs == 1 && (pv == P32 || pv == P16) && (pg == P32 || pg == P16);
}

int op_Dhat_norm(const dd_clover* op, int pg, int pv, bool dagger, const Field& in, const Field& out, const Field& tmp,
                 double2* norm_out, double2* partials, int64_t npartials, cudaStream_t st) {
  if (!dhat_norm_fused(pg, pv, in.nrhs))
    return fail(DD_ERR_UNSUPPORTED, "fused norm: one RHS, FP32 or FP16 vectors and links");
  DD_TRY(check_prec(op, pg));
  HopArgs a, b;
  dhat_args(op, pg, in, out, tmp, a, b);
  DD_TRY(run_hop(pg, pv, a, dagger, EPI_AINV, st));
  const cudaError_t e =
      pg == P32 ? (pv == P32 ? launch_hop_norm<P32, P32, P32>(b, dagger, partials, npartials, norm_out, st)
                             : launch_hop_norm<P32, P16, P16>(b, dagger, partials, npartials, norm_out, st))
                : (pv == P32 ? launch_hop_norm<P16, P32, P32>(b, dagger, partials, npartials, norm_out, st)
                             : launch_hop_norm<P16, P16, P16>(b, dagger, partials, npartials, norm_out, st));
  if (e != cudaSuccess) return cuda_fail(e, "stencil launch with norm");
  return DD_OK;
}

int op_residual(const dd_clover* op, int pg, int pv, const Field& b, const Field& x, const Field& r,
                cudaStream_t st) {
  DD_TRY(check_prec(op, pg));
  HopArgs a = base_args(op, pg, x.nrhs);
  for (int p = 0; p < 2; ++p) {
    a.in[p] = x.h[p];
    a.y[p] = x.h[p];
    a.z[p] = b.h[p];
    a.out[p] = r.h[p];
  }
  return run_hop(pg, pv, a, false, EPI_RESID, st);
}

// r_o = bhat_o - (A_oo x_o - 1/2 H_oe tmp_e), tmp_e = A_ee^{-1} (1/2 H_eo x_o)
int op_dhat_residual(const dd_clover* op, int pg, int pv, const Field& bhat, const Field& x, const Field& r,
                     const Field& tmp, cudaStream_t st) {
  DD_TRY(check_prec(op, pg));
  const int pi = prec_index(pg);
  HopArgs a = base_args(op, pg, x.nrhs);
  a.npar = 1;
  a.p0 = 0;
  a.in[1] = x.h[1];
  a.out[0] = tmp.h[0];
  a.M[0] = op->Ainv(pi);
  a.beta = 0.5;
  DD_TRY(run_hop(pg, pv, a, false, EPI_AINV, st));
  HopArgs b = base_args(op, pg, x.nrhs);
  b.npar = 1;
  b.p0 = 1;
  b.in[0] = tmp.h[0];
  b.y[1] = x.h[1];
  b.z[1] = bhat.h[1];
  b.out[1] = r.h[1];
  b.beta = -0.5;
  return run_hop(pg, pv, b, false, EPI_RESID, st);
}

// bhat_o = b_o - D_oe A_ee^{-1} b_e = b_o + 1/2 H_oe (A_ee^{-1} b_e)
int op_prepare(const dd_clover* op, int pg, int pv, const Field& b, const Field& bhat, const Field& tmp,
               cudaStream_t st) {
  DD_TRY(check_prec(op, pg));
  const int pi = prec_index(pg);
  BlockArgs ba;
  ba.Vh = op->lat->Vh;
  ba.nrhs = b.nrhs;
  ba.p0 = 0;
  ba.npar = 1;
  ba.gstride = ba.Vh * b.nrhs;
  ba.y[0] = b.h[0];
  ba.out[0] = tmp.h[0];
  ba.M[0] = op->Ainv(pi);
  ba.y[1] = ba.out[1] = HalfField{nullptr, nullptr};
  ba.M[1] = nullptr;
  DD_TRY(run_block(pg, pv, ba, st));
  HopArgs a = base_args(op, pg, b.nrhs);
  a.npar = 1;
  a.p0 = 1;
  a.in[0] = tmp.h[0];
  a.y[1] = b.h[1];
  a.out[1] = bhat.h[1];
  a.beta = 0.5;
  return run_hop(pg, pv, a, false, EPI_ADD, st);
}

// x_e = A_ee^{-1} (b_e - D_eo x_o) = A_ee^{-1} (b_e + 1/2 H_eo x_o)
int op_reconstruct(const dd_clover* op, int pg, int pv, const Field& b, const Field& x, cudaStream_t st) {
  DD_TRY(check_prec(op, pg));
  const int pi = prec_index(pg);
  HopArgs a = base_args(op, pg, x.nrhs);
  a.npar = 1;
  a.p0 = 0;
  a.in[1] = x.h[1];
  a.y[0] = b.h[0];
  a.out[0] = x.h[0];
  a.M[0] = op->Ainv(pi);
  a.beta = 0.5;
  return run_hop(pg, pv, a, false, EPI_AINV_ADD, st);
}

}  // namespace dd

// ---------------------------------------------------------------- handles
dd::Geom dd_lattice::geom() const {
  dd::Geom g;
  g.zblock = dims[1];
  g.t0 = 0;
  g.nt = dims[0];
  for (int i = 0; i < 4; ++i) g.n[i] = dims[i];
  g.stride[3] = 1;
  g.stride[2] = dims[3];
  g.stride[1] = dims[3] * dims[2];
  g.stride[0] = dims[3] * dims[2] * dims[1];
  g.Vh = (int)Vh;
  g.t_bc = (float)t_bc;
  return g;
}

const void* dd_gauge::U(int pi, int parity) const {
  if (!links[pi].ptr) return nullptr;
  const size_t elem = (pi == 0 || pi == 3) ? 16 : pi == 1 ? 8 : 4;
  return reinterpret_cast<const char*>(links[pi].ptr) + (size_t)parity * 36 * lat->Vh * elem;
}

const void* dd_gauge::U2(int parity) const {
  if (!links32r.ptr) return nullptr;
  return reinterpret_cast<const char*>(links32r.ptr) + (size_t)parity * recon_groups() * lat->Vh * sizeof(float4);
}

const void* dd_gauge::U2h(int parity) const {
  if (!links16r.ptr) return nullptr;
  return reinterpret_cast<const char*>(links16r.ptr) + (size_t)parity * 6 * lat->Vh * sizeof(uint4);
}

const void* dd_clover::M(int pi, int parity) const {
  if (!clov[pi].ptr) return nullptr;
  const size_t elem = (pi == 0 || pi == 3) ? 16 : pi == 1 ? 8 : 4;
  return reinterpret_cast<const char*>(clov[pi].ptr) + (size_t)parity * 36 * lat->Vh * elem;
}

const void* dd_clover::Ainv(int pi) const { return ainv[pi].ptr; }
