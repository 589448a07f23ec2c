// C ABI entry points (declared in include/dd_wilson.h).
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include "dd_blas.h"
#include "dd_internal.h"
#include "dd_ops.h"
#include "dd_sap.h"
#include "dd_amg.h"

namespace dd {
const char* last_error();
int solve(dd_clover* op, const dd_solve_params* prm, const double* b, double* x, int N, cudaStream_t st,
          dd_stats* stats);
int solve_schur(dd_clover* op, const dd_solve_params* prm, const double* b, double* x, int N, bool host,
                cudaStream_t st, dd_stats* stats);
int force(dd_clover* op, int prec, const double* phi, const double* psi, int nrhs, int with_clover, double* G,
          double* F, cudaStream_t st);
}  // namespace dd

using namespace dd;

namespace {

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

bool valid_prec(int p) { return p == DD_PREC_F64 || p == DD_PREC_F32 || p == DD_PREC_F16; }
// precisions of dd_apply, dd_pack, dd_unpack and dd_field_bytes
bool valid_apply_prec(int p) { return valid_prec(p) || p == DD_PREC_DF64; }

bool host_layout(int layout) { return layout == DD_LAYOUT_CANONICAL_HOST || layout == DD_LAYOUT_CANONICAL_HOST_C64; }
bool c64_layout(int layout) { return layout == DD_LAYOUT_CANONICAL_C64 || layout == DD_LAYOUT_CANONICAL_HOST_C64; }

// Copy a canonical field into device memory when it lives on the host.
int stage_in(DevBuf& buf, const void* src, size_t bytes, int layout, const double** dev, cudaStream_t st) {
  if (host_layout(layout)) {
    DD_TRY(buf.ensure(bytes));
    DD_CUDA(cudaMemcpyAsync(buf.ptr, src, bytes, cudaMemcpyHostToDevice, st));
    *dev = reinterpret_cast<const double*>(buf.ptr);
  } else {
    *dev = reinterpret_cast<const double*>(src);
  }
  return DD_OK;
}

// D or D^H of a full field in canonical host layout, pipelined over C <= 24
// chunks of time slices: the host-to-device copy of chunk c + 1 (stream
// s_in), the pack / stencil / unpack of chunk c (the caller's stream) and the
// device-to-host copy of chunk c - 1 (stream s_out) overlap.  The stencil of
// a chunk needs the input slices one beyond each end, so the last chunk is
// copied first and chunk c is computed once chunk c + 1 is packed.
int apply_host_pipelined(dd_clover* op, int prec, bool dagger, const void* hin, void* hout, int nrhs,
                         cudaStream_t st, bool c64) {
  const size_t esz = c64 ? 8 : 16;  // bytes per canonical complex element
  const dd_lattice* lat = op->lat;
  const int nT = lat->dims[0];
  static const int max_chunks = [] {
    const char* e = getenv("DD_HOST_CHUNKS");  // tuning override
    const int v = e ? atoi(e) : 48;
    return v < 2 ? 2 : v;
  }();
  const int C = nT < max_chunks ? nT : max_chunks;
  const int64_t slice = (int64_t)lat->dims[1] * lat->dims[2] * lat->dims[3];
  const size_t row = (size_t)lat->V * 12 * esz;  // one RHS of the canonical array
  const size_t cb = row * nrhs;
  const size_t nb = field_bytes(lat, prec, 0, nrhs);
  DD_TRY(op->ws_canon_in.ensure(cb));
  DD_TRY(op->ws_canon_out.ensure(cb));
  DD_TRY(op->ws_in.ensure(nb));
  DD_TRY(op->ws_out.ensure(nb));
  DD_TRY(op->pipe.ensure(2 * C + 1));
  HostPipe& hp = op->pipe;
  cudaEvent_t start = hp.ev[2 * C];
  auto t0_of = [&](int c) { return (int)((int64_t)c * nT / C); };
  auto copy_rows = [&](void* dst, const void* src, int c, cudaMemcpyKind kind, cudaStream_t s) -> cudaError_t {
    const size_t off = (size_t)t0_of(c) * slice * 12 * esz;
    const size_t w = (size_t)(t0_of(c + 1) - t0_of(c)) * slice * 12 * esz;
    return cudaMemcpy2DAsync(static_cast<char*>(dst) + off, row, static_cast<const char*>(src) + off, row, w, nrhs,
                             kind, s);
  };
  const double* cin = reinterpret_cast<const double*>(op->ws_canon_in.ptr);
  double* cout = reinterpret_cast<double*>(op->ws_canon_out.ptr);
  Field fin = field_view(lat, prec, 0, op->ws_in.ptr, nrhs);
  Field fout = field_view(lat, prec, 0, op->ws_out.ptr, nrhs);
  // the copy streams start after the work already queued on st
  DD_CUDA(cudaEventRecord(start, st));
  DD_CUDA(cudaStreamWaitEvent(hp.s_in, start, 0));
  DD_CUDA(cudaStreamWaitEvent(hp.s_out, start, 0));
  for (int k = 0; k < C; ++k) {
    const int c = k == 0 ? C - 1 : k - 1;  // last chunk first
    DD_CUDA(copy_rows(op->ws_canon_in.ptr, hin, c, cudaMemcpyHostToDevice, hp.s_in));
    DD_CUDA(cudaEventRecord(hp.ev[c], hp.s_in));
  }
  auto pack_chunk = [&](int c) -> int {
    DD_CUDA(cudaStreamWaitEvent(st, hp.ev[c], 0));
    if (c64)
      return pack_c64(lat, prec, 0, reinterpret_cast<const float*>(cin), fin, st, t0_of(c), t0_of(c + 1) - t0_of(c));
    return pack(lat, prec, 0, cin, fin, st, t0_of(c), t0_of(c + 1) - t0_of(c));
  };
  auto compute_chunk = [&](int c) -> int {
    const int t0 = t0_of(c), nt = t0_of(c + 1) - t0;
    DD_TRY(op_D_slices(op, prec, prec, dagger, fin, fout, t0, nt, st));
    if (c64)
      DD_TRY(unpack_c64(lat, prec, 0, fout, reinterpret_cast<float*>(cout), st, t0, nt));
    else
      DD_TRY(unpack(lat, prec, 0, fout, cout, st, t0, nt));
    DD_CUDA(cudaEventRecord(hp.ev[C + c], st));
    DD_CUDA(cudaStreamWaitEvent(hp.s_out, hp.ev[C + c], 0));
    DD_CUDA(copy_rows(hout, cout, c, cudaMemcpyDeviceToHost, hp.s_out));
    return DD_OK;
  };
  DD_TRY(pack_chunk(C - 1));
  for (int c = 0; c < C - 1; ++c) {
    DD_TRY(pack_chunk(c));
    if (c >= 1) DD_TRY(compute_chunk(c - 1));
  }
  if (C >= 2) DD_TRY(compute_chunk(C - 2));
  DD_TRY(compute_chunk(C - 1));
  DD_CUDA(cudaStreamSynchronize(hp.s_out));
  DD_CUDA(cudaStreamSynchronize(st));
  return DD_OK;
}

}  // namespace

dd::HostPipe::~HostPipe() {
  for (cudaEvent_t e : ev) cudaEventDestroy(e);
  if (s_in) cudaStreamDestroy(s_in);
  if (s_out) cudaStreamDestroy(s_out);
}

int dd::HostPipe::ensure(int nevents) {
  if (!s_in) DD_CUDA(cudaStreamCreateWithFlags(&s_in, cudaStreamNonBlocking));
  if (!s_out) DD_CUDA(cudaStreamCreateWithFlags(&s_out, cudaStreamNonBlocking));
  while ((int)ev.size() < nevents) {
    cudaEvent_t e;
    DD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ev.push_back(e);
  }
  return DD_OK;
}

extern "C" {

const char* dd_error_string(int status) {
  switch (status) {
    case DD_OK: return "DD_OK";
    case DD_ERR_ARG: return "DD_ERR_ARG";
    case DD_ERR_OOM: return "DD_ERR_OOM";
    case DD_ERR_CUDA: return "DD_ERR_CUDA";
    case DD_ERR_SINGULAR: return "DD_ERR_SINGULAR";
    case DD_ERR_NOT_CONVERGED: return "DD_ERR_NOT_CONVERGED";
    case DD_ERR_TIMEOUT: return "DD_ERR_TIMEOUT";
    case DD_ERR_UNSUPPORTED: return "DD_ERR_UNSUPPORTED";
    default: return "unknown status";
  }
}

const char* dd_last_error_detail(void) { return last_error(); }

int dd_version(void) { return 100; }

int dd_device_status(int* flags_out) {
  if (!flags_out) return fail(DD_ERR_ARG, "null flags_out");
  int* flag = device_error_flag();
  if (!flag) return fail(DD_ERR_CUDA, "device status flag unavailable");
  DD_CUDA(cudaDeviceSynchronize());
  DD_CUDA(cudaMemcpy(flags_out, flag, sizeof(int), cudaMemcpyDeviceToHost));
  DD_CUDA(cudaMemset(flag, 0, sizeof(int)));
  return DD_OK;
}

int dd_lattice_create(const int dims[4], int t_bc, dd_lattice** out) {
  if (!dims || !out) return fail(DD_ERR_ARG, "null argument");
  int64_t V = 1;
  for (int i = 0; i < 4; ++i) {
    if (dims[i] < 2 || dims[i] % 2) return fail(DD_ERR_ARG, "every lattice extent must be even and >= 2");
    V *= dims[i];
  }
  if (V >= (int64_t(1) << 31)) return fail(DD_ERR_ARG, "lattice volume must be below 2^31");
  if (t_bc != 1 && t_bc != -1) return fail(DD_ERR_ARG, "t_bc must be +1 or -1");
  dd_lattice* l = new (std::nothrow) dd_lattice;
  if (!l) return fail(DD_ERR_OOM, "host allocation failed");
  for (int i = 0; i < 4; ++i) l->dims[i] = dims[i];
  l->t_bc = t_bc;
  l->V = V;
  l->Vh = V / 2;
  *out = l;
  return DD_OK;
}

int dd_lattice_destroy(dd_lattice* lat) {
  delete lat;
  return DD_OK;
}

int64_t dd_lattice_volume(const dd_lattice* lat) { return lat ? lat->V : 0; }

namespace {

// A gauge handle with the native link buffers of prec_mask (FP64 always).
int gauge_alloc(const dd_lattice* lat, unsigned prec_mask, dd_gauge** out) {
  dd_gauge* g = new (std::nothrow) dd_gauge;
  if (!g) return fail(DD_ERR_OOM, "host allocation failed");
  g->lat = lat;
  g->prec_mask = prec_mask | DD_PREC_F64;
  const int64_t nel = lat->V * 4 * 9;
  int s = g->links[0].alloc(nel * 16);
  if (s == DD_OK && (g->prec_mask & DD_PREC_F32)) s = g->links[1].alloc(nel * 8);
  if (s == DD_OK && (g->prec_mask & DD_PREC_F16)) s = g->links[2].alloc(nel * 4);
  if (s != DD_OK) {
    delete g;
    return s;
  }
  *out = g;
  return DD_OK;
}

constexpr double kSu3Tol = 1e-6;    // links taken as SU(3) (max |U U^H - 1|, |det U - 1|)
constexpr double kLink8Tol = 1e-6;  // largest element error of the eight-real copy

// The compressed copy of precision `prec` with `reals` per link (FP32: 18
// none, 12 two rows, 8 eight reals; FP16: 18, 12); on DD_ERR_UNSUPPORTED the
// previous form is kept.
int compress_links(dd_gauge* g, int prec, int reals) {
  if (prec == DD_PREC_F16) {
    if (reals == 18) {
      g->links16r.release();
      g->recon16 = 0;
      return DD_OK;
    }
    if (reals != 12) return fail(DD_ERR_UNSUPPORTED, "FP16 links take 18 or 12 reals");
    if (!(g->prec_mask & DD_PREC_F16)) return fail(DD_ERR_UNSUPPORTED, "no FP16 links in the gauge handle");
    if (!(g->su3_deviation < kSu3Tol)) return fail(DD_ERR_UNSUPPORTED, "links are not SU(3) to 1e-6");
    return links_to_recon16(g, 0);
  }
  if (reals == 18) {
    g->links32r.release();
    g->recon32 = 0;
    return DD_OK;
  }
  if (!(g->prec_mask & DD_PREC_F32)) return fail(DD_ERR_UNSUPPORTED, "no FP32 links in the gauge handle");
  if (!(g->su3_deviation < kSu3Tol)) return fail(DD_ERR_UNSUPPORTED, "links are not SU(3) to 1e-6");
  if (reals == 12) return links_to_recon32(g, 0);
  const int before = g->recon32;
  double dev = 0.0;
  DD_TRY(links_to_recon8(g, &dev, 0));
  if (dev <= kLink8Tol) return DD_OK;
  const int s = before == 12 ? links_to_recon32(g, 0) : compress_links(g, prec, 18);
  if (s != DD_OK) return s;
  return fail(DD_ERR_UNSUPPORTED, "eight-real links rebuild to " + std::to_string(dev) + " > 1e-6");
}

// After the links are in place: SU(3) check, the compressed FP32 and FP16
// copies when every link is SU(3) to FP32 accuracy (DD_RECON: 12 rows 0 and
// 1, the default; 8 eight reals for FP32, else two rows; 0 none), and a
// device synchronisation.
int gauge_finish(dd_gauge* g) {
  int s = links_su3_deviation(g, &g->su3_deviation, 0);
  const char* e = getenv("DD_RECON");
  const int want = e ? atoi(e) : 12;
  if (s == DD_OK && want != 0 && g->su3_deviation < kSu3Tol) {
    if (g->prec_mask & DD_PREC_F32) {
      if (want == 8) {
        s = compress_links(g, DD_PREC_F32, 8);
        if (s == DD_ERR_UNSUPPORTED) s = compress_links(g, DD_PREC_F32, 12);
      } else {
        s = compress_links(g, DD_PREC_F32, 12);
      }
    }
    if (s == DD_OK && (g->prec_mask & DD_PREC_F16)) s = compress_links(g, DD_PREC_F16, 12);
  }
  if (s == DD_OK && (g->prec_mask & DD_PREC_DF64)) s = links_to_pairs(g, 0);
  if (s == DD_OK && cudaDeviceSynchronize() != cudaSuccess) s = cuda_fail(cudaGetLastError(), "link conversion");
  return s;
}

}  // namespace

int dd_gauge_create(const dd_lattice* lat, const double* U, int location, unsigned prec_mask, dd_gauge** out) {
  if (!lat || !U || !out) return fail(DD_ERR_ARG, "null argument");
  if (location != 0 && location != 1) return fail(DD_ERR_ARG, "location must be 0 (host) or 1 (device)");
  if (prec_mask & ~15u) return fail(DD_ERR_ARG, "bad precision mask");
  dd_gauge* g = nullptr;
  DD_TRY(gauge_alloc(lat, prec_mask, &g));
  const size_t bytes = (size_t)lat->V * 4 * 9 * 16;
  int s = DD_OK;
  DevBuf staging;
  const double* Ud = U;
  if (location == 0) {
    s = staging.alloc(bytes);
    if (s == DD_OK && cudaMemcpy(staging.ptr, U, bytes, cudaMemcpyHostToDevice) != cudaSuccess)
      s = cuda_fail(cudaGetLastError(), "cudaMemcpy of the links");
    Ud = reinterpret_cast<const double*>(staging.ptr);
  }
  if (s == DD_OK) s = links_to_native(lat, Ud, g, 0);
  if (s == DD_OK) s = gauge_finish(g);
  if (s != DD_OK) {
    delete g;
    return s;
  }
  *out = g;
  return DD_OK;
}

int dd_gauge_generate(const dd_lattice* lat, uint64_t seed, double eps, unsigned prec_mask, dd_gauge** out) {
  if (!lat || !out) return fail(DD_ERR_ARG, "null argument");
  if (prec_mask & ~15u) return fail(DD_ERR_ARG, "bad precision mask");
  if (!(eps >= 0.0 && eps <= 1e6)) return fail(DD_ERR_ARG, "eps must be finite and >= 0");
  dd_gauge* g = nullptr;
  DD_TRY(gauge_alloc(lat, prec_mask, &g));
  int s = links_generate(lat, seed, eps, g, 0);
  if (s == DD_OK) s = gauge_finish(g);
  if (s != DD_OK) {
    delete g;
    return s;
  }
  *out = g;
  return DD_OK;
}

int dd_gauge_stored_rows(const dd_gauge* g, int prec) {
  if (!g) return fail(DD_ERR_ARG, "null gauge");
  if (!valid_apply_prec(prec)) return fail(DD_ERR_ARG, "bad precision");
  if (!(g->prec_mask & (unsigned)prec)) return fail(DD_ERR_UNSUPPORTED, "precision not created in the gauge handle");
  return (prec == DD_PREC_F32 && g->recon32 == 12) || (prec == DD_PREC_F16 && g->recon16) ? 2 : 3;
}

int dd_gauge_link_reals(const dd_gauge* g, int prec) {
  if (!g) return fail(DD_ERR_ARG, "null gauge");
  if (!valid_apply_prec(prec)) return fail(DD_ERR_ARG, "bad precision");
  if (!(g->prec_mask & (unsigned)prec)) return fail(DD_ERR_UNSUPPORTED, "precision not created in the gauge handle");
  if (prec == DD_PREC_F32 && g->recon32) return g->recon32;
  return prec == DD_PREC_F16 && g->recon16 ? 12 : 18;
}

int dd_gauge_compress_links(dd_gauge* g, int prec, int reals) {
  if (!g) return fail(DD_ERR_ARG, "null gauge");
  if (prec != DD_PREC_F32 && prec != DD_PREC_F16) return fail(DD_ERR_ARG, "precision must be F32 or F16");
  if (reals != 18 && reals != 12 && reals != 8) return fail(DD_ERR_ARG, "reals per link must be 18, 12 or 8");
  if (cudaDeviceSynchronize() != cudaSuccess) return cuda_fail(cudaGetLastError(), "before link compression");
  int s = compress_links(g, prec, reals);
  if (cudaDeviceSynchronize() != cudaSuccess && s == DD_OK) s = cuda_fail(cudaGetLastError(), "link compression");
  return s;
}

int dd_gauge_destroy(dd_gauge* g) {
  delete g;
  return DD_OK;
}

int dd_gauge_download(const dd_gauge* g, double* U, int location) {
  if (!g || !U) return fail(DD_ERR_ARG, "null argument");
  const size_t bytes = (size_t)g->lat->V * 4 * 9 * 16;
  if (location == 1) {
    DD_TRY(links_to_canonical(g, U, 0));
    DD_CUDA(cudaDeviceSynchronize());
    return DD_OK;
  }
  DevBuf tmp;
  DD_TRY(tmp.alloc(bytes));
  DD_TRY(links_to_canonical(g, reinterpret_cast<double*>(tmp.ptr), 0));
  DD_CUDA(cudaMemcpy(U, tmp.ptr, bytes, cudaMemcpyDeviceToHost));
  return DD_OK;
}

int dd_clover_create(const dd_gauge* g, double m0, double csw, unsigned prec_mask, dd_clover** out) {
  if (!g || !out) return fail(DD_ERR_ARG, "null argument");
  if (prec_mask & ~15u) return fail(DD_ERR_ARG, "bad precision mask");
  dd_clover* op = new (std::nothrow) dd_clover;
  if (!op) return fail(DD_ERR_OOM, "host allocation failed");
  op->gauge = g;
  op->lat = g->lat;
  op->m0 = m0;
  op->csw = csw;
  op->prec_mask = (prec_mask | DD_PREC_F64) & g->prec_mask;
  int s = clover_build(op, 0);
  if (s == DD_OK && cudaDeviceSynchronize() != cudaSuccess) s = cuda_fail(cudaGetLastError(), "clover build");
  if (s != DD_OK) {
    delete op;
    return s;
  }
  *out = op;
  return DD_OK;
}

int dd_clover_destroy(dd_clover* op) {
  delete op;
  return DD_OK;
}

int dd_clover_download(const dd_clover* op, double* A_host) {
  if (!op || !A_host) return fail(DD_ERR_ARG, "null argument");
  const size_t bytes = (size_t)op->lat->V * 144 * 16;
  DevBuf tmp;
  DD_TRY(tmp.alloc(bytes));
  DD_TRY(clover_to_dense(op, reinterpret_cast<double*>(tmp.ptr), 0));
  DD_CUDA(cudaMemcpy(A_host, tmp.ptr, bytes, cudaMemcpyDeviceToHost));
  return DD_OK;
}

size_t dd_field_bytes(const dd_clover* op, int prec, int subset, int nrhs) {
  if (!op || !valid_apply_prec(prec) || nrhs < 1 || (subset != 0 && subset != 1)) return 0;
  return field_bytes(op->lat, prec, subset, nrhs);
}

int dd_pack(const dd_clover* op, int prec, int subset, const double* canon, void* native, int nrhs, void* stream) {
  if (!op || !canon || !native || nrhs < 1) return fail(DD_ERR_ARG, "null argument or nrhs < 1");
  if (!valid_apply_prec(prec) || subset < 0 || subset > 2) return fail(DD_ERR_ARG, "bad precision or subset");
  Field f = field_view(op->lat, prec, subset, native, nrhs);
  return pack(op->lat, prec, subset, canon, f, as_stream(stream));
}

int dd_unpack(const dd_clover* op, int prec, int subset, const void* native, double* canon, int nrhs, void* stream) {
  if (!op || !canon || !native || nrhs < 1) return fail(DD_ERR_ARG, "null argument or nrhs < 1");
  if (!valid_apply_prec(prec) || subset < 0 || subset > 2) return fail(DD_ERR_ARG, "bad precision or subset");
  Field f = field_view(op->lat, prec, subset, const_cast<void*>(native), nrhs);
  return unpack(op->lat, prec, subset, f, canon, as_stream(stream));
}

int dd_pack_paired(const dd_clover* op, int prec, int subset, const double* canon, void* paired, int nrhs,
                   void* stream) {
  if (!op || !canon || !paired || nrhs < 2 || nrhs % 2 != 0)
    return fail(DD_ERR_ARG, "null argument or nrhs not even and >= 2");
  if ((prec != DD_PREC_F32 && prec != DD_PREC_F16) || subset < 0 || subset > 2)
    return fail(DD_ERR_ARG, "paired layout: precision F32 or F16, subset 0..2");
  Field f = field_view(op->lat, prec, subset, paired, nrhs, 1);
  return pack(op->lat, prec, subset, canon, f, as_stream(stream));
}

int dd_unpack_paired(const dd_clover* op, int prec, int subset, const void* paired, double* canon, int nrhs,
                     void* stream) {
  if (!op || !canon || !paired || nrhs < 2 || nrhs % 2 != 0)
    return fail(DD_ERR_ARG, "null argument or nrhs not even and >= 2");
  if ((prec != DD_PREC_F32 && prec != DD_PREC_F16) || subset < 0 || subset > 2)
    return fail(DD_ERR_ARG, "paired layout: precision F32 or F16, subset 0..2");
  Field f = field_view(op->lat, prec, subset, const_cast<void*>(paired), nrhs, 1);
  return unpack(op->lat, prec, subset, f, canon, as_stream(stream));
}

int dd_apply(dd_clover* op, int which, int prec, const void* in, void* out, int nrhs, int layout, void* stream) {
  if (!op || !in || !out || nrhs < 1) return fail(DD_ERR_ARG, "null argument or nrhs < 1");
  if (!valid_apply_prec(prec)) return fail(DD_ERR_ARG, "bad precision");
  if (which < DD_OP_D || which > DD_OP_SC) return fail(DD_ERR_ARG, "bad operator");
  if (layout < DD_LAYOUT_CANONICAL || layout > DD_LAYOUT_CANONICAL_HOST_C64) return fail(DD_ERR_ARG, "bad layout");
  if (layout == DD_LAYOUT_NATIVE_PAIRED) {
    if (nrhs % 2 != 0 || (prec != DD_PREC_F32 && prec != DD_PREC_F16))
      return fail(DD_ERR_ARG, "paired layout: precision F32 or F16 and an even nrhs");
    if (which == DD_OP_SC) return fail(DD_ERR_UNSUPPORTED, "paired layout: D, D^H, Dhat and Dhat^H only");
  }
  const int pi = prec_index(prec);
  if (!op->gauge->links[pi].ptr || !op->clov[pi].ptr)
    return fail(DD_ERR_UNSUPPORTED, "precision not created in the gauge/operator handles");
  cudaStream_t st = as_stream(stream);
  const dd_lattice* lat = op->lat;
  const bool half = which == DD_OP_DHAT || which == DD_OP_DHAT_H;
  const int subset = half ? 1 : 0;
  const size_t nb = field_bytes(lat, prec, subset, nrhs);
  const bool c64 = c64_layout(layout);
  const size_t cb = (size_t)(half ? lat->Vh : lat->V) * 12 * (c64 ? 8 : 16) * nrhs;
  if (host_layout(layout) && (which == DD_OP_D || which == DD_OP_DH))
    return apply_host_pipelined(op, prec, which == DD_OP_DH, in, out, nrhs, st, c64);
  Field fin, fout;
  const double* cin = nullptr;
  // canonical fields with an even RHS count go through the paired-RHS stencil
  // (FP32: bit-identical to the RHS-blocked one; FP16: half2 colour products;
  // DD_RHS_BLOCK=1 keeps one thread per site and RHS, DD_STAGE=1 the
  // row-staged stencil)
  const int paired = layout == DD_LAYOUT_NATIVE_PAIRED ||
                     (layout != DD_LAYOUT_NATIVE && !c64 && nrhs % 2 == 0 && which != DD_OP_SC &&
                      (prec == DD_PREC_F32 || prec == DD_PREC_F16) && rhs_block_limit() >= 2 && !stage_opted_in());
  if (layout == DD_LAYOUT_NATIVE || layout == DD_LAYOUT_NATIVE_PAIRED) {
    fin = field_view(lat, prec, subset, const_cast<void*>(in), nrhs, paired);
    fout = field_view(lat, prec, subset, out, nrhs, paired);
  } else {
    DD_TRY(stage_in(op->ws_canon_in, in, cb, layout, &cin, st));
    DD_TRY(op->ws_in.ensure(nb));
    DD_TRY(op->ws_out.ensure(nb));
    fin = field_view(lat, prec, subset, op->ws_in.ptr, nrhs, paired);
    fout = field_view(lat, prec, subset, op->ws_out.ptr, nrhs, paired);
    if (c64)
      DD_TRY(pack_c64(lat, prec, subset, reinterpret_cast<const float*>(cin), fin, st));
    else
      DD_TRY(pack(lat, prec, subset, cin, fin, st));
  }
  switch (which) {
    case DD_OP_D:
    case DD_OP_DH:
      DD_TRY(op_D(op, prec, prec, which == DD_OP_DH, fin, fout, st));
      break;
    case DD_OP_SC:
      DD_TRY(op_SC(op, prec, prec, fin, fout, st));
      break;
    default: {
      DD_TRY(op->ws_tmp.ensure(field_bytes(lat, prec, 2, nrhs)));
      Field tmp = field_view(lat, prec, 2, op->ws_tmp.ptr, nrhs, paired);
      DD_TRY(op_Dhat(op, prec, prec, which == DD_OP_DHAT_H, fin, fout, tmp, st));
    }
  }
  if (layout != DD_LAYOUT_NATIVE && layout != DD_LAYOUT_NATIVE_PAIRED) {
    double* cout = reinterpret_cast<double*>(out);
    if (host_layout(layout)) {
      DD_TRY(op->ws_canon_out.ensure(cb));
      cout = reinterpret_cast<double*>(op->ws_canon_out.ptr);
    }
    if (c64)
      DD_TRY(unpack_c64(lat, prec, subset, fout, reinterpret_cast<float*>(cout), st));
    else
      DD_TRY(unpack(lat, prec, subset, fout, cout, st));
    if (host_layout(layout)) {
      DD_CUDA(cudaMemcpyAsync(out, cout, cb, cudaMemcpyDeviceToHost, st));
      DD_CUDA(cudaStreamSynchronize(st));
    }
  }
  DD_CUDA(cudaGetLastError());
  return DD_OK;
}

void dd_solve_params_default(dd_solve_params* p) {
  if (!p) return;
  p->tol = 1e-10;
  p->restart = 30;
  p->max_restarts = 100;
  p->max_outer = 30;
  p->inner_prec = DD_PREC_F32;
  p->inner_tol = 1e-6;
  p->even_odd = 1;
  p->verbose = 0;
  p->precond = DD_PRECOND_NONE;
  p->gs_passes = 1;
  p->rhs_batch = 0;
  p->precond_iters = 32;
  for (int mu = 0; mu < 4; ++mu) p->sap_block[mu] = 4;
  p->sap_cycles = 1;
  p->sap_mr_steps = 4;
  p->amg = nullptr;
  p->refine_prec = DD_PREC_F64;
}

int dd_solve(dd_clover* op, const dd_solve_params* params, const void* b, void* x, int nrhs, int layout,
             void* stream, dd_stats* stats) {
  if (!op || !params || !b || !x || nrhs < 1) return fail(DD_ERR_ARG, "null argument or nrhs < 1");
  if (layout != DD_LAYOUT_CANONICAL && layout != DD_LAYOUT_CANONICAL_HOST)
    return fail(DD_ERR_ARG, "dd_solve takes canonical fields");
  if (params->precond < DD_PRECOND_NONE || params->precond > DD_PRECOND_CGNR16)
    return fail(DD_ERR_ARG, "unknown preconditioner");
  if (params->precond == DD_PRECOND_CGNR16 && params->inner_prec != DD_PREC_F16 && params->inner_prec != DD_PREC_F32)
    return fail(DD_ERR_UNSUPPORTED, "DD_PRECOND_CGNR16 takes inner precision F16 or F32");
  if (!valid_apply_prec(params->inner_prec)) return fail(DD_ERR_ARG, "bad inner precision");
  if (params->inner_prec == DD_PREC_DF64 && (params->precond == DD_PRECOND_SAP || params->precond == DD_PRECOND_AMG))
    return fail(DD_ERR_UNSUPPORTED, "SAP and AMG take inner precision F64, F32 or F16");
  if (params->precond == DD_PRECOND_AMG) {
    if (!params->amg || amg_operator(params->amg) != op)
      return fail(DD_ERR_ARG, "DD_PRECOND_AMG needs an AMG handle of this operator");
    if (amg_fine_precision(params->amg) != (params->inner_prec == DD_PREC_F64 ? P64 : P32))
      return fail(DD_ERR_ARG, "AMG fine precision differs from the inner vector precision");
  }
  if (params->precond == DD_PRECOND_SAP) {
    DD_TRY(sap_check_blocks(op->lat, params->sap_block, params->inner_prec == DD_PREC_F64 ? P64 : P32));
    if (params->sap_cycles < 1 || params->sap_mr_steps < 1) return fail(DD_ERR_ARG, "SAP cycles and MR steps >= 1");
  }
  if ((params->precond == DD_PRECOND_CGNR || params->precond == DD_PRECOND_CGNR16) && params->precond_iters < 1)
    return fail(DD_ERR_ARG, "precond_iters must be >= 1");
  if (!(params->tol > 0) || params->max_restarts < 1 || params->max_outer < 0)
    return fail(DD_ERR_ARG, "bad solver parameters");
  if (params->rhs_batch < 0) return fail(DD_ERR_ARG, "rhs_batch must be >= 0");
  if (params->refine_prec != DD_PREC_F64 && params->refine_prec != DD_PREC_DF64)
    return fail(DD_ERR_ARG, "refine_prec: DD_PREC_F64 or DD_PREC_DF64");
  if (params->refine_prec == DD_PREC_DF64 &&
      (!op->gauge->links[prec_index(PDF)].ptr || !op->clov[prec_index(PDF)].ptr))
    return fail(DD_ERR_UNSUPPORTED, "refine_prec DD_PREC_DF64: no FP32-pair copies in the gauge/operator handles");
  cudaStream_t st = as_stream(stream);
  if (params->even_odd)
    return solve_schur(op, params, (const double*)b, (double*)x, nrhs, layout == DD_LAYOUT_CANONICAL_HOST, st, stats);
  const size_t cb = (size_t)op->lat->V * 12 * 16 * nrhs;
  if (layout == DD_LAYOUT_CANONICAL) return solve(op, params, (const double*)b, (double*)x, nrhs, st, stats);
  DevBuf bd, xd;
  DD_TRY(bd.alloc(cb));
  DD_TRY(xd.alloc(cb));
  DD_CUDA(cudaMemcpyAsync(bd.ptr, b, cb, cudaMemcpyHostToDevice, st));
  DD_CUDA(cudaMemcpyAsync(xd.ptr, x, cb, cudaMemcpyHostToDevice, st));
  int s = solve(op, params, (const double*)bd.ptr, (double*)xd.ptr, nrhs, st, stats);
  if (s == DD_OK || s == DD_ERR_NOT_CONVERGED) {
    DD_CUDA(cudaMemcpyAsync(x, xd.ptr, cb, cudaMemcpyDeviceToHost, st));
    DD_CUDA(cudaStreamSynchronize(st));
  }
  return s;
}

int dd_sap(dd_clover* op, int prec, const int block[4], int cycles, int mr_steps, const void* v, void* z, int nrhs,
           int layout, void* stream) {
  if (!op || !block || !v || !z || nrhs < 1) return fail(DD_ERR_ARG, "null argument or nrhs < 1");
  if (!valid_prec(prec)) return fail(DD_ERR_ARG, "bad precision");
  if (layout < DD_LAYOUT_CANONICAL || layout > DD_LAYOUT_NATIVE) return fail(DD_ERR_ARG, "bad layout");
  if (layout == DD_LAYOUT_NATIVE && prec == DD_PREC_F16)
    return fail(DD_ERR_ARG, "SAP: DD_PREC_F16 (FP32 vectors) takes canonical layouts");
  if (cycles < 1 || mr_steps < 1) return fail(DD_ERR_ARG, "SAP: cycles and MR steps must be >= 1");
  const int pg = prec, pv = prec == DD_PREC_F64 ? P64 : P32;
  const dd_lattice* lat = op->lat;
  DD_TRY(sap_check_blocks(lat, block, pv));
  const int pi = prec_index(pg);
  if (!op->gauge->links[pi].ptr || !op->clov[pi].ptr)
    return fail(DD_ERR_UNSUPPORTED, "precision not created in the gauge/operator handles");
  cudaStream_t st = as_stream(stream);
  const size_t nb = field_bytes(lat, pv, 0, nrhs);
  const size_t cb = (size_t)lat->V * 12 * 16 * nrhs;
  DD_TRY(op->ws_sap.ensure(nb));
  Field R = field_view(lat, pv, 0, op->ws_sap.ptr, nrhs);
  if (layout == DD_LAYOUT_NATIVE) {
    Field Vf = field_view(lat, pv, 0, const_cast<void*>(v), nrhs), Zf = field_view(lat, pv, 0, z, nrhs);
    return sap_apply(op, pg, pv, block, cycles, mr_steps, Vf, Zf, R, st);
  }
  const double* cin = nullptr;
  DD_TRY(stage_in(op->ws_canon_in, v, cb, layout, &cin, st));
  DD_TRY(op->ws_in.ensure(nb));
  DD_TRY(op->ws_out.ensure(nb));
  Field Vf = field_view(lat, pv, 0, op->ws_in.ptr, nrhs), Zf = field_view(lat, pv, 0, op->ws_out.ptr, nrhs);
  DD_TRY(pack(lat, pv, 0, cin, Vf, st));
  DD_TRY(sap_apply(op, pg, pv, block, cycles, mr_steps, Vf, Zf, R, st));
  double* cout = reinterpret_cast<double*>(z);
  if (layout == DD_LAYOUT_CANONICAL_HOST) {
    DD_TRY(op->ws_canon_out.ensure(cb));
    cout = reinterpret_cast<double*>(op->ws_canon_out.ptr);
  }
  DD_TRY(unpack(lat, pv, 0, Zf, cout, st));
  if (layout == DD_LAYOUT_CANONICAL_HOST) {
    DD_CUDA(cudaMemcpyAsync(z, cout, cb, cudaMemcpyDeviceToHost, st));
    DD_CUDA(cudaStreamSynchronize(st));
  }
  return DD_OK;
}

int dd_force(dd_clover* op, int prec, const double* phi, const double* psi, int nrhs, int with_clover, double* G,
             double* F, void* stream) {
  if (!op || !phi || !psi || nrhs < 1 || (!G && !F)) return fail(DD_ERR_ARG, "null argument or nrhs < 1");
  if (prec != DD_PREC_F64 && prec != DD_PREC_F32) return fail(DD_ERR_ARG, "force precision must be F64 or F32");
  return force(op, prec, phi, psi, nrhs, with_clover, G, F, as_stream(stream));
}

int dd_dot(const double* a, const double* b, int64_t nsites, int nrhs, double* dots_host, void* stream) {
  if (!a || !b || !dots_host || nsites < 1 || nrhs < 1) return fail(DD_ERR_ARG, "null argument or empty field");
  cudaStream_t st = as_stream(stream);
  // canonical [nrhs][nsites][12] complex: per-RHS contiguous blocks
  DevBuf partials, out;
  DD_TRY(partials.alloc((size_t)blas_partials_len(1) * sizeof(double2)));
  DD_TRY(out.alloc((size_t)nrhs * sizeof(double2)));
  const int64_t L = nsites * 12;
  for (int r = 0; r < nrhs; ++r) {
    VecList vs;
    vs.p[0] = a + 2 * r * L;
    DD_TRY(blas_multidot<P64>(vs, 1, b + 2 * r * L, L, 1, (double2*)out.ptr + r, 0, (double2*)partials.ptr, st));
  }
  DD_CUDA(cudaMemcpyAsync(dots_host, out.ptr, (size_t)nrhs * sizeof(double2), cudaMemcpyDeviceToHost, st));
  DD_CUDA(cudaStreamSynchronize(st));
  return DD_OK;
}

}  // extern "C"
