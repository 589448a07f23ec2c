// Host-side internals of the library: handle structures, error reporting and
// the operator layer that the C ABI, the solver and the batch path share.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dd_wilson.h"
#include "dd_device.cuh"

namespace dd {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
int fail(int status, const std::string& msg);
int cuda_fail(cudaError_t e, const char* where);

#define DD_CUDA(call)                                       \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return ::dd::cuda_fail(e_, #call); \
  } while (0)

#define DD_TRY(call)          \
  do {                        \
    int s_ = (call);          \
    if (s_ != DD_OK) return s_; \
  } while (0)

inline int prec_index(int prec) { return prec == P64 ? 0 : prec == P32 ? 1 : prec == P16 ? 2 : prec == PDF ? 3 : -1; }

// Device buffer owned by a handle.
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  int alloc(size_t n);
  int ensure(size_t n);  // grow-only
  void release();
};

// Copy streams and events of the pipelined host-buffer apply (created on
// first use, released with the handle).
struct HostPipe {
  cudaStream_t s_in = nullptr, s_out = nullptr;
  std::vector<cudaEvent_t> ev;
  HostPipe() = default;
  HostPipe(const HostPipe&) = delete;
  HostPipe& operator=(const HostPipe&) = delete;
  ~HostPipe();
  int ensure(int nevents);
};

}  // namespace dd

struct dd_lattice {
  int dims[4];
  int t_bc;
  int64_t V, Vh;
  dd::Geom geom() const;
};

struct dd_gauge {
  const dd_lattice* lat;
  unsigned prec_mask;
  // native links per precision (index 0: F64, 1: F32, 2: F16, 3: FP32
  // pairs): [parity][mu][9][Vh] complex elements, in 16-byte groups for F32 /
  // F16 (FP32 pairs: one float4 (re.h, re.l, im.h, im.l) per element)
  dd::DevBuf links[4];
  // when every link is SU(3): a second, compressed FP32 copy used by
  // single-RHS launches, either rows 0 and 1 only (recon32 = 12,
  // [parity][12 float4 groups][Vh]; the kernels rebuild row 2) or eight reals
  // per link (recon32 = 8, [parity][8 float4 groups][Vh], dd_link8.cuh)
  dd::DevBuf links32r;
  int recon32 = 0;
  int recon_groups() const { return recon32 == 8 ? 8 : 12; }  // float4 groups per site
  // the same for FP16: rows 0 and 1 only (recon16 = 12, [parity][6 uint4
  // groups][Vh], element 6 mu + e of a site in group (6 mu + e) / 4)
  dd::DevBuf links16r;
  int recon16 = 0;
  double su3_deviation = 0.0;  // max over links of |U U^H - 1| and |det U - 1|
  const void* U(int pi, int parity) const;
  const void* U2(int parity) const;   // the compressed FP32 copy
  const void* U2h(int parity) const;  // the two-row FP16 copy
};

struct dd_clover {
  const dd_gauge* gauge;
  const dd_lattice* lat;
  double m0, csw;
  unsigned prec_mask;
  // self-coupling blocks per precision: [parity][36][Vh] elements
  dd::DevBuf clov[4];
  // A_ee^{-1} per precision: [36][Vh] elements (even sites)
  dd::DevBuf ainv[4];
  // workspace for canonical-layout calls and operator intermediates
  dd::DevBuf ws_in, ws_out, ws_tmp, ws_canon_in, ws_canon_out;
  // residual workspace of dd_sap
  dd::DevBuf ws_sap;
  // FP32 link-derivative accumulator of dd_force: [V][4][20] floats
  dd::DevBuf ws_force;
  dd::HostPipe pipe;
  const void* M(int pi, int parity) const;  // A of a parity
  const void* Ainv(int pi) const;
};

namespace dd {

// A native field: two half fields (parity 0 and 1; a half-lattice field sets
// only one of them).
struct Field {
  HalfField h[2];
  int prec = 0;
  int nrhs = 1;
  int paired = 0;  // paired-RHS layout (dd_pair.cuh): FP32 / FP16, nrhs even
};

// Build a Field view of a native buffer.  subset: 0 full (even then odd),
// 1 odd sites only, 2 even sites only.
// paired = 1: the paired-RHS layout, which takes the same bytes.
Field field_view(const dd_lattice* lat, int prec, int subset, void* base, int nrhs, int paired = 0);
size_t field_bytes(const dd_lattice* lat, int prec, int subset, int nrhs);

// ---- operator layer (all enqueue on `st`) ----
// Precision of the operator handle to use (pg) and of the vectors (pv):
// (F64, F64), (F32, F32), (F16, F16) or (F16, F32).
int op_D(const dd_clover* op, int pg, int pv, bool dagger, const Field& in, const Field& out, cudaStream_t st);
// the same for the output sites of the time slices t0 .. t0 + nt - 1 only
int op_D_slices(const dd_clover* op, int pg, int pv, bool dagger, const Field& in, const Field& out, int t0, int nt,
                cudaStream_t st);
int op_SC(const dd_clover* op, int pg, int pv, const Field& in, const Field& out, cudaStream_t st);
// out_o = Dhat in_o (odd half fields); tmp_e: even half-field workspace
int op_Dhat(const dd_clover* op, int pg, int pv, bool dagger, const Field& in, const Field& out, const Field& tmp,
            cudaStream_t st);
// Whether op_Dhat_norm supports (pg, pv, nrhs): one RHS, FP32 vectors,
// FP32 or FP16 links and blocks.
bool dhat_norm_fused(int pg, int pv, int nrhs);
// op_Dhat that also writes norm_out[0] = (|out|^2, 0) from the second
// stencil launch (partials: hop_norm_blocks(Vh) complex doubles of scratch).
int op_Dhat_norm(const dd_clover* op, int pg, int pv, bool dagger, const Field& in, const Field& out, const Field& tmp,
                 double2* norm_out, double2* partials, int64_t npartials, cudaStream_t st);
// r = b - D x (full fields)
int op_residual(const dd_clover* op, int pg, int pv, const Field& b, const Field& x, const Field& r,
                cudaStream_t st);
// bhat_o = b_o - D_oe A_ee^{-1} b_e   (b full, bhat odd, tmp even)
int op_prepare(const dd_clover* op, int pg, int pv, const Field& b, const Field& bhat, const Field& tmp,
               cudaStream_t st);
// x_e = A_ee^{-1} (b_e - D_eo x_o)   (b full; x full with its odd half given)
int op_reconstruct(const dd_clover* op, int pg, int pv, const Field& b, const Field& x, cudaStream_t st);
// r_o = bhat_o - Dhat x_o (odd half fields; tmp: even half-field workspace)
int op_dhat_residual(const dd_clover* op, int pg, int pv, const Field& bhat, const Field& x, const Field& r,
                     const Field& tmp, cudaStream_t st);

// ---- setup kernels (dd_setup.cu) ----
int links_to_native(const dd_lattice* lat, const double* U_canon_dev, dd_gauge* g, cudaStream_t st);
// synthetic links exp(i eps H) from the counter-based generator, written to
// every native copy of g (dd_gauge_generate)
int links_generate(const dd_lattice* lat, uint64_t seed, double eps, dd_gauge* g, cudaStream_t st);
// max over links of max(|U U^H - 1|, |det U - 1|) from the FP64 copy (synchronises)
int links_su3_deviation(const dd_gauge* g, double* dev, cudaStream_t st);
// build the two-row FP32 copy: [parity][12 groups][Vh] float4
int links_to_recon32(dd_gauge* g, cudaStream_t st);
// eight-real FP32 copy; *dev = max |rebuilt - FP64 link| over all elements
int links_to_recon8(dd_gauge* g, double* dev, cudaStream_t st);
int links_to_recon16(dd_gauge* g, cudaStream_t st);
// the FP32-pair copy of the FP64 links (links[3])
int links_to_pairs(dd_gauge* g, cudaStream_t st);
int links_to_canonical(const dd_gauge* g, double* U_canon_dev, cudaStream_t st);
int clover_build(dd_clover* op, cudaStream_t st);  // FP64 blocks, A_ee^{-1}, demoted copies
int clover_to_dense(const dd_clover* op, double* A_dev /*[V][144] complex*/, cudaStream_t st);
// subset: 0 full; 1 odd / 2 even sites of a half-lattice canonical array
// [nrhs][V/2][12]; 3 even / 4 odd sites of a full canonical array [nrhs][V][12].
// nt > 0 (subset 0 only): only the time slices t0 .. t0 + nt - 1.
int pack(const dd_lattice* lat, int prec, int subset, const double* canon, const Field& f, cudaStream_t st,
         int t0 = 0, int nt = 0);
int unpack(const dd_lattice* lat, int prec, int subset, const Field& f, double* canon, cudaStream_t st, int t0 = 0,
           int nt = 0);
// Vector kernels of the CG preconditioner with FP16-stored vectors
// (dd_cg16.cu): npar = 1 (odd half) or 2 (full field); x32 FP32, the others
// FP16 native fields.
int cg16_convert(const Field& in32, const Field& out16, int64_t Vh, int npar, cudaStream_t st);
int cg16_norm(const Field& x16, int64_t Vh, int npar, double2* partials, double2* out, cudaStream_t st);
int cg16_r(const Field& r16, const Field& w16, int64_t Vh, int npar, const double2* g, const double2* n,
           cudaStream_t st);
int cg16_xp(const Field& x32, const Field& p16, const Field* z16, int64_t Vh, int npar, const double2* g,
            const double2* n, const double2* gn, cudaStream_t st);
// the same for complex64 canonical fields [N][V][12] (native layout only)
int pack_c64(const dd_lattice* lat, int prec, int subset, const float* canon, const Field& f, cudaStream_t st,
             int t0 = 0, int nt = 0);
int unpack_c64(const dd_lattice* lat, int prec, int subset, const Field& f, float* canon, cudaStream_t st,
               int t0 = 0, int nt = 0);

}  // namespace dd
