// Argument blocks of the stencil and self-coupling kernels and the
// declarations of their host launchers (defined in dd_hop.cuh, instantiated
// once per precision triple in dd_hop_*.cu).
#pragma once

#include <cstdlib>

#include "dd_device.cuh"

namespace dd {

enum Epi {
  EPI_D = 0,        // out = M y + beta acc            (D, D^H; Dhat second step)
  EPI_AINV = 1,     // out = M (beta acc)              (Dhat first step)
  EPI_RESID = 2,    // out = z - (M y + beta acc)      (r = b - D x)
  EPI_ADD = 3,      // out = y + beta acc              (right-hand side preparation)
  EPI_AINV_ADD = 4  // out = M (y + beta acc)          (even-site reconstruction)
};

struct HopArgs {
  Geom g;
  int nrhs;
  int p0;            // output parity of the first part of the grid
  int npar;          // number of output parities in this launch (1 or 2)
  int64_t gstride;   // component-group stride of a half field = Vh * nrhs
  HalfField in[2];   // input field by parity (parity 1 - p is read for output parity p)
  HalfField out[2];  // output by parity
  HalfField y[2];    // per output parity: self term (EPI_D: the input's own parity)
  HalfField z[2];    // per output parity: residual base (EPI_RESID)
  const void* U[2];  // links by parity of their site: [mu][9][Vh] complex elements
  const void* M[2];  // 6x6 Hermitian blocks by output parity: [36][Vh] elements
  double beta;
  int rhs_block;  // batched launch: right-hand sides per thread (1 or 2)
  FastDiv fblk;   // division of the thread index by the RHS slots per site (set by the launcher)
  int recon;      // FP32 link form: 0 three rows, 12 rows 0 and 1 (row 2 rebuilt), 8 eight reals (dd_link8.cuh)
  int paired;     // fields in the paired-RHS layout (dd_pair.cuh; nrhs even, FP32 / FP16)
};

// Self-coupling apply without hopping: out = M y on npar parities.
struct BlockArgs {
  int64_t Vh;
  int nrhs;
  int p0, npar;
  int64_t gstride;
  HalfField y[2], out[2];
  const void* M[2];
};

// Largest RHS block of the RHS-blocked stencils (DD_RHS_BLOCK overrides: 1
// disables them, including the paired-RHS stencil of canonical applies).
inline int rhs_block_limit() {
  static int v = 0;
  if (v == 0) {
    const char* e = getenv("DD_RHS_BLOCK");
    v = e ? atoi(e) : 4;
    if (v < 1) v = 1;
  }
  return v;
}

// DD_STAGE=1 opts in to the row-staged stencil of native-layout FP32 applies
// (dd_stage.cuh); canonical applies then keep the native layout.
inline bool stage_opted_in() {
  static const int v = getenv("DD_STAGE") ? atoi(getenv("DD_STAGE")) : 0;
  return v != 0;
}

template <int PG, int PIN, int POUT>
cudaError_t launch_hop(const HopArgs& a, bool dagger, int epi, cudaStream_t st);
// The paired-RHS stencil (dd_hop_pair.cuh): EPI_D or EPI_AINV on paired fields
// with nrhs even; PV is the vector precision (P32 or P16), PG that of links
// and blocks (instantiated for (P32, P32), (P16, P16) and (P16, P32)).
template <int PG, int PV>
cudaError_t launch_hop_pair(const HopArgs& a, bool dagger, int epi, cudaStream_t st);
// traversal slab depth for a lattice and the bytes per site of the stencil (dd_ops.cu)
int zblock_for(const int dims[4], int64_t bytes_per_site);
// Device flag that kernels with bounded waits set when a wait expires (one
// int, allocated and zeroed on first use; nullptr if that fails).
int* device_error_flag();
int64_t stencil_bytes_per_site(int pg, int nrhs);
template <int PG, int PIN, int POUT>
cudaError_t launch_block(const BlockArgs& a, cudaStream_t st);
// Blocks (of 128 threads) of the fused-norm stencil over `sites` sites: the
// partial sums it writes (its scratch: these plus blas_reduce_scratch).
inline int64_t hop_norm_blocks(int64_t sites) { return (sites + 127) / 128; }
// EPI_D stencil of one right-hand side with an FP32 output that also writes
// norm_out[0] = (|out|^2, 0) (instantiated for (P32, P32, P32) and
// (P16, P32, P32)).
template <int PG, int PIN, int POUT>
cudaError_t launch_hop_norm(const HopArgs& a, bool dagger, double2* partials, int64_t npartials,
                            double2* norm_out, cudaStream_t st);

}  // namespace dd
