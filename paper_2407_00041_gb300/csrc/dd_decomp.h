// Argument blocks of the domain-decomposed stencil (kernels in
// dd_decomp.cuh, host side in dd_decomp.cu).
#pragma once

#include "dd_ops.h"

namespace dd {

// Position of one local lattice in the global one.
struct DomGeom {
  int off[4];        // global coordinates of local site 0 (even in every direction)
  int N[4];          // global extents
  int xch[4];        // 1: direction mu is split across ranks and its seams are exchanged
  int64_t nface[4];  // sites of one mu face (both parities): product of the other three local extents
};

// Face messages of one rank: [mu] of the outgoing and incoming buffers.
struct FaceBufs {
  void* lam_send[4];
  void* chi_send[4];
  const void* lam_recv[4];
  const void* chi_recv[4];
};

struct DomHopArgs {
  HopArgs h;             // the local stencil (local geometry, fields, links, blocks)
  DomGeom d;
  FaceBufs f;
  const int* bsites;     // boundary sites of the rank, parity 0 then parity 1, as p * Vh + s
  int64_t nb[2];         // boundary sites per parity
};

// Face message layout for arithmetic type R: the 6 complex numbers of one
// (face site, RHS) slot i (= f * N + r) in 16-byte groups [group][nface * N]
// (three float4 for float, six double2 for double), followed for FP16 input
// fields by the sender's site scale [nface * N] (float).
template <typename R>
__host__ __device__ inline size_t face_msg_bytes(int64_t nface, int nrhs, bool scale) {
  return (size_t)nface * nrhs * (12 * sizeof(R) + (scale ? sizeof(float) : 0));
}

template <int PG, int PIN>
cudaError_t launch_face_pack(const DomHopArgs& A, bool dagger, cudaStream_t st);
template <int PG, int PIN, int POUT>
cudaError_t launch_hop_dd(const DomHopArgs& A, bool dagger, int epi, bool boundary, cudaStream_t st);

}  // namespace dd
