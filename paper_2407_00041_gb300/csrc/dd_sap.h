// Schwarz alternating procedure (SAP) smoother on the GPU (dd_sap.cu).
#pragma once

#include "dd_internal.h"

namespace dd {

// Largest block (sites) of the SAP block solve: one CTA of at most this many
// threads per block.
constexpr int kSapMaxSites = 256;

// DD_OK if `block` cuts the lattice into an even number of blocks along every
// direction with at most kSapMaxSites sites per block; DD_ERR_ARG otherwise.
int sap_check_blocks(const dd_lattice* lat, const int block[4], int pv);

// z = M^{-1} v: `cycles` red-black SAP cycles from z = 0 with `mr_steps`
// minimal-residual steps per block solve.  v, z, r: full native fields of
// precision pv with the same RHS count (r is workspace; v is not changed).
// (pg, pv) = (P64, P64), (P32, P32) or (P16, P32).  Enqueued on st.
int sap_apply(const dd_clover* op, int pg, int pv, const int block[4], int cycles, int mr_steps, const Field& v,
              const Field& z, const Field& r, cudaStream_t st);

}  // namespace dd
