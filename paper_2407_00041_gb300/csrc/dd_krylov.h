// GMRES (Algorithm 2 with M_j = I) on a custom FP64 operator: the solver's
// FGMRES machinery (classical Gram-Schmidt, Givens rotations on the host)
// applied to the AMG coarse system (dd_amg.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>

namespace dd {

struct CoarseKrylov;
// Vectors of L complex doubles (16-byte groups) with N right-hand sides
// innermost (RHS of group g = g mod N); restart length m.  nullptr on failure.
CoarseKrylov* coarse_krylov_create(int64_t L, int N, int m, std::function<int(const void*, void*, cudaStream_t)> op);
void coarse_krylov_destroy(CoarseKrylov* k);
// e = approximate solution of op(e) = f from e = 0, each RHS to ||f - op e|| <
// tol_rel ||f|| or max_restarts cycles; *steps: Arnoldi steps taken.
int coarse_krylov_solve(CoarseKrylov* k, const void* f, void* e, double tol_rel, int max_restarts, cudaStream_t st,
                        int* steps);

}  // namespace dd
