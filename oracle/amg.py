"""Two-level algebraic multigrid (AMG) preconditioner of Section 1.3: the
coarse-grid correction z <- z + P D_c^{-1} R r with the SAP smoother.

TEST INFRASTRUCTURE ONLY (part of the CPU oracle; imported only by tests/,
__graft_entry__.smoke() and bench.py's CPU legs).

Section 1.3 states the method: a projection D_c of D onto a coarser lattice
that acts on the near kernel (eigenvectors of small |eigenvalue|) like D and
couples only nearest neighbours; a restriction R and a prolongation P between
the lattices built from approximations of those eigenvectors (test vectors)
found in a setup phase; the subspace correction together with the smoother
as M_j of FGMRES.  Table 5.2 fixes the depth-one coarse lattices (aggregates
of 4^4 or 8^4 sites on the configurations there), 24 test vectors and 4 setup
iterations.  The thesis gives no formulas for P, R or the setup; the reading
taken here (the aggregation-based construction of the DDalphaAMG papers the
thesis cites) is:
  * aggregates: blocks of a_T x a_Z x a_Y x a_X sites aligned with the
    origin; each carries two sets of coarse degrees of freedom, one per
    chirality (spin components 0, 1: gamma5 = +1; 2, 3: gamma5 = -1);
  * P: for aggregate A and chirality c the restrictions of the N test vectors
    w_1 .. w_N to the 6 |A| components (A, c) are orthonormalised by
    Gram-Schmidt in the order 1 .. N; column i of the result is the fine
    vector of coarse degree of freedom (A, c, i); R = P^H;
  * D_c = R D P (Galerkin), so D_c couples an aggregate with itself and its
    eight neighbours only;
  * one application of the preconditioner to v: z = P D_c^{-1} R v, then
    z += SAP(v - D z) (the smoother of oracle/sap.py, post-smoothing);
  * setup: from N seeded random vectors, k_init times w_i <- SAP(w_i)
    (normalised), then n_setup times: build P, D_c from the w_i and apply
    w_i <- M^{-1} w_i (normalised); P and D_c from the final w_i.
Here the coarse system is solved exactly (a dense solve on the small lattices
of the tests).  Everything is FP64.
"""
from __future__ import annotations

import numpy as np

from . import sap as _sap


def aggregates(dims, agg):
    """Sites (lexicographic) of every aggregate, aggregates in lexicographic
    order of their block coordinates; requires agg to divide dims."""
    dims, agg = tuple(int(d) for d in dims), tuple(int(a) for a in agg)
    for n, a in zip(dims, agg):
        if a < 1 or n % a:
            raise ValueError(f"aggregate extent {a} does not divide {n}")
    c = np.stack(np.unravel_index(np.arange(int(np.prod(dims))), dims), axis=1)
    bc = c // np.array(agg)
    nb = np.array(dims) // np.array(agg)
    key = ((bc[:, 0] * nb[1] + bc[:, 1]) * nb[2] + bc[:, 2]) * nb[3] + bc[:, 3]
    order = np.argsort(key, kind="stable")
    bounds = np.searchsorted(key[order], np.arange(int(np.prod(nb)) + 1))
    return [order[bounds[k]:bounds[k + 1]] for k in range(int(np.prod(nb)))], tuple(int(v) for v in nb)


def chirality_components(c):
    """The 6 components (3 spin + colour) of chirality c (0: spins 0, 1)."""
    spins = (0, 1) if c == 0 else (2, 3)
    return np.array([3 * s + col for s in spins for col in range(3)])


def gram_schmidt(W):
    """Columns of W orthonormalised in order (modified Gram-Schmidt)."""
    Q = np.array(W, dtype=np.complex128, copy=True)
    for i in range(Q.shape[1]):
        for k in range(i):
            Q[:, i] -= np.vdot(Q[:, k], Q[:, i]) * Q[:, k]
        n = np.linalg.norm(Q[:, i])
        if n == 0:
            raise ValueError("test vectors are linearly dependent on an aggregate")
        Q[:, i] /= n
    return Q


class TwoLevel:
    """P, R = P^H and D_c = R D P from test vectors w [N, V, 12]."""

    def __init__(self, apply_D, dims, agg, w):
        self.apply_D = apply_D
        self.dims = tuple(int(d) for d in dims)
        self.V = int(np.prod(self.dims))
        self.agg = tuple(int(a) for a in agg)
        w = np.asarray(w, dtype=np.complex128).reshape(-1, self.V, 12)
        self.N = w.shape[0]
        self.blocks, self.cdims = aggregates(self.dims, self.agg)
        self.nagg = len(self.blocks)
        self.nc = self.nagg * 2 * self.N
        # P[a][c]: (6 |A|, N) with rows (site in A, component of chirality c)
        self.P = []
        for sites in self.blocks:
            per = []
            for c in (0, 1):
                comp = chirality_components(c)
                W = w[:, sites][:, :, comp].reshape(self.N, -1).T
                per.append(gram_schmidt(W))
            self.P.append(per)
        self.Dc = self._coarse_operator()

    def index(self, a, c, i):
        """Coarse degree of freedom (aggregate a, chirality c, vector i)."""
        return (a * 2 + c) * self.N + i

    def prolong(self, vc):
        vc = np.asarray(vc).reshape(self.nagg, 2, self.N)
        out = np.zeros((self.V, 12), dtype=np.complex128)
        for a, sites in enumerate(self.blocks):
            for c in (0, 1):
                comp = chirality_components(c)
                out[np.ix_(sites, comp)] = (self.P[a][c] @ vc[a, c]).reshape(len(sites), 6)
        return out

    def restrict(self, v):
        v = np.asarray(v).reshape(self.V, 12)
        out = np.zeros((self.nagg, 2, self.N), dtype=np.complex128)
        for a, sites in enumerate(self.blocks):
            for c in (0, 1):
                comp = chirality_components(c)
                out[a, c] = self.P[a][c].conj().T @ v[np.ix_(sites, comp)].reshape(-1)
        return out.reshape(-1)

    def _coarse_operator(self):
        """D_c = R D P column by column: D applied to every prolongated unit vector."""
        Dc = np.zeros((self.nc, self.nc), dtype=np.complex128)
        e = np.zeros(self.nc, dtype=np.complex128)
        for k in range(self.nc):
            e[:] = 0
            e[k] = 1
            Dc[:, k] = self.restrict(self.apply_D(self.prolong(e)))
        return Dc

    def coarse_correction(self, r):
        """P D_c^{-1} R r (exact coarse solve)."""
        return self.prolong(np.linalg.solve(self.Dc, self.restrict(r)))

    def apply(self, v, sap_block, sap_cycles, sap_mr):
        """M^{-1} v: coarse-grid correction, then SAP post-smoothing."""
        v = np.asarray(v, dtype=np.complex128).reshape(self.V, 12)
        z = self.coarse_correction(v)
        if sap_cycles > 0:
            r = v - self.apply_D(z)
            z = z + _sap.sap(self.apply_D, self.dims, r, sap_block, sap_cycles, sap_mr)
        return z


def setup(apply_D, dims, agg, w0, n_setup, k_init, sap_block, sap_cycles, sap_mr):
    """The setup phase: k_init SAP smoothings of the seeded vectors w0
    [N, V, 12], then n_setup rounds of w_i <- M^{-1} w_i with the two-level
    method built from the current w (each w_i normalised after every step)."""
    dims = tuple(int(d) for d in dims)
    w = np.array(w0, dtype=np.complex128, copy=True).reshape(len(w0), -1, 12)
    for _ in range(k_init):
        for i in range(len(w)):
            w[i] = _sap.sap(apply_D, dims, w[i], sap_block, sap_cycles, sap_mr)
            w[i] /= np.linalg.norm(w[i])
    for _ in range(n_setup):
        tl = TwoLevel(apply_D, dims, agg, w)
        for i in range(len(w)):
            w[i] = tl.apply(w[i], sap_block, sap_cycles, sap_mr)
            w[i] /= np.linalg.norm(w[i])
    return TwoLevel(apply_D, dims, agg, w), w
