"""Schwarz alternating procedure (SAP): the block smoother that the thesis
names for DDalphaAMG's multigrid (Section 1.3), here as a flexible
preconditioner M_j of Algorithm 2.

TEST INFRASTRUCTURE ONLY (part of the CPU oracle).

The thesis names SAP (additive, red-black or 16-colour multiplicative
Schwarz) and refers to Saad's book for the method.  Reading taken here: the
red-black multiplicative Schwarz method with non-overlapping blocks and
block solves by minimal-residual steps:
  * the lattice is cut into blocks of b_T x b_Z x b_Y x b_X sites aligned with
    the origin; the colour of a block is the parity of the sum of its block
    coordinates (red 0, black 1), so two blocks of one colour never share a
    face (every extent holds an even number of blocks);
  * D_B is D restricted to the sites of block B with every hop that leaves
    the block dropped (a Dirichlet boundary);
  * one cycle on D z = v, residual r = v - D z: for the red blocks, then the
    black blocks: e_B ~= D_B^{-1} r_B on every block of the colour (they are
    independent of one another), z += e, then r = v - D z;
  * the block solve is k minimal-residual steps from e = 0:
    q = D_B rho, alpha = <q, rho> / <q, q> with <a, b> = a^H b,
    e += alpha rho, rho -= alpha q  (rho starts at r_B);
  * M^{-1} v is z after n cycles from z = 0.
Everything is FP64; D comes from the oracle's Eq. 1.13.
"""
from __future__ import annotations

import numpy as np


def block_coords(dims, block):
    """Per site (lexicographic order): block coordinates [V, 4] and colour [V]."""
    dims, block = tuple(int(d) for d in dims), tuple(int(b) for b in block)
    for n, b in zip(dims, block):
        if b < 1 or n % b or (n // b) % 2:
            raise ValueError(f"extent {n} must hold an even number of blocks of {b}")
    c = np.stack(np.unravel_index(np.arange(int(np.prod(dims))), dims), axis=1)
    bc = c // np.array(block)
    return bc, bc.sum(axis=1) % 2


def blocks(dims, block):
    """(sites, colour) of every block, blocks in lexicographic order of their
    block coordinates, sites in lexicographic order."""
    bc, col = block_coords(dims, block)
    nb = np.array(dims) // np.array(block)
    key = ((bc[:, 0] * nb[1] + bc[:, 1]) * nb[2] + bc[:, 2]) * nb[3] + bc[:, 3]
    order = np.argsort(key, kind="stable")
    bounds = np.searchsorted(key[order], np.arange(int(np.prod(nb)) + 1))
    out = []
    for k in range(int(np.prod(nb))):
        s = order[bounds[k]:bounds[k + 1]]
        out.append((s, int(col[s[0]])))
    return out


def block_op(apply_D, V, sites):
    """D_B: x_B -> (D applied to x_B padded with zeros)|_B."""
    def DB(x):
        full = np.zeros((V, 12), dtype=np.complex128)
        full[sites] = x.reshape(-1, 12)
        return apply_D(full)[sites]
    return DB


def mr(DB, r, steps, record=None):
    """k minimal-residual steps on D_B e = r from e = 0."""
    e = np.zeros_like(r)
    rho = r.copy()
    for _ in range(steps):
        q = DB(rho)
        alpha = np.vdot(q, rho) / np.vdot(q, q).real
        e = e + alpha * rho
        rho = rho - alpha * q
        if record is not None:
            record.append(np.linalg.norm(rho))
    return e


def sap(apply_D, dims, v, block, cycles, mr_steps, block_solver=None, trace=None):
    """M^{-1} v after `cycles` red-black SAP cycles from z = 0.  apply_D(x) is
    the full operator on [V, 12] fields; block_solver(DB, r_B, sites), if
    given, replaces the MR block solve (used by tests with exact solves);
    trace, if a list, receives the residual after every half cycle."""
    V = int(np.prod(dims))
    v = np.asarray(v, dtype=np.complex128).reshape(V, 12)
    z = np.zeros_like(v)
    r = v.copy()
    blist = blocks(dims, block)
    for _ in range(cycles):
        for colour in (0, 1):
            for sites, c in blist:
                if c != colour:
                    continue
                DB = block_op(apply_D, V, sites)
                if block_solver is None:
                    e = mr(DB, r[sites], mr_steps)
                else:
                    e = block_solver(DB, r[sites], sites)
                z[sites] += e
            r = v - apply_D(z)
            if trace is not None:
                trace.append(r.copy())
    return z
