"""Pins of the oracle's two-level AMG (oracle/amg.py) against what does not
depend on it: the independent dense assembly of Eq. 1.13 (tests/_dense.py),
numpy's Householder QR for the aggregate-wise orthonormalisation, and exact
properties of the Galerkin construction D_c = P^H D P."""
import numpy as np
import pytest

import oracle
import synthetic
from oracle import amg
from oracle import sap as osap
from tests import _dense

M0, CSW = -0.4, 1.0


def _system(dims):
    U = synthetic.gauge(dims)
    A = oracle.clover(U, dims, M0, CSW)
    apply = lambda x: oracle.apply_D(U, A, x.reshape(-1, 12), dims)
    return U, A, apply


@pytest.fixture(scope="module")
def small():
    dims, agg, N = (4, 4, 4, 4), (2, 2, 2, 2), 4
    U, A, apply = _system(dims)
    w = synthetic.spinor(dims, nrhs=N, seed=7).reshape(N, -1, 12)
    tl = amg.TwoLevel(apply, dims, agg, w)
    D = _dense.dense_D(U, dims, M0, CSW, t_bc=-1, A=_dense.clover_field(U, dims, M0, CSW))
    return dims, agg, N, U, A, apply, w, tl, D


def _dense_P(dims, agg, w):
    """Prolongation as a dense (12 V, n_c) matrix from numpy's QR (Householder),
    each column's phase fixed so that R has a positive real diagonal (the
    Gram-Schmidt convention)."""
    V = int(np.prod(dims))
    N = len(w)
    c = np.stack(np.unravel_index(np.arange(V), dims), axis=1)
    bc = c // np.array(agg)
    nb = np.array(dims) // np.array(agg)
    key = ((bc[:, 0] * nb[1] + bc[:, 1]) * nb[2] + bc[:, 2]) * nb[3] + bc[:, 3]
    nagg = int(np.prod(nb))
    P = np.zeros((12 * V, nagg * 2 * N), dtype=np.complex128)
    for a in range(nagg):
        sites = np.nonzero(key == a)[0]  # lexicographic
        for ch, spins in enumerate(((0, 1), (2, 3))):
            comp = np.array([3 * s + col for s in spins for col in range(3)])
            rows = (12 * sites[:, None] + comp[None, :]).reshape(-1)
            W = np.stack([w[i][np.ix_(sites, comp)].reshape(-1) for i in range(N)], axis=1)
            Q, R = np.linalg.qr(W)
            ph = np.diag(R) / np.abs(np.diag(R))
            Q = Q * ph[None, :]
            P[rows, (a * 2 + ch) * N:(a * 2 + ch + 1) * N] = Q
    return P


def test_aggregates_partition():
    bl, cd = amg.aggregates((4, 8, 4, 4), (2, 4, 2, 2))
    assert cd == (2, 2, 2, 2) and len(bl) == 16
    assert np.array_equal(np.sort(np.concatenate(bl)), np.arange(512))
    assert all(len(s) == 32 for s in bl)
    with pytest.raises(ValueError):
        amg.aggregates((4, 4, 4, 6), (2, 2, 2, 4))


def test_prolongation_is_orthonormal_and_matches_householder(small):
    dims, agg, N, U, A, apply, w, tl, D = small
    for a in range(tl.nagg):
        for c in (0, 1):
            Pa = tl.P[a][c]
            assert np.linalg.norm(Pa.conj().T @ Pa - np.eye(N)) < 1e-13
    Pd = _dense_P(dims, agg, w)
    rng = np.random.default_rng(3)
    y = rng.standard_normal(tl.nc) + 1j * rng.standard_normal(tl.nc)
    assert np.linalg.norm(tl.prolong(y).reshape(-1) - Pd @ y) < 1e-12 * np.linalg.norm(y)
    x = rng.standard_normal((tl.V, 12)) + 1j * rng.standard_normal((tl.V, 12))
    assert np.linalg.norm(tl.restrict(x) - Pd.conj().T @ x.reshape(-1)) < 1e-12 * np.linalg.norm(x)


def test_coarse_operator_is_the_galerkin_product_of_the_dense_assembly(small):
    dims, agg, N, U, A, apply, w, tl, D = small
    Pd = _dense_P(dims, agg, w)
    ref = Pd.conj().T @ D @ Pd
    assert np.linalg.norm(tl.Dc - ref) < 1e-12 * np.linalg.norm(ref)


def test_coarse_operator_couples_nearest_neighbours_only(small):
    dims, agg, N, U, A, apply, w, tl, D = small
    cd = tl.cdims
    coords = np.stack(np.unravel_index(np.arange(tl.nagg), cd), axis=1)
    blk = 2 * N
    scale = np.linalg.norm(tl.Dc)
    for a in range(tl.nagg):
        for b in range(tl.nagg):
            d = (coords[a] - coords[b]) % np.array(cd)
            d = np.minimum(d, np.array(cd) - d)
            near = d.sum() <= 1
            B = tl.Dc[a * blk:(a + 1) * blk, b * blk:(b + 1) * blk]
            if not near:
                assert np.linalg.norm(B) < 1e-14 * scale


def test_coarse_gamma5_structure(small):
    """D^H = gamma5 D gamma5 and P keeps chirality, so D_c^H = G D_c G with G
    = +1 on chirality-0 and -1 on chirality-1 coarse degrees of freedom."""
    dims, agg, N, U, A, apply, w, tl, D = small
    G = np.tile(np.concatenate([np.ones(N), -np.ones(N)]), tl.nagg)
    lhs = tl.Dc.conj().T
    rhs = G[:, None] * tl.Dc * G[None, :]
    assert np.linalg.norm(lhs - rhs) < 1e-12 * np.linalg.norm(lhs)


def test_coarse_correction_reproduces_the_range_of_P(small):
    """Galerkin projection: P D_c^{-1} R D (P y) = P y."""
    dims, agg, N, U, A, apply, w, tl, D = small
    rng = np.random.default_rng(5)
    y = rng.standard_normal(tl.nc) + 1j * rng.standard_normal(tl.nc)
    Py = tl.prolong(y)
    got = tl.coarse_correction(apply(Py))
    assert np.linalg.norm(got - Py) < 1e-10 * np.linalg.norm(Py)


def test_square_prolongation_gives_the_exact_inverse():
    """Aggregates of one site with N = 6 test vectors: P is unitary, D_c is
    unitarily equivalent to D and the coarse correction is D^{-1}; FGMRES with
    this M_j stops after one Arnoldi step with the exact solution."""
    dims = (2, 2, 2, 2)
    U, A, apply = _system(dims)
    w = synthetic.spinor(dims, nrhs=6, seed=11).reshape(6, -1, 12)
    tl = amg.TwoLevel(apply, dims, (1, 1, 1, 1), w)
    b = synthetic.spinor(dims, nrhs=1)[0].reshape(-1, 12)
    z = tl.coarse_correction(b)
    assert np.linalg.norm(apply(z) - b) < 1e-11 * np.linalg.norm(b)
    x, st = oracle.fgmres(lambda v: apply(v).reshape(-1), b.reshape(-1), m=10, tol=1e-10,
                          M=lambda j, v: tl.apply(v, (1, 1, 1, 2), 0, 1).reshape(-1))
    assert st.converged and sum(st.inner_steps) == 1


def test_setup_and_two_level_fgmres_beat_the_smoother_alone():
    """On a 4^4 lattice the setup (SAP-smoothed vectors, two rounds of the
    two-level method) gives a preconditioner under which FGMRES needs fewer
    Arnoldi steps than with SAP alone at the same smoothing."""
    dims, agg, N = (4, 4, 4, 4), (2, 2, 2, 2), 8
    U, A, apply = _system(dims)
    w0 = synthetic.spinor(dims, nrhs=N, seed=21).reshape(N, -1, 12)
    blk = (2, 2, 2, 2)
    tl, w = amg.setup(apply, dims, agg, w0, n_setup=2, k_init=2, sap_block=blk, sap_cycles=1, sap_mr=3)
    b = synthetic.spinor(dims, nrhs=1)[0].reshape(-1)
    op = lambda v: apply(v).reshape(-1)
    _, st_amg = oracle.fgmres(op, b, m=30, tol=1e-10, max_restarts=50,
                              M=lambda j, v: tl.apply(v, blk, 1, 3).reshape(-1))
    _, st_sap = oracle.fgmres(op, b, m=30, tol=1e-10, max_restarts=50,
                              M=lambda j, v: osap.sap(apply, dims, v, blk, 1, 3).reshape(-1))
    assert st_amg.converged
    assert sum(st_amg.inner_steps) < sum(st_sap.inner_steps), (st_amg.inner_steps, st_sap.inner_steps)
