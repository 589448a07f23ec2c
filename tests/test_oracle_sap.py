"""Pins of the oracle's SAP smoother (oracle/sap.py) against what does not
depend on it: the independent dense assembly of Eq. 1.13 (tests/_dense.py),
numpy's least-squares routine, and the structure of the red-black
multiplicative Schwarz method."""
import numpy as np
import pytest

import oracle
import synthetic
from oracle import sap
from tests import _dense

M0, CSW = -0.4, 1.0


@pytest.fixture(scope="module")
def small():
    dims = (4, 4, 4, 4)
    U = synthetic.gauge(dims)
    A = oracle.clover(U, dims, M0, CSW)
    D = _dense.dense_D(U, dims, M0, CSW, t_bc=-1, A=_dense.clover_field(U, dims, M0, CSW))
    apply = lambda x: oracle.apply_D(U, A, x.reshape(-1, 12), dims)
    return dims, U, A, D, apply


def _rows(sites):
    return (12 * np.asarray(sites)[:, None] + np.arange(12)[None, :]).reshape(-1)


def test_blocks_partition_and_colours():
    dims, block = (4, 8, 4, 4), (2, 2, 2, 2)
    bl = sap.blocks(dims, block)
    assert len(bl) == 2 * 4 * 2 * 2
    allsites = np.sort(np.concatenate([s for s, _ in bl]))
    assert np.array_equal(allsites, np.arange(int(np.prod(dims))))
    # two blocks of one colour never share a face
    bc, col = sap.block_coords(dims, block)
    for mu in range(4):
        c = np.stack(np.unravel_index(np.arange(int(np.prod(dims))), dims), axis=1)
        c2 = c.copy()
        c2[:, mu] = (c2[:, mu] + 1) % dims[mu]
        j = np.ravel_multi_index(tuple(c2.T), dims)
        crossing = np.any(bc != bc[j], axis=1)
        assert np.all(col[crossing] != col[j][crossing])
    with pytest.raises(ValueError):
        sap.blocks((4, 4, 4, 6), (2, 2, 2, 2))  # three blocks in X


def test_block_operator_is_the_dense_submatrix(small):
    dims, U, A, D, apply = small
    V = int(np.prod(dims))
    rng = np.random.default_rng(1)
    for sites, _ in sap.blocks(dims, (2, 2, 2, 2))[:5]:
        DB = sap.block_op(apply, V, sites)
        x = rng.standard_normal((len(sites), 12)) + 1j * rng.standard_normal((len(sites), 12))
        R = _rows(sites)
        ref = D[np.ix_(R, R)] @ x.reshape(-1)
        assert np.linalg.norm(DB(x).reshape(-1) - ref) < 1e-13 * np.linalg.norm(ref)


def test_one_mr_step_is_the_least_squares_step(small):
    dims, U, A, D, apply = small
    V = int(np.prod(dims))
    sites, _ = sap.blocks(dims, (2, 2, 2, 2))[3]
    DB = sap.block_op(apply, V, sites)
    r = synthetic.spinor(dims)[0].reshape(-1, 12)[sites]
    e = sap.mr(DB, r, 1)
    R = _rows(sites)
    Dr = D[np.ix_(R, R)] @ r.reshape(-1)
    alpha = np.linalg.lstsq(Dr[:, None], r.reshape(-1), rcond=None)[0][0]
    assert np.linalg.norm(e.reshape(-1) - alpha * r.reshape(-1)) < 1e-13 * np.linalg.norm(e)


def test_mr_residuals_do_not_grow(small):
    dims, U, A, D, apply = small
    V = int(np.prod(dims))
    sites, _ = sap.blocks(dims, (2, 2, 2, 2))[6]
    DB = sap.block_op(apply, V, sites)
    r = synthetic.spinor(dims)[0].reshape(-1, 12)[sites]
    norms = []
    e = sap.mr(DB, r, 12, record=norms)
    assert all(b <= a * (1 + 1e-12) for a, b in zip([np.linalg.norm(r)] + norms, norms))
    # the recorded residual is the true one
    assert abs(np.linalg.norm(r - DB(e)) - norms[-1]) < 1e-12 * np.linalg.norm(r)


def test_exact_block_solves_clear_the_residual_of_each_colour(small):
    """With exact block solves, after the red half cycle the residual vanishes
    on every red block (red blocks couple only to black ones), after the black
    half cycle on every black block."""
    dims, U, A, D, apply = small
    V = int(np.prod(dims))
    block = (2, 2, 2, 2)

    def exact(DB, rB, sites):
        R = _rows(sites)
        return np.linalg.solve(D[np.ix_(R, R)], rB.reshape(-1)).reshape(-1, 12)

    v = synthetic.spinor(dims)[0].reshape(-1, 12)
    trace = []
    sap.sap(apply, dims, v, block, 1, 0, block_solver=exact, trace=trace)
    _, col = sap.block_coords(dims, block)
    assert np.linalg.norm(trace[0][col == 0]) < 1e-12 * np.linalg.norm(v)
    assert np.linalg.norm(trace[0][col == 1]) > 1e-3 * np.linalg.norm(v)
    assert np.linalg.norm(trace[1][col == 1]) < 1e-12 * np.linalg.norm(v)


def test_sap_preconditioned_fgmres_converges(small):
    """Algorithm 2 with M_j = two SAP cycles reaches the 1e-10 tolerance, and
    needs fewer Arnoldi steps than without preconditioner."""
    dims, U, A, D, apply = small
    b = synthetic.spinor(dims)[0].reshape(-1)
    M = lambda j, v: sap.sap(apply, dims, v, (2, 2, 2, 2), 2, 4).reshape(-1)
    A1 = lambda x: apply(x).reshape(-1)
    x, st = oracle.fgmres(A1, b, m=16, tol=1e-10, max_restarts=50, M=M)
    assert st.converged
    assert np.linalg.norm(b - D @ x) < 1e-10 * np.linalg.norm(b)
    _, st0 = oracle.fgmres(A1, b, m=16, tol=1e-10, max_restarts=50)
    assert sum(st.inner_steps) < sum(st0.inner_steps)
