"""GPU solver: FGMRES (Algorithm 2) inside FP64 iterative refinement.

Parity for an iteration is on results: the FP64 true residual of the GPU
solution, recomputed by the CPU oracle, must be below the tolerance, and the
solution must match the oracle's own FGMRES solution.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
import paper_2407_00041_gb300 as dd
from tests._gpu import CSW, M0, make, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sys44():
    dims = (4, 4, 4, 4)
    U, lat, g, op = make(dims)
    A = oracle.clover(U, dims, M0, CSW)
    b = synthetic.spinor(dims, nrhs=3)
    xs = []
    for r in range(3):
        x, st = oracle.fgmres(lambda v: oracle.apply_D(U, A, v.reshape(-1, 12), dims).reshape(-1),
                              b[r].reshape(-1), m=30, tol=1e-12, max_restarts=400)
        assert st.converged
        xs.append(x.reshape(b[r].shape))
    return dims, U, A, op, b, np.stack(xs), (lat, g)


def oracle_residual(U, A, dims, b, x):
    r = b.reshape(-1, 12) - oracle.apply_D(U, A, x.reshape(-1, 12), dims)
    return np.linalg.norm(r) / np.linalg.norm(b)


@pytest.mark.parametrize("inner", [dd.DD_PREC_F64, dd.DD_PREC_F32, dd.DD_PREC_F16])
@pytest.mark.parametrize("even_odd", [1, 0])
@pytest.mark.parametrize("precond", [dd.DD_PRECOND_NONE, dd.DD_PRECOND_NORMAL, dd.DD_PRECOND_CGNR])
def test_solve_to_1e10(sys44, inner, even_odd, precond):
    dims, U, A, op, b, xref, _ = sys44
    bt = torch.from_numpy(b[:1]).cuda()
    x = torch.zeros_like(bt)
    status, st = op.solve(bt, x, 1, tol=1e-10, inner_prec=inner, even_odd=even_odd, restart=30, precond=precond,
                          precond_iters=8)
    assert status == 0, st
    assert st["converged"] == 1 and st["true_residual"] < 1e-10
    xn = x.cpu().numpy()[0]
    assert oracle_residual(U, A, dims, b[0], xn) < 1e-10
    assert rel(xn, xref[0]) < 1e-8
    if inner != dd.DD_PREC_F64:
        assert st["outer_iterations"] >= 2  # refinement did the last digits


@pytest.mark.parametrize("inner,precond", [(dd.DD_PREC_F32, dd.DD_PRECOND_CGNR), (dd.DD_PREC_F16, dd.DD_PRECOND_CGNR),
                                           (dd.DD_PREC_F16, dd.DD_PRECOND_CGNR16),
                                           (dd.DD_PREC_F32, dd.DD_PRECOND_CGNR16)])
def test_cg_norms_fused_into_the_stencil(inner, precond, monkeypatch):
    """The CG preconditioner takes |Dhat p|^2 and |Dhat^H r|^2 from the
    second stencil launch of Dhat (per-block partial sums; 1080 odd sites =
    eight blocks of 128 and a ragged block of 56) and, with DD_FUSED_NORM=0,
    from a separate reduction of the stored vector (with FP16 CG vectors:
    the fused norm is that of the FP32 result before its rounding to FP16).
    Both solves meet the tolerance against the oracle, agree, and take the
    same number of Arnoldi steps to within one."""
    dims = (10, 6, 6, 6)
    U, lat, g, op = make(dims)
    A = oracle.clover(U, dims, M0, CSW)
    b = synthetic.spinor(dims, nrhs=1)
    xs, steps = [], []
    for fused in (True, False):
        if fused:
            monkeypatch.delenv("DD_FUSED_NORM", raising=False)
        else:
            monkeypatch.setenv("DD_FUSED_NORM", "0")
        bt = torch.from_numpy(b).cuda()
        x = torch.zeros_like(bt)
        status, st = op.solve(bt, x, 1, tol=1e-10, inner_prec=inner, restart=8, precond=precond,
                              precond_iters=16)
        assert status == 0 and st["true_residual"] < 1e-10, st
        xn = x.cpu().numpy()[0]
        assert oracle_residual(U, A, dims, b[0], xn) < 1e-10
        xs.append(xn)
        steps.append(st["inner_iterations"])
    assert rel(xs[0], xs[1]) < 1e-8
    assert abs(steps[0] - steps[1]) <= 1, steps


def test_multi_rhs_solve(sys44):
    dims, U, A, op, b, xref, _ = sys44
    bt = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bt)
    status, st = op.solve(bt, x, 3, tol=1e-10, inner_prec=dd.DD_PREC_F32, restart=16, gs_passes=2)
    assert status == 0, st
    xn = x.cpu().numpy()
    for r in range(3):
        assert oracle_residual(U, A, dims, b[r], xn[r]) < 1e-10
    # the same right-hand sides solved in batches of 2 and 1, on host buffers
    for batch, pc in ((2, dd.DD_PRECOND_NORMAL), (1, dd.DD_PRECOND_CGNR)):
        xh = np.zeros_like(b)
        status, st = op.solve(np.ascontiguousarray(b), xh, 3, layout=dd.DD_LAYOUT_CANONICAL_HOST, tol=1e-10,
                              rhs_batch=batch, precond=pc, precond_iters=6, restart=8)
        assert status == 0, st
        for r in range(3):
            assert oracle_residual(U, A, dims, b[r], xh[r]) < 1e-10
            assert rel(xh[r], xref[r]) < 1e-8


def test_host_layout_and_initial_guess(sys44):
    dims, U, A, op, b, xref, _ = sys44
    b0 = np.ascontiguousarray(b[:1])
    x = np.ascontiguousarray(xref[:1] * (1 + 1e-6))  # good initial guess
    status, st = op.solve(b0, x, 1, layout=dd.DD_LAYOUT_CANONICAL_HOST, tol=1e-10)
    assert status == 0 and oracle_residual(U, A, dims, b0[0], x[0]) < 1e-10
    assert st["outer_iterations"] <= 2


def test_not_converged_reports_best_iterate(sys44):
    dims, U, A, op, b, xref, _ = sys44
    bt = torch.from_numpy(b[:1]).cuda()
    x = torch.zeros_like(bt)
    status, st = op.solve(bt, x, 1, tol=1e-10, max_outer=1, inner_tol=1e-3, max_restarts=1, restart=4)
    assert status == dd.DD_ERR_NOT_CONVERGED
    assert st["converged"] == 0 and 1e-10 < st["true_residual"] < 1.0
    assert oracle_residual(U, A, dims, b[0], x.cpu().numpy()[0]) == pytest.approx(st["true_residual"], rel=1e-6)


def test_nan_rhs_is_rejected(sys44):
    dims, U, A, op, b, xref, _ = sys44
    bb = b[:1].copy()
    bb[0, 3, 1, 2] = np.nan
    bt = torch.from_numpy(bb).cuda()
    x = torch.zeros_like(bt)
    with pytest.raises(dd.DDError) as e:
        op.solve(bt, x, 1)
    assert e.value.status == dd.DD_ERR_ARG


@pytest.mark.parametrize("even_odd", [1, 0])
@pytest.mark.parametrize("nrhs", [1, 2])
def test_solve_with_fp16_cg_vectors(even_odd, nrhs):
    """DD_PRECOND_CGNR16: the CG preconditioner with its vectors in FP16
    (per-site scales) inside the FP16-inner solve reaches 1e-10, certified by
    the oracle, with FP64 refinement."""
    dims = (8, 8, 4, 4)
    U, lat, g, op = make(dims)
    A = oracle.clover(U, dims, M0, CSW)
    b = synthetic.spinor(dims, nrhs=nrhs)
    bt = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bt)
    status, st = op.solve(bt, x, nrhs, tol=1e-10, inner_prec=dd.DD_PREC_F16, even_odd=even_odd, restart=8,
                          precond=dd.DD_PRECOND_CGNR16, precond_iters=16, inner_tol=1e-3)
    assert status == 0, st
    assert st["converged"] == 1 and st["true_residual"] < 1e-10
    xn = x.cpu().numpy()
    for r in range(nrhs):
        assert oracle_residual(U, A, dims, b[r], xn[r]) < 1e-10


def test_fp16_cg_vectors_need_a_reduced_precision_inner_solve():
    dims = (4, 4, 4, 4)
    U, lat, g, op = make(dims)
    b = torch.from_numpy(synthetic.spinor(dims, nrhs=1)).cuda()
    x = torch.zeros_like(b)
    with pytest.raises(dd.DDError) as e:
        op.solve(b, x, 1, inner_prec=dd.DD_PREC_F64, precond=dd.DD_PRECOND_CGNR16)
    assert e.value.status == dd.DD_ERR_UNSUPPORTED


@pytest.mark.parametrize("even_odd", [1, 0])
@pytest.mark.parametrize("nrhs", [1, 2])
def test_solve_with_fp16_cg_vectors_fp32_operator(even_odd, nrhs):
    """DD_PRECOND_CGNR16 inside the FP32-inner solve: the CG vectors in FP16
    read by the FP32-link stencil; 1e-10 reached and certified by the oracle,
    with FP64 refinement."""
    dims = (8, 8, 4, 4)
    U, lat, g, op = make(dims)
    A = oracle.clover(U, dims, M0, CSW)
    b = synthetic.spinor(dims, nrhs=nrhs)
    bt = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bt)
    status, st = op.solve(bt, x, nrhs, tol=1e-10, inner_prec=dd.DD_PREC_F32, even_odd=even_odd, restart=8,
                          precond=dd.DD_PRECOND_CGNR16, precond_iters=16, inner_tol=1e-6)
    assert status == 0, st
    assert st["converged"] == 1 and st["true_residual"] < 1e-10
    xn = x.cpu().numpy()
    for r in range(nrhs):
        assert oracle_residual(U, A, dims, b[r], xn[r]) < 1e-10
