"""FP64-accurate applies in FP32-pair arithmetic (DD_PREC_DF64): D, D^H,
Dhat, Dhat^H and the self coupling against the FP64 oracle at the FP64
tolerance (1e-13), on several lattice shapes and RHS counts, and against the
library's own FP64 applies.  The pair arithmetic keeps about 48 significant
bits (Dekker's double-word numbers), so its results differ from true FP64
ones at the 1e-14 level, far inside the tolerance."""
import numpy as np
import pytest
import torch

import oracle
import synthetic
import paper_2407_00041_gb300 as dd
from tests._gpu import CSW, M0, TOL, apply, rel

pytestmark = pytest.mark.gpu

ALL = dd.DD_PREC_F64 | dd.DD_PREC_F32 | dd.DD_PREC_F16 | dd.DD_PREC_DF64


def make_df(dims, eps=0.3):
    U = synthetic.gauge(dims, eps=eps)
    lat = dd.Lattice(dims, -1)
    g = dd.Gauge(lat, U, precisions=ALL)
    op = dd.Operator(g, M0, CSW, precisions=ALL)
    return U, lat, g, op


@pytest.fixture(scope="module", params=[(4, 4, 4, 4), (6, 4, 2, 8), (8, 6, 4, 2)], ids=lambda d: "x".join(map(str, d)))
def system(request):
    dims = request.param
    U, lat, g, op = make_df(dims)
    A = oracle.clover(U, dims, M0, CSW)
    return dims, U, A, op, (lat, g)


@pytest.mark.parametrize("nrhs", [1, 3])
def test_D_DH_against_oracle_and_fp64(system, nrhs):
    dims, U, A, op, _ = system
    psi = synthetic.spinor(dims, nrhs=nrhs)
    for which, ref_fn in ((dd.DD_OP_D, oracle.apply_D), (dd.DD_OP_DH, oracle.apply_DH)):
        got = apply(op, which, dd.DD_PREC_DF64, psi)
        f64 = apply(op, which, dd.DD_PREC_F64, psi)
        for r in range(nrhs):
            ref = ref_fn(U, A, psi[r].reshape(-1, 12), dims)
            assert rel(got[r], ref) < TOL[dd.DD_PREC_F64]
        assert rel(got, f64) < 1e-13
        assert not np.array_equal(got, f64)  # a result of its own, not the FP64 kernel's


@pytest.mark.parametrize("nrhs", [1, 2])
def test_Dhat_and_self_coupling(system, nrhs):
    dims, U, A, op, _ = system
    eo = oracle.EvenOdd(U, A, dims)
    full = synthetic.spinor(dims, nrhs=nrhs)
    v = np.stack([full[r].reshape(-1, 12)[eo.odd] for r in range(nrhs)])
    got = apply(op, dd.DD_OP_DHAT, dd.DD_PREC_DF64, v)
    gotH = apply(op, dd.DD_OP_DHAT_H, dd.DD_PREC_DF64, v)
    sc = apply(op, dd.DD_OP_SC, dd.DD_PREC_DF64, full)
    for r in range(nrhs):
        assert rel(got[r], eo.Dhat(v[r])) < TOL[dd.DD_PREC_F64]
        assert rel(gotH[r], eo.DhatH(v[r])) < TOL[dd.DD_PREC_F64]
        ref = np.einsum("sij,sj->si", A, full[r].reshape(-1, 12))
        assert rel(sc[r], ref) < TOL[dd.DD_PREC_F64]


def test_native_layout_and_pack_roundtrip(system):
    """Native DF64 fields have the FP64 byte count; pack then unpack keeps
    about 48 bits; the native-layout apply equals the canonical one."""
    dims, U, A, op, _ = system
    psi = synthetic.spinor(dims, nrhs=2)
    x = torch.from_numpy(psi).cuda()
    nb = op.field_bytes(dd.DD_PREC_DF64, 0, 2)
    assert nb == op.field_bytes(dd.DD_PREC_F64, 0, 2)
    fi = torch.empty(nb, dtype=torch.uint8, device="cuda")
    fo = torch.empty_like(fi)
    op.pack(dd.DD_PREC_DF64, 0, x, fi, 2)
    back = torch.empty_like(x)
    op.unpack(dd.DD_PREC_DF64, 0, fi, back, 2)
    op.apply(dd.DD_OP_D, dd.DD_PREC_DF64, fi, fo, 2, dd.DD_LAYOUT_NATIVE)
    out = torch.empty_like(x)
    op.unpack(dd.DD_PREC_DF64, 0, fo, out, 2)
    torch.cuda.synchronize()
    assert rel(back.cpu().numpy(), psi) < 1e-14
    can = apply(op, dd.DD_OP_D, dd.DD_PREC_DF64, psi)
    assert np.array_equal(out.cpu().numpy(), can)


def test_rough_links_and_wide_value_range():
    """eps = 3 links and a spinor scaled by 1e6 and 1e-6 on alternate time
    slices: the pairs keep the relative accuracy across the range."""
    dims = (4, 4, 4, 4)
    U, lat, g, op = make_df(dims, eps=3.0)
    A = oracle.clover(U, dims, M0, CSW)
    psi = synthetic.spinor(dims, nrhs=1)
    t = np.arange(int(np.prod(dims))) // (dims[1] * dims[2] * dims[3])
    psi = psi * np.where(t % 2 == 0, 1e6, 1e-6)[None, :, None, None]
    got = apply(op, dd.DD_OP_D, dd.DD_PREC_DF64, psi)
    ref = oracle.apply_D(U, A, psi[0].reshape(-1, 12), dims)
    assert rel(got[0], ref) < TOL[dd.DD_PREC_F64]


def test_precision_checks():
    dims = (4, 4, 4, 4)
    U = synthetic.gauge(dims)
    lat = dd.Lattice(dims, -1)
    g = dd.Gauge(lat, U)  # no FP32-pair copies
    op = dd.Operator(g, M0, CSW)
    psi = synthetic.spinor(dims, nrhs=1)
    with pytest.raises(dd.DDError) as e:
        apply(op, dd.DD_OP_D, dd.DD_PREC_DF64, psi)
    assert e.value.status == dd.DD_ERR_UNSUPPORTED
    _, _, g2, op2 = make_df(dims)
    b = torch.from_numpy(psi).cuda()
    x = torch.zeros_like(b)
    with pytest.raises(dd.DDError) as e:
        op2.solve(b, x, 1, inner_prec=dd.DD_PREC_DF64, precond=dd.DD_PRECOND_SAP, sap_block=(2, 2, 2, 2))
    assert e.value.status == dd.DD_ERR_UNSUPPORTED
    assert g2.link_reals(dd.DD_PREC_DF64) == 18


@pytest.mark.parametrize("even_odd", [1, 0])
@pytest.mark.parametrize("precond", [dd.DD_PRECOND_NONE, dd.DD_PRECOND_CGNR])
def test_solve_with_pair_inner(even_odd, precond):
    """FGMRES with the FP32-pair stencil on FP64 vectors: one refinement
    step reaches 1e-10 (the inner operator is accurate to ~1e-14), the oracle
    recomputes the residual, and the solution matches the FP64 solve."""
    dims = (8, 8, 4, 4)
    U, lat, g, op = make_df(dims)
    A = oracle.clover(U, dims, M0, CSW)
    b = synthetic.spinor(dims, nrhs=1)
    bt = torch.from_numpy(b).cuda()
    xs = {}
    for inner in (dd.DD_PREC_DF64, dd.DD_PREC_F64):
        x = torch.zeros_like(bt)
        status, st = op.solve(bt, x, 1, tol=1e-10, inner_prec=inner, even_odd=even_odd, restart=16, precond=precond,
                              precond_iters=8)
        assert status == 0, st
        assert st["converged"] == 1 and st["true_residual"] < 1e-10
        xs[inner] = x.cpu().numpy()[0]
        res = b[0].reshape(-1, 12) - oracle.apply_D(U, A, xs[inner].reshape(-1, 12), dims)
        assert np.linalg.norm(res) / np.linalg.norm(b[0]) < 1e-10
        if inner == dd.DD_PREC_DF64:
            assert st["outer_iterations"] == 1
    assert rel(xs[dd.DD_PREC_DF64], xs[dd.DD_PREC_F64]) < 1e-8


@pytest.mark.parametrize("inner,precond,even_odd", [(dd.DD_PREC_F32, dd.DD_PRECOND_CGNR, 1),
                                                    (dd.DD_PREC_F16, dd.DD_PRECOND_CGNR16, 1),
                                                    (dd.DD_PREC_F32, dd.DD_PRECOND_CGNR, 0)])
def test_refinement_in_pair_arithmetic(inner, precond, even_odd):
    """refine_prec = DD_PREC_DF64: the refinement's r = b - D x (and the
    even-odd preparation and reconstruction) in FP32-pair arithmetic on the
    FP64 iterate.  The solve reaches 1e-10, certified by the oracle, and
    agrees with the FP64-refined solve."""
    dims = (8, 8, 4, 4)
    U, lat, g, op = make_df(dims)
    A = oracle.clover(U, dims, M0, CSW)
    b = synthetic.spinor(dims, nrhs=1)
    bt = torch.from_numpy(b).cuda()
    xs = {}
    for rp in (dd.DD_PREC_F64, dd.DD_PREC_DF64):
        x = torch.zeros_like(bt)
        status, st = op.solve(bt, x, 1, tol=1e-10, inner_prec=inner, even_odd=even_odd, restart=8, precond=precond,
                              precond_iters=16, inner_tol=1e-3 if inner == dd.DD_PREC_F16 else 1e-6,
                              refine_prec=rp)
        assert status == 0, st
        assert st["converged"] == 1 and st["true_residual"] < 1e-10
        xs[rp] = x.cpu().numpy()[0]
        res = b[0].reshape(-1, 12) - oracle.apply_D(U, A, xs[rp].reshape(-1, 12), dims)
        assert np.linalg.norm(res) / np.linalg.norm(b[0]) < 1e-10
    assert rel(xs[dd.DD_PREC_DF64], xs[dd.DD_PREC_F64]) < 1e-8


def test_refinement_precision_checks():
    dims = (4, 4, 4, 4)
    U = synthetic.gauge(dims)
    lat = dd.Lattice(dims, -1)
    g = dd.Gauge(lat, U)  # no FP32-pair copies
    op = dd.Operator(g, M0, CSW)
    b = torch.from_numpy(synthetic.spinor(dims, nrhs=1)).cuda()
    x = torch.zeros_like(b)
    with pytest.raises(dd.DDError) as e:
        op.solve(b, x, 1, refine_prec=dd.DD_PREC_DF64)
    assert e.value.status == dd.DD_ERR_UNSUPPORTED
    with pytest.raises(dd.DDError) as e:
        op.solve(b, x, 1, refine_prec=dd.DD_PREC_F32)
    assert e.value.status == dd.DD_ERR_ARG
