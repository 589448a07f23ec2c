"""GPU SAP smoother (red-black multiplicative Schwarz with minimal-residual
block solves, Section 1.3's smoother) through the C ABI, against the oracle's
restatement in oracle/sap.py; and SAP as the flexible preconditioner M_j of the
solver (Algorithm 2), certified by the oracle's residual.

Tolerances: FP64 1e-12 (rounding of a few MR steps), FP32 2e-5, FP16 links
and blocks with FP32 vectors 5e-3 (relative L2 of z = M^{-1} v).  Block shapes
cover 16 sites (a partial warp), 32, 64 and 256 sites and non-cubic blocks."""
import numpy as np
import pytest
import torch

import oracle
import synthetic
import paper_2407_00041_gb300 as dd
from oracle import sap as osap
from tests._gpu import CSW, M0, make, rel

pytestmark = pytest.mark.gpu

TOL = {dd.DD_PREC_F64: 1e-12, dd.DD_PREC_F32: 2e-5, dd.DD_PREC_F16: 5e-3}
CASES = [
    ((4, 4, 4, 4), (2, 2, 2, 2)),  # 16 sites per block: one partial warp
    ((4, 8, 4, 8), (2, 4, 2, 2)),
    ((8, 8, 4, 4), (4, 4, 2, 2)),
    ((8, 8, 8, 8), (4, 4, 4, 4)),
]


@pytest.fixture(scope="module", params=CASES, ids=lambda c: "x".join(map(str, c[0])) + "_b" + "x".join(map(str, c[1])))
def case(request):
    dims, block = request.param
    U, lat, g, op = make(dims)
    A = oracle.clover(U, dims, M0, CSW)
    return dims, block, U, A, op, (lat, g)


def _oracle_sap(U, A, dims, v, block, cycles, mr):
    apply = lambda x: oracle.apply_D(U, A, x.reshape(-1, 12), dims)
    return osap.sap(apply, dims, v.reshape(-1, 12), block, cycles, mr)


@pytest.mark.parametrize("prec", [dd.DD_PREC_F64, dd.DD_PREC_F32, dd.DD_PREC_F16])
@pytest.mark.parametrize("cycles,mr", [(1, 1), (1, 3), (2, 2)])
def test_sap_matches_oracle(case, prec, cycles, mr):
    dims, block, U, A, op, _ = case
    if int(np.prod(dims)) > 4096 and (cycles, mr) != (1, 3):
        pytest.skip("the oracle's block loop is slow on the largest lattice; one setting there")
    n = 2
    v = synthetic.spinor(dims, nrhs=n)
    x = torch.from_numpy(v).cuda()
    z = torch.empty_like(x)
    op.sap(prec, block, cycles, mr, x, z, n)
    torch.cuda.synchronize()
    got = z.cpu().numpy()
    for r in range(n):
        ref = _oracle_sap(U, A, dims, v[r], block, cycles, mr)
        assert rel(got[r].reshape(-1, 12), ref) < TOL[prec], (r, rel(got[r].reshape(-1, 12), ref))


def test_sap_native_equals_canonical(case):
    dims, block, U, A, op, _ = case
    n = 3
    v = synthetic.spinor(dims, nrhs=n)
    x = torch.from_numpy(v).cuda()
    zc = torch.empty_like(x)
    op.sap(dd.DD_PREC_F64, block, 1, 2, x, zc, n)
    nb = op.field_bytes(dd.DD_PREC_F64, 0, n)
    fi = torch.empty(nb, dtype=torch.uint8, device="cuda")
    fo = torch.empty_like(fi)
    op.pack(dd.DD_PREC_F64, 0, x, fi, n)
    op.sap(dd.DD_PREC_F64, block, 1, 2, fi, fo, n, dd.DD_LAYOUT_NATIVE)
    zn = torch.empty_like(x)
    op.unpack(dd.DD_PREC_F64, 0, fo, zn, n)
    torch.cuda.synchronize()
    assert torch.equal(zc, zn)


def test_sap_reduces_the_residual(case):
    """One exact property of the method without the oracle: every MR step
    minimises the block residual, so ||v - D z|| < ||v|| after a cycle."""
    dims, block, U, A, op, _ = case
    v = synthetic.spinor(dims, nrhs=1)
    x = torch.from_numpy(v).cuda()
    z = torch.empty_like(x)
    op.sap(dd.DD_PREC_F64, block, 1, 4, x, z, 1)
    torch.cuda.synchronize()
    zz = z.cpu().numpy()[0].reshape(-1, 12)
    res = v[0].reshape(-1, 12) - oracle.apply_D(U, A, zz, dims)
    assert np.linalg.norm(res) < 0.9 * np.linalg.norm(v[0])


def test_sap_argument_checks(case):
    dims, block, U, A, op, _ = case
    x = torch.zeros((1, int(np.prod(dims)), 12), dtype=torch.complex128, device="cuda")
    z = torch.empty_like(x)
    for bad in ((dims[0], 2, 2, 2), (3, 2, 2, 2), (0, 2, 2, 2)):
        with pytest.raises(dd.DDError) as e:
            op.sap(dd.DD_PREC_F64, bad, 1, 1, x, z, 1)
        assert e.value.status == dd.DD_ERR_ARG
    with pytest.raises(dd.DDError) as e:
        op.sap(dd.DD_PREC_F64, block, 0, 1, x, z, 1)
    assert e.value.status == dd.DD_ERR_ARG


@pytest.mark.parametrize("inner", [dd.DD_PREC_F64, dd.DD_PREC_F32, dd.DD_PREC_F16])
@pytest.mark.parametrize("even_odd", [1, 0])
def test_solve_with_sap_preconditioner(inner, even_odd):
    dims, block = (8, 8, 8, 8), (4, 4, 2, 2)
    U, lat, g, op = make(dims)
    A = oracle.clover(U, dims, M0, CSW)
    b = synthetic.spinor(dims, nrhs=2)
    bt = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bt)
    status, st = op.solve(bt, x, 2, tol=1e-10, inner_prec=inner, even_odd=even_odd, restart=16,
                          precond=dd.DD_PRECOND_SAP, sap_block=block, sap_cycles=2, sap_mr_steps=4)
    assert status == 0, st
    assert st["converged"] == 1 and st["true_residual"] < 1e-10
    xn = x.cpu().numpy()
    for r in range(2):
        res = b[r].reshape(-1, 12) - oracle.apply_D(U, A, xn[r].reshape(-1, 12), dims)
        assert np.linalg.norm(res) / np.linalg.norm(b[r]) < 1e-10


def test_sap_preconditioner_needs_fewer_arnoldi_steps():
    """The smoother does its job inside Algorithm 2: on the same system the
    SAP-preconditioned solve takes fewer Arnoldi steps than M = I."""
    dims, block = (8, 8, 8, 8), (4, 4, 2, 2)
    U, lat, g, op = make(dims)
    b = torch.from_numpy(synthetic.spinor(dims, nrhs=1)).cuda()
    steps = {}
    for pc in (dd.DD_PRECOND_NONE, dd.DD_PRECOND_SAP):
        x = torch.zeros_like(b)
        status, st = op.solve(b, x, 1, tol=1e-10, inner_prec=dd.DD_PREC_F32, even_odd=1, restart=16, precond=pc,
                              sap_block=block, sap_cycles=2, sap_mr_steps=4, max_restarts=400)
        if pc == dd.DD_PRECOND_SAP:
            assert status == 0, st
        steps[pc] = st["inner_iterations"]
    assert steps[dd.DD_PRECOND_SAP] < steps[dd.DD_PRECOND_NONE], steps
