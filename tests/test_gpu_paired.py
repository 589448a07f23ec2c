"""The paired-RHS layout and its packed stencil, through the C ABI.

With FP32 vectors every arithmetic step of one right-hand side in the paired
stencil is the FP32 operation of the native-layout RHS-blocked stencil, in the
same order, so the two layouts must give bit-identical results (compared here
exactly, after unpacking both to the canonical layout).  With FP16 vectors the
paired stencil forms the spin projection and colour products in half2
arithmetic (FP16 sums) where the native one widens to FP32 first: the two
agree to PAIR16_TOL.  The oracle checks the values to the stated tolerances
(FP32 1e-6, FP16 storage 5e-3).  Shapes span several 128-thread tiles with a
ragged tail (6x4x2x8: 192 sites per parity; with 6 pairs per site, 1152
threads per parity)."""
import numpy as np
import pytest
import torch

import oracle
import synthetic
import paper_2407_00041_gb300 as dd
from tests._gpu import CSW, M0, TOL, make, rel

pytestmark = pytest.mark.gpu

SHAPES = [(4, 4, 4, 4), (6, 4, 2, 8), (2, 2, 2, 2), (8, 6, 4, 2)]
PRECS = [dd.DD_PREC_F32, dd.DD_PREC_F16]
OPS = [dd.DD_OP_D, dd.DD_OP_DH, dd.DD_OP_DHAT, dd.DD_OP_DHAT_H]
# FP16 paired (half2 colour products) against FP16 native (FP32 colour
# products), relative L2 distance: both round their output to FP16 (2.4e-4),
# the FP16 sums add about 3e-4 per colour product
PAIR16_TOL = 2e-3


@pytest.fixture(scope="module", params=SHAPES, ids=lambda d: "x".join(map(str, d)))
def system(request):
    dims = request.param
    U, lat, g, op = make(dims)
    A = oracle.clover(U, dims, M0, CSW)
    return dims, U, A, op, (lat, g)


def _run(op, which, prec, psi_dev, nrhs, paired):
    subset = 1 if which in (dd.DD_OP_DHAT, dd.DD_OP_DHAT_H) else 0
    nb = op.field_bytes(prec, subset, nrhs)
    xi = torch.empty(nb, dtype=torch.uint8, device="cuda")
    xo = torch.full_like(xi, 0xFF)  # NaN bytes: every output word must be written
    out = torch.empty_like(psi_dev)
    if paired:
        op.pack_paired(prec, subset, psi_dev, xi, nrhs)
        op.apply(which, prec, xi, xo, nrhs, dd.DD_LAYOUT_NATIVE_PAIRED)
        op.unpack_paired(prec, subset, xo, out, nrhs)
    else:
        op.pack(prec, subset, psi_dev, xi, nrhs)
        op.apply(which, prec, xi, xo, nrhs, dd.DD_LAYOUT_NATIVE)
        op.unpack(prec, subset, xo, out, nrhs)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("nrhs", [2, 4, 12])
@pytest.mark.parametrize("which", OPS)
def test_paired_equals_native(system, prec, nrhs, which):
    dims, U, A, op, _ = system
    full = synthetic.spinor(dims, nrhs=nrhs).reshape(nrhs, -1, 12)
    if which in (dd.DD_OP_DHAT, dd.DD_OP_DHAT_H):
        eo = oracle.EvenOdd(U, A, dims)
        psi = np.ascontiguousarray(full[:, eo.odd])
    else:
        psi = full
    x = torch.from_numpy(psi).cuda()
    got = _run(op, which, prec, x, nrhs, True)
    ref = _run(op, which, prec, x, nrhs, False)
    assert np.isfinite(got).all()
    if prec == dd.DD_PREC_F32:
        assert np.array_equal(got, ref)
    else:
        for r in range(nrhs):
            assert rel(got[r], ref[r]) < PAIR16_TOL
        assert not np.array_equal(got, ref)  # the half2 path ran


@pytest.mark.parametrize("prec", PRECS)
def test_paired_against_oracle(system, prec):
    dims, U, A, op, _ = system
    n = 6
    psi = synthetic.spinor(dims, nrhs=n).reshape(n, -1, 12)
    x = torch.from_numpy(psi).cuda()
    got = _run(op, dd.DD_OP_D, prec, x, n, True)
    gotH = _run(op, dd.DD_OP_DH, prec, x, n, True)
    eo = oracle.EvenOdd(U, A, dims)
    v = np.ascontiguousarray(psi[:, eo.odd])
    gotS = _run(op, dd.DD_OP_DHAT, prec, torch.from_numpy(v).cuda(), n, True)
    for r in range(n):
        assert rel(got[r], oracle.apply_D(U, A, psi[r], dims)) < TOL[prec]
        assert rel(gotH[r], oracle.apply_DH(U, A, psi[r], dims)) < TOL[prec]
        assert rel(gotS[r], eo.Dhat(v[r])) < TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("subset", [0, 1, 2])
def test_pack_roundtrip_matches_native(system, prec, subset):
    dims, U, A, op, _ = system
    n = 4
    V = int(np.prod(dims))
    ns = V if subset == 0 else V // 2
    psi = synthetic.spinor(dims, nrhs=n).reshape(n, -1, 12)[:, :ns]
    x = torch.from_numpy(np.ascontiguousarray(psi)).cuda()
    nb = op.field_bytes(prec, 0 if subset == 0 else 1, n)
    f = torch.empty(nb, dtype=torch.uint8, device="cuda")
    a = torch.empty_like(x)
    b = torch.empty_like(x)
    op.pack_paired(prec, subset, x, f, n)
    op.unpack_paired(prec, subset, f, a, n)
    op.pack(prec, subset, x, f, n)
    op.unpack(prec, subset, f, b, n)
    torch.cuda.synchronize()
    assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())
    if prec == dd.DD_PREC_F32:
        assert np.array_equal(a.cpu().numpy(), psi.astype(np.complex64).astype(np.complex128))


def test_zero_input_gives_zero(system):
    dims, U, A, op, _ = system
    n = 2
    x = torch.zeros((n, int(np.prod(dims)), 12), dtype=torch.complex128, device="cuda")
    for prec in PRECS:
        got = _run(op, dd.DD_OP_D, prec, x, n, True)
        assert not np.any(got)


def test_paired_argument_checks(system):
    dims, U, A, op, _ = system
    V = int(np.prod(dims))
    nb = op.field_bytes(dd.DD_PREC_F32, 0, 4)
    f = torch.empty(nb, dtype=torch.uint8, device="cuda")
    g = torch.empty_like(f)
    x = torch.zeros((3, V, 12), dtype=torch.complex128, device="cuda")
    with pytest.raises(dd.DDError) as e:
        op.apply(dd.DD_OP_D, dd.DD_PREC_F32, f, g, 3, dd.DD_LAYOUT_NATIVE_PAIRED)
    assert e.value.status == dd.DD_ERR_ARG
    with pytest.raises(dd.DDError) as e:
        op.apply(dd.DD_OP_D, dd.DD_PREC_F64, f, g, 2, dd.DD_LAYOUT_NATIVE_PAIRED)
    assert e.value.status == dd.DD_ERR_ARG
    with pytest.raises(dd.DDError) as e:
        op.apply(dd.DD_OP_SC, dd.DD_PREC_F32, f, g, 2, dd.DD_LAYOUT_NATIVE_PAIRED)
    assert e.value.status == dd.DD_ERR_UNSUPPORTED
    with pytest.raises(dd.DDError) as e:
        op.pack_paired(dd.DD_PREC_F32, 0, x, f, 3)
    assert e.value.status == dd.DD_ERR_ARG
    with pytest.raises(dd.DDError) as e:
        op.pack_paired(dd.DD_PREC_F64, 0, x, f, 2)
    assert e.value.status == dd.DD_ERR_ARG
