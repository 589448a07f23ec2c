"""GPU parity: the CUDA path against the CPU oracle, element by element.

Tolerances (relative L2): FP64 1e-13, FP32 1e-6, FP16 storage 5e-3.
Lattice shapes cover several 128-thread tiles with a ragged tail
(e.g. 6x4x2x8: 192 sites per parity), non-cubic shapes and extent 2.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
import paper_2407_00041_gb300 as dd
from tests._gpu import CSW, M0, TOL, apply, make, rel

pytestmark = pytest.mark.gpu

SHAPES = [(4, 4, 4, 4), (6, 4, 2, 8), (2, 2, 2, 2), (8, 6, 4, 2), (4, 8, 8, 8)]
PRECS = [dd.DD_PREC_F64, dd.DD_PREC_F32, dd.DD_PREC_F16]


def g5(psi):
    p = psi.reshape(psi.shape[0], -1, 4, 3).copy()
    p[:, :, 2:] *= -1
    return p


@pytest.fixture(scope="module", params=SHAPES, ids=lambda d: "x".join(map(str, d)))
def system(request):
    dims = request.param
    U, lat, g, op = make(dims)
    A = oracle.clover(U, dims, M0, CSW)
    return dims, U, A, op, (lat, g)


def test_clover_matches_oracle(system):
    dims, U, A, op, _ = system
    assert rel(op.clover_dense(), A) < 1e-13


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("nrhs", [1, 3, 4, 5, 6, 16])
def test_D_and_DH(system, prec, nrhs):
    dims, U, A, op, _ = system
    psi = synthetic.spinor(dims, nrhs=nrhs)
    got = apply(op, dd.DD_OP_D, prec, psi)
    gotH = apply(op, dd.DD_OP_DH, prec, psi)
    for r in range(nrhs):
        ref = oracle.apply_D(U, A, psi[r].reshape(-1, 12), dims)
        assert rel(got[r], ref) < TOL[prec]
        refH = oracle.apply_DH(U, A, psi[r].reshape(-1, 12), dims)
        assert rel(gotH[r], refH) < TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_self_coupling(system, prec):
    dims, U, A, op, _ = system
    psi = synthetic.spinor(dims, nrhs=2)
    got = apply(op, dd.DD_OP_SC, prec, psi)
    for r in range(2):
        ref = np.einsum("xij,xj->xi", A, psi[r].reshape(-1, 12))
        assert rel(got[r], ref) < TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("nrhs", [1, 2, 4, 5, 16])
def test_Dhat(system, prec, nrhs):
    dims, U, A, op, _ = system
    eo = oracle.EvenOdd(U, A, dims)
    full = synthetic.spinor(dims, nrhs=nrhs)
    v = np.stack([full[r].reshape(-1, 12)[eo.odd] for r in range(nrhs)])
    got = apply(op, dd.DD_OP_DHAT, prec, v)
    gotH = apply(op, dd.DD_OP_DHAT_H, prec, v)
    for r in range(nrhs):
        assert rel(got[r], eo.Dhat(v[r])) < TOL[prec]
        assert rel(gotH[r], eo.DhatH(v[r])) < TOL[prec]


def test_host_layout_roundtrip(system):
    dims, U, A, op, _ = system
    psi = synthetic.spinor(dims, nrhs=2)
    got = apply(op, dd.DD_OP_D, dd.DD_PREC_F64, psi, layout=dd.DD_LAYOUT_CANONICAL_HOST)
    for r in range(2):
        assert rel(got[r], oracle.apply_D(U, A, psi[r].reshape(-1, 12), dims)) < 1e-13


@pytest.mark.parametrize("prec", PRECS)
def test_pack_unpack_roundtrip(system, prec):
    dims, U, A, op, _ = system
    nrhs = 3
    psi = torch.from_numpy(synthetic.spinor(dims, nrhs=nrhs)).cuda()
    for subset, nsites in ((0, psi.shape[1]), (1, psi.shape[1] // 2)):
        x = psi[:, :nsites].contiguous()
        nat = torch.empty(op.field_bytes(prec, subset, nrhs), dtype=torch.uint8, device="cuda")
        back = torch.empty_like(x)
        op.pack(prec, subset, x, nat, nrhs)
        op.unpack(prec, subset, nat, back, nrhs)
        torch.cuda.synchronize()
        tol = {1: 0.0, 2: 1e-7, 4: 1e-3}[prec]
        assert rel(back.cpu().numpy(), x.cpu().numpy()) <= tol


def test_native_layout_matches_canonical(system):
    """The native-layout entry point (what the bench times) gives the same
    result as the canonical one, which takes the paired stencil for two RHS:
    exactly in FP64 and FP32, and within 2e-3 for FP16 storage (the paired FP16
    stencil forms its colour products in half2 arithmetic)."""
    dims, U, A, op, _ = system
    nrhs = 2
    psi = torch.from_numpy(synthetic.spinor(dims, nrhs=nrhs)).cuda()
    for prec in PRECS:
        nat_in = torch.empty(op.field_bytes(prec, 0, nrhs), dtype=torch.uint8, device="cuda")
        nat_out = torch.empty_like(nat_in)
        op.pack(prec, 0, psi, nat_in, nrhs)
        op.apply(dd.DD_OP_D, prec, nat_in, nat_out, nrhs, dd.DD_LAYOUT_NATIVE)
        out = torch.empty_like(psi)
        op.unpack(prec, 0, nat_out, out, nrhs)
        torch.cuda.synchronize()
        ref = apply(op, dd.DD_OP_D, prec, psi.cpu().numpy())
        assert rel(out.cpu().numpy(), ref) <= (2e-3 if prec == dd.DD_PREC_F16 else 0.0)


def test_periodic_time_boundary():
    dims = (4, 2, 4, 2)
    U, lat, g, op = make(dims, t_bc=+1)
    A = oracle.clover(U, dims, M0, CSW)
    psi = synthetic.spinor(dims)
    got = apply(op, dd.DD_OP_D, dd.DD_PREC_F64, psi)
    assert rel(got[0], oracle.apply_D(U, A, psi[0].reshape(-1, 12), dims, t_bc=+1)) < 1e-13


def test_gamma5_hermiticity_on_gpu(system):
    dims, U, A, op, _ = system
    psi = synthetic.spinor(dims, seed=31)
    phi = synthetic.spinor(dims, seed=32)
    Dpsi = apply(op, dd.DD_OP_D, dd.DD_PREC_F64, psi)
    DHphi = apply(op, dd.DD_OP_DH, dd.DD_PREC_F64, phi)
    lhs = np.vdot(phi, Dpsi)
    assert abs(lhs - np.vdot(DHphi, psi)) / abs(lhs) < 1e-13
    assert rel(DHphi, g5(apply(op, dd.DD_OP_D, dd.DD_PREC_F64, g5(phi)))) < 1e-13


def test_free_field_plane_wave_on_gpu():
    dims = (8, 4, 4, 4)
    V = int(np.prod(dims))
    U = np.broadcast_to(np.eye(3, dtype=np.complex128), (V, 4, 3, 3)).copy()
    _, lat, g, op = make(dims, U=U)
    coords = np.array(np.unravel_index(np.arange(V), dims)).T
    p = np.array([np.pi * 3 / dims[0], 2 * np.pi / dims[1], 4 * np.pi / dims[2], 0.0])
    u = synthetic.gaussian(12, seed=5)
    phase = np.exp(1j * coords @ p)
    psi = (phase[:, None] * u[None, :])[None]
    gam = [oracle.gamma(mu) for mu in range(4)]
    Dp = (M0 + np.sum(1 - np.cos(p))) * np.eye(4) + sum(1j * np.sin(p[m]) * gam[m] for m in range(4))
    expect = phase[:, None] * (np.kron(Dp, np.eye(3)) @ u)[None, :]
    assert rel(apply(op, dd.DD_OP_D, dd.DD_PREC_F64, psi)[0], expect) < 1e-13


def test_zero_input_gives_zero_fp16():
    dims = (4, 4, 2, 2)
    U, lat, g, op = make(dims)
    psi = np.zeros((1, int(np.prod(dims)), 4, 3), dtype=np.complex128)
    assert np.all(apply(op, dd.DD_OP_D, dd.DD_PREC_F16, psi) == 0)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("dims", [(8, 4, 4, 4), (6, 4, 2, 8), (2, 4, 4, 2)], ids=lambda d: "x".join(map(str, d)))
def test_host_layout_pipelined_equals_device(dims, prec):
    """D and D^H on host buffers run chunk-pipelined over time slices (copies
    overlapped with the stencil); every output equals the device-buffer
    apply bit for bit."""
    U, lat, g, op = make(dims)
    psi = synthetic.spinor(dims, nrhs=3)
    for which in (dd.DD_OP_D, dd.DD_OP_DH):
        host = apply(op, which, prec, psi, layout=dd.DD_LAYOUT_CANONICAL_HOST)
        dev = apply(op, which, prec, psi)
        assert np.array_equal(host, dev)


def test_two_row_links_and_non_su3_fallback():
    """SU(3) links: single-RHS FP32 and FP16 applies read two-row copies and
    rebuild the third row; links that are not SU(3) get no two-row copy.  Both
    match the oracle, which uses the links as given."""
    dims = (6, 4, 2, 8)
    U = synthetic.gauge(dims)
    _, lat, g, op = make(dims, U=U)
    assert dd.lib.dd_gauge_stored_rows(g.h, dd.DD_PREC_F32) == 2
    assert dd.lib.dd_gauge_stored_rows(g.h, dd.DD_PREC_F16) == 2
    assert dd.lib.dd_gauge_stored_rows(g.h, dd.DD_PREC_F64) == 3
    assert g.link_reals(dd.DD_PREC_F16) == 12
    # a non-unitary perturbation of every link
    W = U * (1.0 + 0.01 * synthetic.gaussian(U.size, seed=9).real.reshape(U.shape))
    _, lat2, g2, op2 = make(dims, U=W)
    assert dd.lib.dd_gauge_stored_rows(g2.h, dd.DD_PREC_F32) == 3
    assert dd.lib.dd_gauge_stored_rows(g2.h, dd.DD_PREC_F16) == 3
    psi = synthetic.spinor(dims, nrhs=1)  # one RHS: the launches that read the two-row copies
    for links, o in ((U, op), (W, op2)):
        A = oracle.clover(links, dims, M0, CSW)
        for prec in (dd.DD_PREC_F32, dd.DD_PREC_F16):
            for which, ref_fn in ((dd.DD_OP_D, oracle.apply_D), (dd.DD_OP_DH, oracle.apply_DH)):
                got = apply(o, which, prec, psi)
                assert rel(got[0], ref_fn(links, A, psi[0].reshape(-1, 12), dims)) < TOL[prec]


def test_fp16_two_row_against_three_row():
    """FP16 single-RHS D, D^H and Dhat from the two-row copy (row 2 from
    exact products of the stored halves, rounded once) against the three-row
    FP16 links of the same handle and the oracle; the rebuilt row differs from
    the stored one by FP16 rounding only."""
    dims = (4, 8, 8, 8)
    U = synthetic.gauge(dims, eps=1.0)
    _, lat, g, op = make(dims, U=U)
    A = oracle.clover(U, dims, M0, CSW)
    eo = oracle.EvenOdd(U, A, dims)
    psi = synthetic.spinor(dims, nrhs=1)
    v = psi[0].reshape(-1, 12)[eo.odd][None]
    got = {}
    for reals in (12, 18):
        g.compress_links(reals, dd.DD_PREC_F16)
        assert g.link_reals(dd.DD_PREC_F16) == reals
        got[reals] = [apply(op, w, dd.DD_PREC_F16, psi) for w in (dd.DD_OP_D, dd.DD_OP_DH)] + \
                     [apply(op, w, dd.DD_PREC_F16, v) for w in (dd.DD_OP_DHAT, dd.DD_OP_DHAT_H)]
        refs = [oracle.apply_D(U, A, psi[0].reshape(-1, 12), dims), oracle.apply_DH(U, A, psi[0].reshape(-1, 12), dims),
                eo.Dhat(v[0]), eo.DhatH(v[0])]
        for a, b in zip(got[reals], refs):
            assert rel(a[0], b) < TOL[dd.DD_PREC_F16]
    for a, b in zip(got[12], got[18]):
        assert rel(a, b) < 2e-3


@pytest.mark.parametrize("eps", [0.3, 1.0, 3.0])
def test_eight_real_fp32_links(eps):
    """The eight-real FP32 copy (column shift, row swap and phases in two
    float4 words per link): single-RHS D, D^H and Dhat match the oracle at the
    FP32 tolerance for smooth and rough SU(3) fields (eps = 1 and 3 take all
    three column shifts); switching back to 12 and 18 reals reproduces the
    two-row and three-row results."""
    dims = (6, 4, 2, 8)
    U = synthetic.gauge(dims, eps=eps)
    _, lat, g, op = make(dims, U=U)
    assert g.link_reals(dd.DD_PREC_F32) == 12 and g.link_reals(dd.DD_PREC_F64) == 18
    psi = synthetic.spinor(dims, nrhs=1)
    A = oracle.clover(U, dims, M0, CSW)
    ref12 = {w: apply(op, w, dd.DD_PREC_F32, psi) for w in (dd.DD_OP_D, dd.DD_OP_DH)}
    g.compress_links(8)
    assert g.link_reals(dd.DD_PREC_F32) == 8
    assert dd.lib.dd_gauge_stored_rows(g.h, dd.DD_PREC_F32) == 3
    for which, ref_fn in ((dd.DD_OP_D, oracle.apply_D), (dd.DD_OP_DH, oracle.apply_DH)):
        got = apply(op, which, dd.DD_PREC_F32, psi)
        assert rel(got[0], ref_fn(U, A, psi[0].reshape(-1, 12), dims)) < TOL[dd.DD_PREC_F32]
        assert rel(got, ref12[which]) < 1e-6
        assert not np.array_equal(got, ref12[which])  # the rebuilt links differ in the last bits
    eo = oracle.EvenOdd(U, A, dims)
    v = psi[0].reshape(-1, 12)[eo.odd][None]
    for which, ref_fn in ((dd.DD_OP_DHAT, eo.Dhat), (dd.DD_OP_DHAT_H, eo.DhatH)):
        got = apply(op, which, dd.DD_PREC_F32, v)
        assert rel(got[0], ref_fn(v[0])) < TOL[dd.DD_PREC_F32]
    g.compress_links(12)
    assert g.link_reals(dd.DD_PREC_F32) == 12
    assert np.array_equal(apply(op, dd.DD_OP_D, dd.DD_PREC_F32, psi), ref12[dd.DD_OP_D])
    g.compress_links(18)
    assert g.link_reals(dd.DD_PREC_F32) == 18
    got = apply(op, dd.DD_OP_D, dd.DD_PREC_F32, psi)
    assert rel(got[0], oracle.apply_D(U, A, psi[0].reshape(-1, 12), dims)) < TOL[dd.DD_PREC_F32]


def test_eight_real_needs_su3_links_and_valid_forms():
    dims = (4, 4, 2, 4)
    U = synthetic.gauge(dims)
    W = U * (1.0 + 0.01 * synthetic.gaussian(U.size, seed=9).real.reshape(U.shape))
    _, lat, g, op = make(dims, U=W)
    assert g.link_reals(dd.DD_PREC_F32) == 18
    for reals in (8, 12):
        with pytest.raises(dd.DDError) as e:
            g.compress_links(reals)
        assert e.value.status == dd.DD_ERR_UNSUPPORTED
        assert g.link_reals(dd.DD_PREC_F32) == 18
    _, lat2, g2, op2 = make(dims, U=U)
    for reals, prec in ((0, dd.DD_PREC_F32), (9, dd.DD_PREC_F32), (16, dd.DD_PREC_F16), (12, dd.DD_PREC_F64)):
        with pytest.raises(dd.DDError) as e:
            g2.compress_links(reals, prec)
        assert e.value.status == dd.DD_ERR_ARG
    with pytest.raises(dd.DDError) as e:
        g2.compress_links(8, dd.DD_PREC_F16)
    assert e.value.status == dd.DD_ERR_UNSUPPORTED
    assert g2.link_reals(dd.DD_PREC_F32) == 12 and g2.link_reals(dd.DD_PREC_F16) == 12
    g64 = dd.Gauge(lat2, U, precisions=dd.DD_PREC_F64)
    with pytest.raises(dd.DDError) as e:
        g64.compress_links(8)
    assert e.value.status == dd.DD_ERR_UNSUPPORTED


def native_apply(op, which, prec, psi):
    """The apply on the native layout (pack, apply, unpack)."""
    nrhs = psi.shape[0]
    subset = 1 if which in (dd.DD_OP_DHAT, dd.DD_OP_DHAT_H) else 0
    x = torch.from_numpy(np.ascontiguousarray(psi)).cuda()
    nb = op.field_bytes(prec, subset, nrhs)
    fi = torch.empty(nb, dtype=torch.uint8, device="cuda")
    fo = torch.empty_like(fi)
    op.pack(prec, subset, x, fi, nrhs)
    op.apply(which, prec, fi, fo, nrhs, dd.DD_LAYOUT_NATIVE)
    out = torch.empty_like(x)
    op.unpack(prec, subset, fo, out, nrhs)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("prec", [dd.DD_PREC_F32, dd.DD_PREC_F16])
def test_complex64_canonical_layouts(prec):
    """complex64 canonical fields on the device and on the host (pipelined
    for D and D^H): the results equal the native-layout applies of the same
    (complex64-representable) input, rounded to complex64, bit for bit.
    (complex128 canonical fields with an even RHS count take the paired
    stencil, whose FP16 form rounds differently, so the reference is the
    native layout.)"""
    dims = (6, 4, 2, 8)
    U, lat, g, op = make(dims)
    A = oracle.clover(U, dims, M0, CSW)
    eo = oracle.EvenOdd(U, A, dims)
    for nrhs in (1, 2):
        psi = synthetic.spinor(dims, nrhs=nrhs).astype(np.complex64)
        half = np.ascontiguousarray(np.stack([psi[r].reshape(-1, 12)[eo.odd] for r in range(nrhs)]))
        for which in (dd.DD_OP_D, dd.DD_OP_DH, dd.DD_OP_DHAT, dd.DD_OP_DHAT_H, dd.DD_OP_SC):
            x = half if which in (dd.DD_OP_DHAT, dd.DD_OP_DHAT_H) else psi
            ref = native_apply(op, which, prec, x.astype(np.complex128)).astype(np.complex64)
            xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
            od = torch.empty_like(xd)
            op.apply(which, prec, xd, od, nrhs, dd.DD_LAYOUT_CANONICAL_C64)
            oh = np.empty_like(x)
            op.apply(which, prec, np.ascontiguousarray(x), oh, nrhs, dd.DD_LAYOUT_CANONICAL_HOST_C64)
            torch.cuda.synchronize()
            assert np.array_equal(od.cpu().numpy(), ref.reshape(od.shape))
            assert np.array_equal(oh, ref.reshape(oh.shape))


def test_singular_self_coupling_and_empty_calls():
    """Degenerate cases.  Unit links make the clover term of Eq. 1.11 vanish
    (every plaquette is 1), so each 6x6 block is (4 + m0) 1: at m0 = -4 the
    blocks are zero and creating the operator reports DD_ERR_SINGULAR (no
    inverse is formed); at m0 = -3.5 the self coupling is 0.5 psi exactly.
    An apply or solve of zero right-hand sides is an argument error."""
    dims = (4, 4, 2, 2)
    V = int(np.prod(dims))
    U = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    U[:] = np.eye(3)
    lat = dd.Lattice(dims, -1)
    g = dd.Gauge(lat, U)
    with pytest.raises(dd.DDError) as e:
        dd.Operator(g, -4.0, CSW)
    assert e.value.status == dd.DD_ERR_SINGULAR
    op = dd.Operator(g, -3.5, CSW)
    psi = synthetic.spinor(dims, nrhs=1)
    for prec in (dd.DD_PREC_F64, dd.DD_PREC_F32):
        sc = apply(op, dd.DD_OP_SC, prec, psi)
        assert rel(sc, 0.5 * psi.reshape(sc.shape)) < TOL[prec]
    x = torch.from_numpy(psi).cuda()
    y = torch.empty_like(x)
    with pytest.raises(dd.DDError) as e:
        op.apply(dd.DD_OP_D, dd.DD_PREC_F64, x, y, 0)
    assert e.value.status == dd.DD_ERR_ARG
    with pytest.raises(dd.DDError) as e:
        op.solve(x, y, 0)
    assert e.value.status == dd.DD_ERR_ARG
