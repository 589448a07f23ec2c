"""Parity at the full workload sizes, in the launch configuration bench.py
times (native layout, one full-lattice launch), on sampled outputs that the
oracle computes site by site: the 48^3 x 96 lattice at FP64 / FP32 / FP16
storage, the 32^4 lattice with 12 right-hand sides, and the batched launch of
8^4 x 1, 16^4 x 5, 24^4 x 17, 32^4 x 32.

Samples: the two boundary time slices (antiperiodic hops) plus random sites
of the whole lattice."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synthetic
import paper_2407_00041_gb300 as dd
from tests._gpu import CSW, M0, TOL, rel

pytestmark = pytest.mark.gpu

EPS = 0.3


def _sample(dims, nrand, seed):
    per = dims[1] * dims[2] * dims[3]
    V = int(np.prod(dims))
    rng = np.random.default_rng(seed)
    edge = np.concatenate([np.arange(per), np.arange(V - per, V)])
    return np.unique(np.concatenate([edge, rng.integers(0, V, nrand)])).astype(np.int64)


def _native_apply(op, prec, psi_dev, nrhs, which=dd.DD_OP_D):
    nb = op.field_bytes(prec, 0, nrhs)
    xi = torch.empty(nb, dtype=torch.uint8, device="cuda")
    xo = torch.empty_like(xi)
    op.pack(prec, 0, psi_dev, xi, nrhs)
    op.apply(which, prec, xi, xo, nrhs, dd.DD_LAYOUT_NATIVE)
    out = torch.empty_like(psi_dev)
    op.unpack(prec, 0, xo, out, nrhs)
    torch.cuda.synchronize()
    return out


def _check_sites(U, dims, psi_host, out_dev, sites, rhs, tol):
    A = oracle.clover_sites(U, dims, M0, CSW, sites)
    idx = torch.from_numpy(sites).cuda()
    for r in rhs:
        got = out_dev[r].reshape(-1, 12)[idx].cpu().numpy()
        ref = oracle.apply_D_sites(U, A, psi_host[r], dims, sites)
        assert rel(got, ref) < tol, (r, rel(got, ref))


def test_48c96_all_precisions_sampled():
    dims = (96, 48, 48, 48)
    U = synthetic.gauge(dims, eps=EPS)
    psi = synthetic.spinor(dims, nrhs=1)
    lat = dd.Lattice(dims, -1)
    g = dd.Gauge(lat, U)
    op = dd.Operator(g, M0, CSW)
    psi_dev = torch.from_numpy(psi).cuda()
    sites = _sample(dims, 20000, 1)
    for prec in (dd.DD_PREC_F64, dd.DD_PREC_F32, dd.DD_PREC_F16):
        out = _native_apply(op, prec, psi_dev, 1)
        _check_sites(U, dims, psi, out, sites, [0], TOL[prec])
        del out
    g.compress_links(8)  # the eight-real FP32 links rebuild within 1e-6 on all 42M links
    assert g.link_reals(dd.DD_PREC_F32) == 8
    out = _native_apply(op, dd.DD_PREC_F32, psi_dev, 1)
    _check_sites(U, dims, psi, out, sites, [0], TOL[dd.DD_PREC_F32])


def test_32c4_twelve_rhs_sampled():
    dims = (32, 32, 32, 32)
    n = 12
    U = synthetic.gauge(dims, eps=EPS)
    psi = synthetic.spinor(dims, nrhs=n)
    lat = dd.Lattice(dims, -1)
    g = dd.Gauge(lat, U)
    op = dd.Operator(g, M0, CSW)
    psi_dev = torch.from_numpy(psi).cuda()
    sites = _sample(dims, 5000, 2)
    for prec in (dd.DD_PREC_F32, dd.DD_PREC_F16):
        for which in (dd.DD_OP_D, dd.DD_OP_DH):
            out = _native_apply(op, prec, psi_dev, n, which)
            if which == dd.DD_OP_D:
                _check_sites(U, dims, psi, out, sites, range(n), TOL[prec])
            else:
                # D^H = gamma5 D gamma5 on the sampled sites
                g5 = psi.copy()
                g5[:, :, 2:] *= -1
                A = oracle.clover_sites(U, dims, M0, CSW, sites)
                idx = torch.from_numpy(sites).cuda()
                for r in (0, n - 1):
                    ref = oracle.apply_D_sites(U, A, g5[r], dims, sites).reshape(-1, 4, 3)
                    ref[:, 2:] *= -1
                    got = out[r].reshape(-1, 12)[idx].cpu().numpy()
                    assert rel(got, ref.reshape(-1, 12)) < TOL[prec]
            del out


def test_32c4_twelve_rhs_paired_layout_sampled():
    """The bench's multi-RHS launch: the paired-RHS layout at 32^4 x 12 (FP32,
    FP16 storage), D and D^H, sampled against the oracle; FP32 bit-identical
    to the native-layout apply on every site, FP16 (half2 colour products)
    within 2e-3 of it for every RHS."""
    dims = (32, 32, 32, 32)
    n = 12
    U = synthetic.gauge(dims, eps=EPS)
    psi = synthetic.spinor(dims, nrhs=n)
    lat = dd.Lattice(dims, -1)
    g = dd.Gauge(lat, U)
    op = dd.Operator(g, M0, CSW)
    psi_dev = torch.from_numpy(psi).cuda()
    sites = _sample(dims, 5000, 3)
    nb = op.field_bytes(dd.DD_PREC_F32, 0, n)
    xi = torch.empty(nb, dtype=torch.uint8, device="cuda")
    xo = torch.empty_like(xi)
    for prec in (dd.DD_PREC_F32, dd.DD_PREC_F16):
        for which in (dd.DD_OP_D, dd.DD_OP_DH):
            out = torch.empty_like(psi_dev)
            op.pack_paired(prec, 0, psi_dev, xi, n)
            op.apply(which, prec, xi, xo, n, dd.DD_LAYOUT_NATIVE_PAIRED)
            op.unpack_paired(prec, 0, xo, out, n)
            ref = _native_apply(op, prec, psi_dev, n, which)
            if prec == dd.DD_PREC_F32:
                assert torch.equal(out, ref)
            else:
                for r in range(n):
                    assert ((out[r] - ref[r]).norm() / ref[r].norm()).item() < 2e-3
            del ref
            if which == dd.DD_OP_D:
                _check_sites(U, dims, psi, out, sites, (0, 5, n - 1), TOL[prec])
            del out


def test_batch_of_uneven_lattices_full_size():
    shapes = [(8, 8, 8, 8), (16, 16, 16, 16), (24, 24, 24, 24), (32, 32, 32, 32)]
    nrhs = [1, 5, 17, 32]
    prec = dd.DD_PREC_F32
    keep, ops, ins, outs, refs, psis = [], [], [], [], [], []
    for dims, n in zip(shapes, nrhs):
        U = synthetic.gauge(dims, eps=EPS)
        lat = dd.Lattice(dims, -1)
        g = dd.Gauge(lat, U)
        op = dd.Operator(g, M0, CSW)
        keep.append((U, lat, g))
        ops.append(op)
        psi = synthetic.spinor(dims, nrhs=n)
        psis.append(psi)
        x = torch.from_numpy(psi).cuda()
        nb = op.field_bytes(prec, 0, n)
        xi = torch.empty(nb, dtype=torch.uint8, device="cuda")
        op.pack(prec, 0, x, xi, n)
        ins.append(xi)
        outs.append(torch.empty_like(xi))
        ref = torch.empty_like(xi)
        op.apply(dd.DD_OP_D, prec, xi, ref, n, dd.DD_LAYOUT_NATIVE)
        refs.append(ref)
        del x
    arr = lambda v, t=ctypes.c_void_p: (t * len(v))(*v)
    b = ctypes.c_void_p()
    dd.check(dd.lib.dd_batch_create(arr([o.h.value for o in ops]), len(ops), prec, arr(nrhs, ctypes.c_int),
                                    ctypes.byref(b)), "dd_batch_create")
    st = torch.cuda.current_stream().cuda_stream
    try:
        chosen = (ctypes.c_int * 3)()
        pin, pout = arr([x.data_ptr() for x in ins]), arr([x.data_ptr() for x in outs])
        dd.check(dd.lib.dd_batch_tune(b, pin, pout, st, chosen), "tune")
        dd.check(dd.lib.dd_apply_batched_graph(b, pin, pout, st), "graph")
        torch.cuda.synchronize()
    finally:
        dd.lib.dd_batch_destroy(b)
    for (U, lat, g), op, dims, n, o, r, psi in zip(keep, ops, shapes, nrhs, outs, refs, psis):
        uo = torch.empty((n, lat.V, 12), dtype=torch.complex128, device="cuda")
        ur = torch.empty_like(uo)
        op.unpack(prec, 0, o, uo, n)
        op.unpack(prec, 0, r, ur, n)
        torch.cuda.synchronize()
        assert ((uo - ur).norm() / ur.norm()).item() < 1e-6  # batched == single applies
        sites = _sample(dims, 2000, 3)
        _check_sites(U, dims, psi.reshape(n, -1, 12), uo, sites, sorted({0, n - 1}), TOL[prec])


@pytest.mark.parametrize("inner", [dd.DD_PREC_F32, dd.DD_PREC_F16])
def test_48c96_mixed_solve_oracle_residual_sampled(inner):
    """The bench's solve (even-odd FGMRES(8), 64 CG steps per preconditioner
    application, FP64 refinement) at full size; the oracle recomputes
    b - D x on sampled sites from the downloaded solution."""
    dims = (96, 48, 48, 48)
    U = synthetic.gauge(dims, eps=EPS)
    b = synthetic.spinor(dims, nrhs=1)
    lat = dd.Lattice(dims, -1)
    g = dd.Gauge(lat, U)
    op = dd.Operator(g, M0, CSW)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    status, st = op.solve(bd, x, 1, tol=1e-10, inner_prec=inner, restart=8, max_restarts=100, max_outer=10,
                          precond=dd.DD_PRECOND_CGNR, precond_iters=64)
    assert status == dd.DD_OK and st["true_residual"] < 1e-10
    xh = x.cpu().numpy()
    sites = _sample(dims, 20000, 4)
    A = oracle.clover_sites(U, dims, M0, CSW, sites)
    Dx = oracle.apply_D_sites(U, A, xh[0], dims, sites)
    bs = b[0].reshape(-1, 12)[sites]
    assert rel(Dx, bs) < 1e-10  # the solve's own tolerance, recomputed by the oracle on the sample


def test_48c96_fp16_cg_vectors_pair_refinement_oracle_residual_sampled():
    """The bench's fastest solve at full size: FP16 links and blocks inside,
    the CG vectors of M_j in FP16 (32 steps, inner tolerance 1e-3), the
    refinement's applications in FP32-pair arithmetic; the oracle
    recomputes b - D x on sampled sites from the downloaded solution."""
    dims = (96, 48, 48, 48)
    U = synthetic.gauge(dims, eps=EPS)
    b = synthetic.spinor(dims, nrhs=1)
    lat = dd.Lattice(dims, -1)
    precs = dd.DD_PREC_F64 | dd.DD_PREC_F32 | dd.DD_PREC_F16 | dd.DD_PREC_DF64
    g = dd.Gauge(lat, U, precisions=precs)
    op = dd.Operator(g, M0, CSW, precisions=precs)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    status, st = op.solve(bd, x, 1, tol=1e-10, inner_prec=dd.DD_PREC_F16, restart=8, max_restarts=100,
                          max_outer=20, precond=dd.DD_PRECOND_CGNR16, precond_iters=32, inner_tol=1e-3,
                          refine_prec=dd.DD_PREC_DF64)
    assert status == dd.DD_OK and st["true_residual"] < 1e-10, st
    xh = x.cpu().numpy()
    del op, g
    sites = _sample(dims, 20000, 5)
    A = oracle.clover_sites(U, dims, M0, CSW, sites)
    Dx = oracle.apply_D_sites(U, A, xh[0], dims, sites)
    bs = b[0].reshape(-1, 12)[sites]
    assert rel(Dx, bs) < 1e-10


def test_64c128_8rhs_mixed_solve_oracle_residual():
    """The 64^3 x 128 lattice with 8 Gaussian right-hand sides fitted in one
    GPU: FP64 and FP16 copies of links and self coupling only, b and x in host
    memory, right-hand sides in batches of 2, even-odd FGMRES(8) with 64 CG
    steps per preconditioner application, FP16 links / FP32 vectors inside and
    FP64 refinement to 1e-10.  The oracle recomputes ||b - D x|| / ||b|| on
    both boundary time slices of every right-hand side."""
    dims = (128, 64, 64, 64)
    N = 8
    V = int(np.prod(dims))
    lat = dd.Lattice(dims, -1)
    g = dd.Gauge.generate(lat, seed=synthetic.SEED_GAUGE, eps=EPS, precisions=dd.DD_PREC_F64 | dd.DD_PREC_F16)
    op = dd.Operator(g, M0, CSW, precisions=dd.DD_PREC_F64 | dd.DD_PREC_F16)
    b = synthetic.spinor(dims, nrhs=N)
    x = np.zeros_like(b)
    status, st = op.solve(b, x, N, layout=dd.DD_LAYOUT_CANONICAL_HOST, tol=1e-10, inner_prec=dd.DD_PREC_F16,
                          restart=8, rhs_batch=2, precond=dd.DD_PRECOND_CGNR, precond_iters=64, max_restarts=200,
                          max_outer=10)
    assert status == dd.DD_OK and st["converged"] == 1 and st["true_residual"] < 1e-10, st
    del op, g
    per = dims[1] * dims[2] * dims[3]
    sites = np.concatenate([np.arange(per), np.arange(V - per, V)]).astype(np.int64)
    U = np.empty((V, 4, 3, 3), dtype=np.complex128)  # only the four slices below are filled and read
    for t in (dims[0] - 2, dims[0] - 1, 0, 1):
        U[t * per:(t + 1) * per] = synthetic.gauge_sites(np.arange(t * per, (t + 1) * per), eps=EPS)
    A = oracle.clover_sites(U, dims, M0, CSW, sites)
    for r in range(N):
        Dx = oracle.apply_D_sites(U, A, x[r], dims, sites)
        bs = b[r].reshape(-1, 12)[sites]
        assert rel(Dx, bs) < 1e-10, (r, rel(Dx, bs))
