"""Domain decomposition (Sections 2.1, 2.2, Algorithm 3) on virtual ranks of
one GPU: the decomposed D, D^H, Dhat and Dhat^H against the single-domain
apply (bit for bit where both run the one-thread-per-(site, RHS) stencil)
and against the oracle; the allreduce of per-rank inner products against the
global inner product."""
import numpy as np
import pytest
import torch

import oracle
import synthetic
import paper_2407_00041_gb300 as dd
from tests._gpu import CSW, M0, TOL, make, rel

pytestmark = pytest.mark.gpu

OPS = [dd.DD_OP_D, dd.DD_OP_DH, dd.DD_OP_DHAT, dd.DD_OP_DHAT_H]


def _single_and_decomposed(op, dec, which, prec, psi, nrhs):
    """Native outputs of the single-domain apply and of the decomposed apply
    (gathered into the global native layout), as uint8 tensors."""
    subset = 1 if which in (dd.DD_OP_DHAT, dd.DD_OP_DHAT_H) else 0
    x = torch.from_numpy(np.ascontiguousarray(psi)).cuda()
    nb = op.field_bytes(prec, subset, nrhs)
    xi = torch.empty(nb, dtype=torch.uint8, device="cuda")
    op.pack(prec, subset, x, xi, nrhs)
    ref = torch.empty_like(xi)
    op.apply(which, prec, xi, ref, nrhs, dd.DD_LAYOUT_NATIVE)
    dec.scatter(prec, subset, xi, nrhs)
    dec.apply(which, prec, nrhs)
    got = torch.zeros_like(xi)
    dec.gather(prec, subset, got, nrhs)
    torch.cuda.synchronize()
    return xi, ref, got, subset


def _unpack(op, prec, subset, native, nrhs, nsites):
    out = torch.empty((nrhs, nsites, 12), dtype=torch.complex128, device="cuda")
    op.unpack(prec, subset, native, out, nrhs)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("dims,grid", [((8, 4, 4, 8), (2, 1, 1, 1)), ((8, 4, 4, 8), (1, 1, 1, 2)),
                                       ((8, 4, 4, 4), (2, 2, 1, 1)), ((4, 4, 8, 4), (1, 2, 2, 1)),
                                       ((8, 8, 8, 8), (2, 2, 2, 2)), ((4, 4, 4, 4), (1, 1, 1, 1))])
@pytest.mark.parametrize("prec", [dd.DD_PREC_F64, dd.DD_PREC_F32, dd.DD_PREC_F16])
def test_decomposed_equals_single_domain_bitwise(dims, grid, prec):
    U, lat, g, op = make(dims)
    dec = dd.Decomposition(op, grid)
    assert dec.nranks == int(np.prod(grid))
    for nrhs in (1, 3):
        psi = synthetic.spinor(dims, nrhs=nrhs).reshape(nrhs, -1, 12)
        for which in OPS:
            sub_psi = psi[:, oracle.eo_sites(dims)[1]] if which in (dd.DD_OP_DHAT, dd.DD_OP_DHAT_H) else psi
            _, ref, got, _ = _single_and_decomposed(op, dec, which, prec, sub_psi, nrhs)
            assert torch.equal(ref, got), (grid, prec, nrhs, which)


@pytest.mark.parametrize("prec", [dd.DD_PREC_F64, dd.DD_PREC_F32, dd.DD_PREC_F16])
def test_decomposed_against_oracle_two_rhs(prec):
    """Two right-hand sides (the RHS-blocked single-domain kernel rounds
    differently, so the reference here is the oracle)."""
    dims, grid = (8, 4, 4, 8), (2, 1, 2, 1)
    U, lat, g, op = make(dims)
    A = oracle.clover(U, dims, M0, CSW)
    dec = dd.Decomposition(op, grid)
    psi = synthetic.spinor(dims, nrhs=2).reshape(2, -1, 12)
    even, odd = oracle.eo_sites(dims)
    eo = oracle.EvenOdd(U, A, dims)
    for which in OPS:
        hat = which in (dd.DD_OP_DHAT, dd.DD_OP_DHAT_H)
        sub = psi[:, odd] if hat else psi
        _, _, got, subset = _single_and_decomposed(op, dec, which, prec, sub, 2)
        out = _unpack(op, prec, subset, got, 2, sub.shape[1])
        for r in range(2):
            if which == dd.DD_OP_D:
                ref = oracle.apply_D(U, A, psi[r], dims)
            elif which == dd.DD_OP_DH:
                ref = oracle.apply_DH(U, A, psi[r], dims)
            elif which == dd.DD_OP_DHAT:
                ref = eo.Dhat(sub[r])
            else:
                ref = eo.DhatH(sub[r])
            assert rel(out[r], ref) < TOL[prec], (which, r, rel(out[r], ref))


def test_decomposed_periodic_time_and_rank_geometry():
    dims, grid = (8, 4, 4, 4), (4, 1, 2, 1)
    U, lat, g, op = make(dims, t_bc=+1)
    dec = dd.Decomposition(op, grid)
    seen = set()
    for k in range(dec.nranks):
        inf = dec.info(k)
        assert inf["local"] == (2, 4, 2, 4)
        assert inf["offset"] == tuple(c * n for c, n in zip(inf["coord"], inf["local"]))
        seen.add(inf["coord"])
        # every site of a rank two sites thick in T touches a T seam
        assert inf["boundary_sites"] == 2 * 4 * 2 * 4
    assert len(seen) == dec.nranks
    psi = synthetic.spinor(dims, nrhs=1).reshape(1, -1, 12)
    _, ref, got, _ = _single_and_decomposed(op, dec, dd.DD_OP_D, dd.DD_PREC_F64, psi, 1)
    assert torch.equal(ref, got)
    A = oracle.clover(U, dims, M0, CSW)
    out = _unpack(op, dd.DD_PREC_F64, 0, got, 1, lat.V)
    assert rel(out[0], oracle.apply_D(U, A, psi[0], dims, t_bc=+1)) < 1e-13


def test_decomposed_dot_allreduce():
    dims, grid = (8, 4, 4, 8), (2, 2, 1, 1)
    U, lat, g, op = make(dims)
    dec = dd.Decomposition(op, grid)
    psi = synthetic.spinor(dims, nrhs=2).reshape(2, -1, 12)
    for prec in (dd.DD_PREC_F64, dd.DD_PREC_F32):
        xi, _, got, _ = _single_and_decomposed(op, dec, dd.DD_OP_D, prec, psi, 2)
        dots = dec.dot(prec, 0, 2)
        a = _unpack(op, prec, 0, got, 2, lat.V)
        b = _unpack(op, prec, 0, xi, 2, lat.V)
        for r in range(2):
            ref = np.vdot(a[r], b[r])
            tol = 1e-12 if prec == dd.DD_PREC_F64 else 1e-6  # FP32 fields are summed in FP32 per warp
            assert abs(dots[r] - ref) <= tol * abs(ref), (prec, r, dots[r], ref)


def test_decomposed_48c96_time_split_bitwise():
    """The 48^3 x 96 lattice split into 2 x 1 x 1 x 2 ranks, one RHS, FP32 and
    FP16 storage: bit-identical to the single-domain apply."""
    dims = (96, 48, 48, 48)
    lat = dd.Lattice(dims, -1)
    g = dd.Gauge.generate(lat)
    op = dd.Operator(g, M0, CSW)
    dec = dd.Decomposition(op, (2, 1, 1, 2))
    psi = synthetic.spinor(dims, nrhs=1).reshape(1, -1, 12)
    for prec in (dd.DD_PREC_F32, dd.DD_PREC_F16):
        for which in (dd.DD_OP_D, dd.DD_OP_DHAT):
            sub = psi[:, oracle.eo_sites(dims)[1]] if which == dd.DD_OP_DHAT else psi
            _, ref, got, _ = _single_and_decomposed(op, dec, which, prec, sub, 1)
            assert torch.equal(ref, got), (prec, which)
    del dec, op, g
    torch.cuda.empty_cache()


def test_decomposition_argument_checks():
    U, lat, g, op = make((4, 4, 4, 4))
    with pytest.raises(dd.DDError):
        dd.Decomposition(op, (3, 1, 1, 1))
    with pytest.raises(dd.DDError):
        dd.Decomposition(op, (4, 1, 1, 1))  # local extent 1
    dec = dd.Decomposition(op, (2, 1, 1, 1))
    with pytest.raises(dd.DDError):
        dec.apply(dd.DD_OP_D, dd.DD_PREC_F32, 1)  # nothing scattered yet
