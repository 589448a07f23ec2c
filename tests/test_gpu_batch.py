"""Batched uneven lattices in one persistent launch (plus autotune and CUDA
graph replay) against per-lattice applies and the CPU oracle."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synthetic
import paper_2407_00041_gb300 as dd
from tests._gpu import CSW, M0, TOL, make, rel

pytestmark = pytest.mark.gpu


def _arr(vals, t=ctypes.c_void_p):
    return (t * len(vals))(*vals)


def _close(op, prec, a, b, n):
    """Batched and single applies may run different kernel bodies (blocks of
    RHS, row staging), so they agree to the rounding of the storage format."""
    shape = (n, op.lattice.V, 12)
    ua = torch.empty(shape, dtype=torch.complex128, device="cuda")
    ub = torch.empty_like(ua)
    op.unpack(prec, 0, a, ua, n)
    op.unpack(prec, 0, b, ub, n)
    torch.cuda.synchronize()
    return ((ua - ub).norm() / ub.norm()).item() < {dd.DD_PREC_F32: 1e-6, dd.DD_PREC_F16: 5e-3}[prec]


@pytest.mark.parametrize("prec", [dd.DD_PREC_F32, dd.DD_PREC_F16])
def test_batched_matches_single_and_oracle(prec):
    shapes = [(4, 4, 4, 4), (2, 4, 6, 8), (8, 8, 8, 8), (6, 4, 4, 2)]
    nrhs = [1, 5, 3, 17]
    ops, keep, ins, outs, refs, psis = [], [], [], [], [], []
    for dims, n in zip(shapes, nrhs):
        U, lat, g, op = make(dims, U=synthetic.gauge(dims, seed=sum(dims)))
        keep.append((U, lat, g, op))
        ops.append(op)
        psi = torch.from_numpy(synthetic.spinor(dims, nrhs=n)).cuda()
        psis.append(psi)
        nb = op.field_bytes(prec, 0, n)
        xi = torch.empty(nb, dtype=torch.uint8, device="cuda")
        xo = torch.empty_like(xi)
        op.pack(prec, 0, psi, xi, n)
        ins.append(xi)
        outs.append(xo)
        ref = torch.empty_like(xi)
        op.apply(dd.DD_OP_D, prec, xi, ref, n, dd.DD_LAYOUT_NATIVE)
        refs.append(ref)
    b = ctypes.c_void_p()
    dd.check(dd.lib.dd_batch_create(_arr([o.h.value for o in ops]), len(ops), prec, _arr(nrhs, ctypes.c_int),
                                    ctypes.byref(b)), "dd_batch_create")
    st = torch.cuda.current_stream().cuda_stream
    pin = _arr([x.data_ptr() for x in ins])
    pout = _arr([x.data_ptr() for x in outs])
    try:
        dd.check(dd.lib.dd_apply_batched(b, pin, pout, st), "dd_apply_batched")
        torch.cuda.synchronize()
        first = [o.clone() for o in outs]
        for o, r, op, n in zip(outs, refs, ops, nrhs):
            # single applies of FP32 fields run the row-staged kernel, which
            # sums the same terms in another rounding order
            assert _close(op, prec, o, r, n)
        chosen = (ctypes.c_int * 3)()
        dd.check(dd.lib.dd_batch_tune(b, pin, pout, st, chosen), "dd_batch_tune")
        assert chosen[0] in (64, 128, 256) and chosen[2] >= 0  # 0: one CTA per work item
        for o in outs:
            o.zero_()
        dd.check(dd.lib.dd_apply_batched_graph(b, pin, pout, st), "graph capture")
        dd.check(dd.lib.dd_apply_batched_graph(b, pin, pout, st), "graph replay")
        torch.cuda.synchronize()
        for o, f in zip(outs, first):
            assert torch.equal(o, f)  # the tuned and replayed launch: same arithmetic, same bits
        # wrong pointers for a captured graph are refused
        bad = _arr([x.data_ptr() for x in refs])
        assert dd.lib.dd_apply_batched_graph(b, pin, bad, st) == dd.DD_ERR_ARG
    finally:
        dd.lib.dd_batch_destroy(b)
    # oracle check of every lattice and RHS
    for (U, lat, g, op), dims, n, o, psi in zip(keep, shapes, nrhs, outs, psis):
        A = oracle.clover(U, dims, M0, CSW)
        got = torch.empty_like(psi)
        op.unpack(prec, 0, o, got, n)
        torch.cuda.synchronize()
        got = got.cpu().numpy()
        p = psi.cpu().numpy()
        for r in range(n):
            assert rel(got[r], oracle.apply_D(U, A, p[r].reshape(-1, 12), dims)) < TOL[prec]


def test_batch_argument_checks():
    U, lat, g, op = make((4, 4, 4, 4))
    b = ctypes.c_void_p()
    assert dd.lib.dd_batch_create(_arr([op.h.value]), 1, dd.DD_PREC_F64, _arr([1], ctypes.c_int),
                                  ctypes.byref(b)) == dd.DD_ERR_ARG
    assert dd.lib.dd_batch_create(_arr([op.h.value]), 1, dd.DD_PREC_F32, _arr([0], ctypes.c_int),
                                  ctypes.byref(b)) == dd.DD_ERR_ARG


def test_batch_with_paired_layout():
    """Lattices with an even RHS count in the paired-RHS layout, the others
    native: the batched launch (one kernel per lattice, forked streams, graph
    replay) equals the single paired / native applies bit for bit."""
    prec = dd.DD_PREC_F32
    shapes = [(4, 4, 4, 4), (6, 4, 4, 2), (8, 8, 8, 8)]
    nrhs = [1, 4, 12]
    ops, keep, ins, outs, refs = [], [], [], [], []
    for dims, n in zip(shapes, nrhs):
        U, lat, g, op = make(dims, U=synthetic.gauge(dims, seed=sum(dims)))
        keep.append((U, lat, g, op))
        ops.append(op)
        psi = torch.from_numpy(synthetic.spinor(dims, nrhs=n)).cuda()
        nb = op.field_bytes(prec, 0, n)
        xi = torch.empty(nb, dtype=torch.uint8, device="cuda")
        xo = torch.empty_like(xi)
        ref = torch.empty_like(xi)
        layout = dd.DD_LAYOUT_NATIVE_PAIRED if n % 2 == 0 else dd.DD_LAYOUT_NATIVE
        if n % 2 == 0:
            op.pack_paired(prec, 0, psi, xi, n)
        else:
            op.pack(prec, 0, psi, xi, n)
        op.apply(dd.DD_OP_D, prec, xi, ref, n, layout)
        ins.append(xi)
        outs.append(xo)
        refs.append(ref)
    b = ctypes.c_void_p()
    dd.check(dd.lib.dd_batch_create(_arr([o.h.value for o in ops]), len(ops), prec, _arr(nrhs, ctypes.c_int),
                                    ctypes.byref(b)), "dd_batch_create")
    st = torch.cuda.current_stream().cuda_stream
    pin = _arr([x.data_ptr() for x in ins])
    pout = _arr([x.data_ptr() for x in outs])
    try:
        assert dd.lib.dd_batch_set_layout(b, dd.DD_LAYOUT_CANONICAL) == dd.DD_ERR_ARG
        dd.check(dd.lib.dd_batch_set_layout(b, dd.DD_LAYOUT_NATIVE_PAIRED), "dd_batch_set_layout")
        chosen = (ctypes.c_int * 3)()
        dd.check(dd.lib.dd_batch_tune(b, pin, pout, st, chosen), "dd_batch_tune")
        assert chosen[2] == -1
        dd.check(dd.lib.dd_apply_batched_graph(b, pin, pout, st), "graph capture")
        for o in outs:
            o.zero_()
        dd.check(dd.lib.dd_apply_batched_graph(b, pin, pout, st), "graph replay")
        torch.cuda.synchronize()
        for o, r in zip(outs, refs):
            assert torch.equal(o, r)
    finally:
        dd.lib.dd_batch_destroy(b)
