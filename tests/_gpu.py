"""Helpers of the GPU tests: build operators from seeded inputs and run the
library through its C ABI on canonical device fields."""
import numpy as np
import torch

import synthetic
import paper_2407_00041_gb300 as dd

M0, CSW = -0.4, 1.0
TOL = {dd.DD_PREC_F64: 1e-13, dd.DD_PREC_F32: 1e-6, dd.DD_PREC_F16: 5e-3}


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def make(dims, U=None, m0=M0, csw=CSW, t_bc=-1):
    if U is None:
        U = synthetic.gauge(dims)
    lat = dd.Lattice(dims, t_bc)
    g = dd.Gauge(lat, U)
    op = dd.Operator(g, m0, csw)
    return U, lat, g, op


def apply(op, which, prec, psi, layout=dd.DD_LAYOUT_CANONICAL):
    """psi: complex128 numpy [nrhs, nsites, 4, 3] (or [nrhs, nsites, 12])."""
    nrhs = psi.shape[0]
    if layout == dd.DD_LAYOUT_CANONICAL_HOST:
        x = np.ascontiguousarray(psi)
        out = np.empty_like(x)
        op.apply(which, prec, x, out, nrhs, layout)
        return out
    x = torch.from_numpy(np.ascontiguousarray(psi)).cuda()
    out = torch.empty_like(x)
    op.apply(which, prec, x, out, nrhs, layout)
    torch.cuda.synchronize()
    return out.cpu().numpy()
