"""The allocation-free inner product (dd_dot_noalloc) against the allocating
one (dd_dot), through the C ABI.

dd_dot_noalloc exists for callers that cannot allocate device memory at the
point they need a reduction; its scratch is a fixed array inside the library.
This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest
import torch

import synthetic
import paper_2407_00041_gb300 as dd

pytestmark = pytest.mark.gpu


def _dots(fn, a, b, nsites, nrhs):
    out = np.empty((nrhs, 2), dtype=np.float64)
    st = torch.cuda.current_stream().cuda_stream
    dd.check(fn(a.data_ptr(), b.data_ptr(), nsites, nrhs, out.ctypes.data, st), fn.__name__)
    return out[:, 0] + 1j * out[:, 1]


def test_noalloc_dot_matches_allocating_dot_twice():
    dims = (8, 6, 4, 10)
    nsites = int(np.prod(dims))
    nrhs = 5
    a = torch.from_numpy(synthetic.spinor(dims, nrhs=nrhs, seed=71)).cuda()
    b = torch.from_numpy(synthetic.spinor(dims, nrhs=nrhs, seed=72)).cuda()
    ref = _dots(dd.lib.dd_dot, a, b, nsites, nrhs)
    exact = np.array([np.vdot(a[r].cpu().numpy(), b[r].cpu().numpy()) for r in range(nrhs)])
    assert np.max(np.abs(ref - exact) / np.abs(exact)) < 1e-13
    for _ in range(2):  # the scratch keeps the previous call's contents
        got = _dots(dd.lib.dd_dot_noalloc, a, b, nsites, nrhs)
        assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-13
    # a different size right after reuses the same scratch
    got = _dots(dd.lib.dd_dot_noalloc, a[:2], b[:2], nsites // 2, 2)
    ref2 = _dots(dd.lib.dd_dot, a[:2].contiguous(), b[:2].contiguous(), nsites // 2, 2)
    assert np.max(np.abs(got - ref2) / np.abs(ref2)) < 1e-13


def test_noalloc_dot_rejects_too_many_rhs():
    a = torch.zeros((65, 16, 12), dtype=torch.complex128, device="cuda")
    out = np.empty((65, 2))
    st = torch.cuda.current_stream().cuda_stream
    s = dd.lib.dd_dot_noalloc(a.data_ptr(), a.data_ptr(), 16, 65, out.ctypes.data, st)
    assert s == dd.DD_ERR_ARG
    assert b"64" in dd.lib.dd_last_error_detail()
