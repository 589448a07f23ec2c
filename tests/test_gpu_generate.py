"""dd_gauge_generate: the device-side link generator against the host-side
generator of the same counter-based stream (SplitMix64 + Box-Muller,
U = exp(i eps H)), on small lattices completely and on sampled links of the
48^3 x 96 lattice; the operator built on generated links against the one
built on host-generated links."""
import numpy as np
import pytest
import torch

import synthetic
import paper_2407_00041_gb300 as dd
from tests._gpu import CSW, M0, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 8)])
def test_generated_links_equal_host_generator(dims):
    lat = dd.Lattice(dims, -1)
    g = dd.Gauge.generate(lat, seed=synthetic.SEED_GAUGE, eps=0.3)
    got = g.download()
    ref = synthetic.gauge(dims, eps=0.3)
    assert np.max(np.abs(got - ref)) < 1e-14
    # special unitary
    eye = np.eye(3)
    uu = np.einsum("xmab,xmcb->xmac", got, got.conj())
    assert np.max(np.abs(uu - eye)) < 1e-14
    assert np.max(np.abs(np.linalg.det(got) - 1)) < 1e-14
    assert dd.binding._lib.dd_gauge_stored_rows(g.h, dd.DD_PREC_F32) == 2


def test_generated_links_seed_and_eps():
    dims = (4, 4, 4, 4)
    lat = dd.Lattice(dims, -1)
    a = dd.Gauge.generate(lat, seed=7, eps=0.5).download()
    assert np.max(np.abs(a - synthetic.gauge(dims, seed=7, eps=0.5))) < 1e-14
    b = dd.Gauge.generate(lat, seed=8, eps=0.5).download()
    assert np.max(np.abs(a - b)) > 0.1
    one = dd.Gauge.generate(lat, seed=7, eps=0.0).download()
    assert np.array_equal(one, np.broadcast_to(np.eye(3, dtype=np.complex128), one.shape))
    with pytest.raises(dd.DDError):
        dd.Gauge.generate(lat, seed=7, eps=float("nan"))
    with pytest.raises(dd.DDError):
        dd.Gauge.generate(lat, seed=7, eps=-1.0)


def test_generated_48c96_sampled_links_and_operator():
    dims = (96, 48, 48, 48)
    V = int(np.prod(dims))
    lat = dd.Lattice(dims, -1)
    g = dd.Gauge.generate(lat)
    Ud = torch.empty((V, 4, 3, 3), dtype=torch.complex128, device="cuda")
    g.download(Ud)
    rng = np.random.default_rng(5)
    per = dims[1] * dims[2] * dims[3]
    sites = np.unique(np.concatenate([np.arange(64), np.arange(V - 64, V), rng.integers(0, V, 4000),
                                      [per - 1, V - per]])).astype(np.int64)
    got = Ud[torch.from_numpy(sites).cuda()].cpu().numpy()
    ref = synthetic.gauge_sites(sites, eps=0.3)
    assert np.max(np.abs(got - ref)) < 1e-14
    # the operator on generated links applies like the one on uploaded links
    op = dd.Operator(g, M0, CSW)
    g2 = dd.Gauge(lat, Ud)
    op2 = dd.Operator(g2, M0, CSW)
    psi = torch.from_numpy(synthetic.spinor((96, 48, 48, 48), 1)).cuda()
    o1, o2 = torch.empty_like(psi), torch.empty_like(psi)
    op.apply(dd.DD_OP_D, dd.DD_PREC_F64, psi, o1, 1)
    op2.apply(dd.DD_OP_D, dd.DD_PREC_F64, psi, o2, 1)
    torch.cuda.synchronize()
    assert torch.equal(o1, o2)
    del op, op2, g2, Ud, psi, o1, o2
    torch.cuda.empty_cache()
