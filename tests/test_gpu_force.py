"""GPU link derivative and autograd adjoint against the CPU oracle and finite
differences (the hand-written adjoint kernel behind torch.autograd.Function).

L = Re <phi, D psi>.  grad psi = D^H phi; grad U = G (torch's convention
dL/dRe U + i dL/dIm U); F = P(G U^H) is the su(3) force.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
import paper_2407_00041_gb300 as dd
from tests._gpu import CSW, M0, make, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (4, 2, 6, 4)])
@pytest.mark.parametrize("with_clover", [False, True])
@pytest.mark.parametrize("prec,tol", [(dd.DD_PREC_F64, 1e-12), (dd.DD_PREC_F32, 2e-5)])
def test_force_matches_oracle(dims, with_clover, prec, tol):
    U, lat, g, op = make(dims)
    nrhs = 2
    psi = synthetic.spinor(dims, nrhs=nrhs, seed=synthetic.SEED_RHS)
    phi = synthetic.spinor(dims, nrhs=nrhs, seed=synthetic.SEED_PHI)
    G, F = dd.su3_force(op, torch.from_numpy(phi).cuda(), torch.from_numpy(psi).cuda(), with_clover, prec)
    Gr = np.zeros((int(np.prod(dims)), 4, 3, 3), dtype=np.complex128)
    for r in range(nrhs):
        Gr += oracle.force(U, phi[r], psi[r], dims, csw=CSW, with_clover=with_clover)[0]
    Fr = oracle.su3_project(U, Gr)
    assert rel(G.cpu().numpy(), Gr) < tol
    assert rel(F.cpu().numpy(), Fr) < tol


def _local_sites(dims, x):
    c = np.array(np.unravel_index(x, dims))
    offs = np.stack(np.meshgrid(*[np.arange(-2, 3)] * 4, indexing="ij"), -1).reshape(-1, 4)
    cc = (c[None] + offs) % np.array(dims)[None]
    return np.unique(np.ravel_multi_index(tuple(cc.T), dims))


def _local_L(U, phi, psi, dims, sites):
    A = oracle.clover_sites(U, dims, M0, CSW, sites)
    return np.real(np.vdot(phi[sites], oracle.apply_D_sites(U, A, psi, dims, sites)))


def _expm_ah(X):
    w, v = np.linalg.eigh(1j * X)
    return v @ np.diag(np.exp(-1j * w)) @ v.conj().T


def test_autograd_24x4_against_oracle_and_finite_differences():
    """24^4 lattice, FP64: autograd backward of L = Re <phi, D psi> with respect
    to psi and to all 4 * 24^4 links, against the oracle adjoint (hopping
    part, whole field) and central finite differences (h = 1e-6, FP64) of the
    oracle's L, with the self coupling rebuilt from the perturbed links."""
    dims = (24, 24, 24, 24)
    U, lat, g, op = make(dims)
    psi = synthetic.spinor(dims, seed=synthetic.SEED_RHS)
    phi = synthetic.spinor(dims, seed=synthetic.SEED_PHI)
    psi_t = torch.from_numpy(psi).cuda().requires_grad_(True)
    U_t = torch.from_numpy(U).cuda().requires_grad_(True)
    phi_t = torch.from_numpy(phi).cuda()
    for with_clover in (False, True):
        psi_t.grad = None
        U_t.grad = None
        eta = dd.dirac(psi_t, U_t, op, dd.DD_PREC_F64, with_clover)
        L = (phi_t.conj() * eta).sum().real
        L.backward()
        G = U_t.grad.cpu().numpy()
        F = oracle.su3_project(U, G)
        if not with_clover:
            A = oracle.clover(U, dims, M0, CSW)
            Gh, Fh = oracle.force(U, phi[0], psi[0], dims, csw=CSW, with_clover=False)
            assert rel(G, Gh) < 1e-12
            gpsi = oracle.apply_DH(U, A, phi[0].reshape(-1, 12), dims)
            assert rel(psi_t.grad.cpu().numpy()[0].reshape(-1, 12), gpsi) < 1e-13
            assert abs(L.item() - np.real(np.vdot(phi[0], oracle.apply_D(U, A, psi[0], dims)))) < 1e-9 * abs(L.item())
            continue
        rng = np.random.default_rng(11)
        h = 1e-6
        for _ in range(6):
            x, mu = int(rng.integers(U.shape[0])), int(rng.integers(4))
            X = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
            X = 0.5 * (X - X.conj().T)
            X -= np.trace(X) / 3 * np.eye(3)
            sites = _local_sites(dims, x)
            vals = []
            for sgn in (+1, -1):
                Up = U.copy()
                Up[x, mu] = _expm_ah(sgn * h * X) @ U[x, mu]
                vals.append(_local_L(Up, phi[0], psi[0], dims, sites))
            fd = (vals[0] - vals[1]) / (2 * h)
            an = float(np.real(np.sum(np.conj(F[x, mu]) * X)))
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (x, mu, fd, an)
