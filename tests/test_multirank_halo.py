"""The halo-exchange data plane of the domain decomposition (Algorithm 3,
Sections 2.1 and 2.2) on CPU: gloo ranks each own one local lattice of the
global one, build the face messages of Algorithm 3 from their own sites
(lambda = (I - gamma_mu) psi on the lowest mu slice, chi = (I + gamma_mu)
U_mu^H psi on the highest), exchange them with ``decomp.exchange`` and apply
D to their local sites using only their own data and the received faces.  The
result must equal the oracle's single-domain D on those sites, and the
allreduce of the ranks' partial inner products the global inner product.

The arithmetic here is the test's own numpy restatement of Eq. 1.13 split as
Algorithm 3 splits it; the product code under test is the rank plan (local
lattice, offsets, neighbours, face order) and the exchange."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

M0, CSW = -0.4, 1.0


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _local_D(plan, U_l, A_l, psi_l, recv, t_bc, gamma):
    """D on the rank's sites from its own fields and the received faces."""
    n = plan.local
    V = psi_l.shape[0]
    cl = np.stack(np.unravel_index(np.arange(V), n), axis=1)  # local coordinates (T, Z, Y, X)
    cg = cl + np.array(plan.offset)
    strides = np.array([n[1] * n[2] * n[3], n[2] * n[3], n[3], 1])
    eye = np.eye(4)
    out = np.einsum("sab,sb->sa", A_l, psi_l.reshape(V, 12))
    hop = np.zeros((V, 4, 3), dtype=np.complex128)
    psi4 = psi_l.reshape(V, 4, 3)
    for mu in range(4):
        Pm, Pp = eye - gamma[mu], eye + gamma[mu]
        Uf = U_l[:, mu]  # U_mu(x), x local
        # forward: (I - gamma) U_mu(x) psi(x + mu)
        fwd_cross = plan.split(mu) & (cl[:, mu] == n[mu] - 1)
        nb = cl.copy()
        nb[:, mu] = (nb[:, mu] + 1) % n[mu]
        j = nb @ strides
        proj = np.einsum("ab,sbc->sac", Pm, psi4[j])
        if fwd_cross.any():
            f = _face_index(cl[fwd_cross], mu, n)
            proj[fwd_cross] = recv[(mu, 0)][f].reshape(-1, 4, 3)
        term = np.einsum("scd,sad->sac", Uf, proj)
        sign = np.where((mu == 0) & (cg[:, 0] == plan.dims[0] - 1), t_bc, 1.0)
        hop += sign[:, None, None] * term
        # backward: (I + gamma) U_mu(x - mu)^H psi(x - mu)
        bwd_cross = plan.split(mu) & (cl[:, mu] == 0)
        nb = cl.copy()
        nb[:, mu] = (nb[:, mu] - 1) % n[mu]
        j = nb @ strides
        term = np.einsum("ab,sbc->sac", Pp, np.einsum("sdc,sad->sac", U_l[j, mu].conj(), psi4[j]))
        if bwd_cross.any():
            f = _face_index(cl[bwd_cross], mu, n)
            term[bwd_cross] = recv[(mu, 1)][f].reshape(-1, 4, 3)
        sign = np.where((mu == 0) & (cg[:, 0] == 0), t_bc, 1.0)
        hop += sign[:, None, None] * term
    return out - 0.5 * hop.reshape(V, 12)


def _face_index(c, mu, n):
    f = np.zeros(len(c), dtype=np.int64)
    for d in range(4):
        if d != mu:
            f = f * n[d] + c[:, d]
    return f


def _worker(rank, world, port, dims, grid, t_bc, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world, init_method=f"tcp://127.0.0.1:{port}")
    try:
        import oracle
        import synthetic
        from paper_2407_00041_gb300 import decomp
        plan = decomp.HaloPlan(tuple(dims), tuple(grid), rank)
        # every rank draws the global inputs (counter based) but keeps only its own sites
        U = synthetic.gauge(dims)
        A = oracle.clover(U, dims, M0, CSW)
        psi = synthetic.spinor(dims, nrhs=1)[0].reshape(-1, 12)
        sites = plan.local_sites()
        U_l, A_l, psi_l = U[sites], A[sites], psi[sites]
        gamma = [oracle.gamma(mu) for mu in range(4)]
        # the face messages of Algorithm 3 from the rank's own sites
        sends, recvs = {}, {}
        for mu, kind, dst, src in plan.messages():
            fs = plan.face_sites(mu, 0 if kind == decomp.LAMBDA else 1)
            p4 = psi_l[fs].reshape(-1, 4, 3)
            if kind == decomp.LAMBDA:
                m = np.einsum("ab,sbc->sac", np.eye(4) - gamma[mu], p4)
            else:
                m = np.einsum("ab,sbc->sac", np.eye(4) + gamma[mu], np.einsum("sdc,sad->sac", U_l[fs, mu].conj(), p4))
            sends[(mu, kind)] = torch.from_numpy(np.ascontiguousarray(m.reshape(-1, 12)))
            recvs[(mu, kind)] = torch.empty_like(sends[(mu, kind)])
            assert m.shape[0] == plan.face_size(mu)
        decomp.exchange(plan, sends, recvs)
        rec = {k: v.numpy() for k, v in recvs.items()}
        eta = _local_D(plan, U_l, A_l, psi_l, rec, t_bc, gamma)
        ref = oracle.apply_D(U, A, psi, dims, t_bc=t_bc)[sites]
        err = float(np.linalg.norm(eta - ref) / np.linalg.norm(ref))
        # allreduce of the partial inner products <eta, psi> over the ranks
        part = torch.tensor([np.vdot(eta, psi_l).real, np.vdot(eta, psi_l).imag], dtype=torch.float64)
        dist.all_reduce(part)
        full = np.vdot(oracle.apply_D(U, A, psi, dims, t_bc=t_bc), psi)
        derr = abs(complex(part[0].item(), part[1].item()) - full) / abs(full)
        q.put((rank, err, derr, len(plan.messages())))
    finally:
        dist.destroy_process_group()


def _run(dims, grid, t_bc=-1):
    world, port = int(np.prod(grid)), _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_worker, args=(r, world, port, dims, grid, t_bc, q)) for r in range(world)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(300)
        assert p.exitcode == 0
    return sorted(q.get() for _ in range(world))


@pytest.mark.parametrize("grid", [(2, 1, 1, 1), (1, 1, 1, 2), (1, 2, 1, 1)])
def test_two_rank_halo_exchange_matches_single_domain(grid):
    res = _run((8, 4, 4, 4), grid)
    for rank, err, derr, nmsg in res:
        assert err < 1e-14, (rank, err)
        assert derr < 1e-14, (rank, derr)
        assert nmsg == 2  # one split direction: lambda and chi


def test_four_rank_halo_exchange_two_split_directions_periodic():
    res = _run((4, 4, 2, 4), (2, 1, 1, 2), t_bc=+1)
    for rank, err, derr, nmsg in res:
        assert err < 1e-14 and derr < 1e-14, (rank, err, derr)
        assert nmsg == 4


def test_halo_plan_geometry():
    from paper_2407_00041_gb300 import decomp
    plan = decomp.HaloPlan((8, 4, 4, 8), (2, 1, 2, 2), 5)
    # rank 5 = ((t * 1 + z) * 2 + y) * 2 + x with X fastest
    assert plan.coords == (1, 0, 0, 1) and plan.local == (4, 4, 2, 4) and plan.offset == (4, 0, 0, 4)
    assert decomp.rank_of(plan.coords, plan.grid) == 5
    assert plan.neighbour(0, -1) == plan.neighbour(0, +1) == 1
    assert plan.neighbour(2, +1) == 7 and plan.neighbour(3, -1) == 4
    assert [m[:2] for m in plan.messages()] == [(0, 0), (0, 1), (2, 0), (2, 1), (3, 0), (3, 1)]
    f0, f1 = plan.face_sites(3, 0), plan.face_sites(3, 1)
    assert len(f0) == plan.face_size(3) == 4 * 4 * 2 and np.all(f1 - f0 == 3)
    with pytest.raises(ValueError):
        decomp.HaloPlan((6, 4, 4, 4), (2, 1, 1, 1), 0)  # local extent 3 is odd
