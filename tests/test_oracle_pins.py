"""Pins of the CPU oracle against facts fixed by the thesis and by mathematics.

Each test checks the oracle against something other than itself: the Clifford
algebra, an independent dense assembly of Eq. 1.13, the free-field closed-form
spectrum, gamma5-hermiticity, gauge covariance, a closed form of the clover
term for an abelian field, and brute-force linear algebra.
"""
import os

import numpy as np
import pytest

import oracle
import synthetic
from tests import _dense

M0, CSW = -0.4, 1.0


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


def g5_field(psi):
    """gamma5 = diag(1, 1, -1, -1) in spin, applied to [V, 12] fields."""
    p = np.array(psi, dtype=np.complex128).reshape(-1, 4, 3).copy()
    p[:, 2:] *= -1
    return p.reshape(-1, 12)


# ---------------------------------------------------------------- gamma basis

def test_gamma_clifford_and_hermitian():
    g = [oracle.gamma(mu) for mu in range(4)]
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T)
        for nu in range(4):
            ac = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(ac, 2.0 * np.eye(4) * (mu == nu))
    g5 = g[3] @ g[2] @ g[1] @ g[0]  # gamma_X gamma_Y gamma_Z gamma_T
    assert np.allclose(g5, np.diag([1, 1, -1, -1]))
    # the independent test-side construction agrees
    for mu, gd in enumerate(_dense.gammas()):
        assert np.allclose(g[mu], gd)


def test_gamma_T_projector_couples_spins_0_2_and_1_3():
    """Listing 4.2: (1 - gamma_T) pairs spin 0 with spin 2 and spin 1 with spin 3."""
    P = np.eye(4) - oracle.gamma(0)
    assert np.allclose(P, [[1, 0, -1, 0], [0, 1, 0, -1], [-1, 0, 1, 0], [0, -1, 0, 1]])


def test_T_projection_matches_listing_4_2_fixture():
    """The oracle's (1 - gamma_T) acting on the 12 components of a site
    reproduces the index pattern of the projection in Listing 4.2 (fixture
    tests/golden/listing_4_2_T_projection.txt): output component c of the
    upper two spins reads components c and c + 6 only, the second with a
    coefficient of unit modulus."""
    path = os.path.join(os.path.dirname(__file__), "golden", "listing_4_2_T_projection.txt")
    rows = [list(map(int, ln.split())) for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 6
    P12 = np.kron(np.eye(4) - oracle.gamma(0), np.eye(3))  # component = 3 * spin + colour
    for out, first, second, spin in rows:
        nz = set(np.flatnonzero(np.abs(P12[out]) > 1e-12))
        assert nz == {first, second}
        assert np.isclose(P12[out, first], 1.0)
        assert np.isclose(abs(P12[out, second]), 1.0)
        assert second // 3 == spin + 2 and out // 3 == spin


# ----------------------------------------------------------------- generator

def test_links_special_unitary_and_site_addressable():
    dims = (4, 2, 2, 4)
    U = synthetic.gauge(dims)
    M = U.reshape(-1, 3, 3)
    eye = np.eye(3)
    assert np.max(np.abs(np.einsum("nab,ncb->nac", M, M.conj()) - eye)) < 1e-14
    assert np.max(np.abs(np.linalg.det(M) - 1.0)) < 1e-14
    sites = [0, 5, 17, 63]
    assert np.array_equal(synthetic.gauge_sites(sites), U[sites])
    psi = synthetic.spinor(dims, nrhs=2)
    assert np.array_equal(synthetic.spinor_sites(dims, sites, r=1), psi[1][sites])
    # Gaussian moments (loose): mean 0, E|z|^2 = 2
    z = synthetic.gaussian(200000, seed=7)
    assert abs(z.mean()) < 0.02 and abs(np.mean(np.abs(z) ** 2) - 2.0) < 0.03


def test_links_are_exp_of_traceless_hermitian():
    """U = exp(i eps H): the generator H = -i log(U) / eps is Hermitian and traceless."""
    U = synthetic.gauge((2, 2, 2, 2), eps=0.3).reshape(-1, 3, 3)
    w, v = np.linalg.eig(U)
    H = np.einsum("nab,nb,ncb->nac", v, np.angle(w) / 0.3, np.linalg.inv(v).transpose(0, 2, 1))
    assert np.max(np.abs(H - H.conj().transpose(0, 2, 1))) < 1e-10
    assert np.max(np.abs(np.trace(H, axis1=1, axis2=2))) < 1e-10


# ----------------------------------------------------------- P1 brute force

@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 2, 2), (2, 2, 2, 4), (4, 4, 4, 4)])
def test_dense_brute_force(dims):
    U = synthetic.gauge(dims)
    A = oracle.clover(U, dims, M0, CSW)
    Ad = _dense.clover_field(U, dims, M0, CSW)
    assert rel(A, Ad) < 1e-14
    D = _dense.dense_D(U, dims, M0, CSW, t_bc=-1, A=Ad)
    psi = synthetic.spinor(dims, nrhs=1)[0].reshape(-1)
    out = oracle.apply_D(U, A, psi.reshape(-1, 12), dims).reshape(-1)
    assert rel(out, D @ psi) < 1e-14
    if np.prod(dims) <= 16:  # every column on 2^4
        V12 = 12 * int(np.prod(dims))
        cols = np.stack([oracle.apply_D(U, A, e.reshape(-1, 12), dims).reshape(-1) for e in np.eye(V12)], 1)
        assert np.max(np.abs(cols - D)) < 1e-14


@pytest.mark.parametrize("t_bc", [-1, 1])
def test_site_sampled_apply_and_clover_match_the_dense_assembly(t_bc):
    """clover_sites and apply_D_sites (the oracle of the full-size GPU tests)
    against the rows of the independent dense assembly of Eq. 1.13: an
    asymmetric lattice, an unsorted site list with a repeat, both time
    boundaries included."""
    dims = (4, 2, 4, 6)
    per = dims[1] * dims[2] * dims[3]
    V = int(np.prod(dims))
    U = synthetic.gauge(dims)
    psi = synthetic.spinor(dims, nrhs=1)[0].reshape(-1, 12)
    rng = np.random.default_rng(7)
    sites = np.concatenate([[V - 1, 0, per - 1, V - per], rng.integers(0, V, 20), [5, 5]]).astype(np.int64)
    Ad = _dense.clover_field(U, dims, M0, CSW)
    As = oracle.clover_sites(U, dims, M0, CSW, sites)
    assert rel(As, Ad[sites]) < 1e-14
    D = _dense.dense_D(U, dims, M0, CSW, t_bc=t_bc, A=Ad)
    ref = (D @ psi.reshape(-1)).reshape(-1, 12)[sites]
    got = oracle.apply_D_sites(U, As, psi, dims, sites, t_bc=t_bc)
    assert rel(got, ref) < 1e-14


def test_periodic_time_bc():
    dims = (2, 2, 2, 4)
    U = synthetic.gauge(dims)
    A = oracle.clover(U, dims, M0, CSW)
    D = _dense.dense_D(U, dims, M0, CSW, t_bc=+1, A=A)
    psi = synthetic.spinor(dims)[0].reshape(-1)
    assert rel(oracle.apply_D(U, A, psi.reshape(-1, 12), dims, t_bc=+1).reshape(-1), D @ psi) < 1e-14


# -------------------------------------------------------------- P2 free field

def _free_links(dims):
    V = int(np.prod(dims))
    return np.broadcast_to(np.eye(3, dtype=np.complex128), (V, 4, 3, 3)).copy()


def test_free_field_clover_vanishes():
    dims = (4, 2, 2, 2)
    U = _free_links(dims)
    for mu in range(4):
        for nu in range(4):
            if mu != nu:
                assert np.allclose(oracle.Q(U, dims, 3, mu, nu), 4 * np.eye(3))
    A = oracle.clover(U, dims, M0, CSW)
    assert np.allclose(A, (M0 + 4.0) * np.eye(12))


def test_free_field_plane_waves():
    """D e^{ip.x} u = D(p) e^{ip.x} u, D(p) = m0 + sum(1 - cos p) + i sum gamma_mu sin p_mu."""
    dims = (8, 4, 6, 4)
    U = _free_links(dims)
    A = oracle.clover(U, dims, M0, CSW)
    g = [oracle.gamma(mu) for mu in range(4)]
    coords = np.array(np.unravel_index(np.arange(int(np.prod(dims))), dims)).T
    rng = np.random.default_rng(3)
    for kT, kZ, kY, kX in [(0, 0, 0, 0), (1, 2, 3, 1), (7, 3, 5, 2), (3, 1, 0, 3)]:
        p = np.array([np.pi * (2 * kT + 1) / dims[0], 2 * np.pi * kZ / dims[1],
                      2 * np.pi * kY / dims[2], 2 * np.pi * kX / dims[3]])
        u = rng.normal(size=12) + 1j * rng.normal(size=12)
        phase = np.exp(1j * coords @ p)
        psi = phase[:, None] * u[None, :]
        Dp = (M0 + np.sum(1 - np.cos(p))) * np.eye(4, dtype=np.complex128)
        for mu in range(4):
            Dp = Dp + 1j * np.sin(p[mu]) * g[mu]
        expect = phase[:, None] * (np.kron(Dp, np.eye(3)) @ u)[None, :]
        assert rel(oracle.apply_D(U, A, psi, dims), expect) < 1e-14


def test_free_field_spectrum():
    dims = (4, 2, 2, 4)
    U = _free_links(dims)
    A = oracle.clover(U, dims, M0, CSW)
    V12 = 12 * int(np.prod(dims))
    D = np.stack([oracle.apply_D(U, A, e.reshape(-1, 12), dims).reshape(-1) for e in np.eye(V12)], 1)
    ev = np.linalg.eigvals(D)
    expect = []
    for kT in range(dims[0]):
        for kZ in range(dims[1]):
            for kY in range(dims[2]):
                for kX in range(dims[3]):
                    p = np.array([np.pi * (2 * kT + 1) / dims[0], 2 * np.pi * kZ / dims[1],
                                  2 * np.pi * kY / dims[2], 2 * np.pi * kX / dims[3]])
                    re = M0 + np.sum(1 - np.cos(p))
                    im = np.sqrt(np.sum(np.sin(p) ** 2))
                    expect += [re + 1j * im] * 6 + [re - 1j * im] * 6
    key = lambda z: (round(z.real, 8), round(z.imag, 8))
    a = sorted(ev, key=key)
    b = sorted(expect, key=key)
    assert np.max(np.abs(np.array(a) - np.array(b))) < 1e-10


# ---------------------------------------------------- P3 gamma5-hermiticity

def test_gamma5_hermiticity_and_adjoint():
    dims = (4, 4, 2, 4)
    U = synthetic.gauge(dims)
    A = oracle.clover(U, dims, M0, CSW)
    psi = synthetic.spinor(dims, seed=11)[0].reshape(-1, 12)
    phi = synthetic.spinor(dims, seed=12)[0].reshape(-1, 12)
    lhs = np.vdot(phi, oracle.apply_D(U, A, psi, dims))
    g5Dg5phi = g5_field(oracle.apply_D(U, A, g5_field(phi), dims))
    assert abs(lhs - np.vdot(g5Dg5phi, psi)) / abs(lhs) < 1e-14
    DH = oracle.apply_DH(U, A, phi, dims)
    assert abs(lhs - np.vdot(DH, psi)) / abs(lhs) < 1e-14
    assert rel(DH, g5Dg5phi) < 1e-14


# ------------------------------------------------------- P4 gauge covariance

def test_gauge_covariance():
    dims = (4, 2, 4, 2)
    V = int(np.prod(dims))
    U = synthetic.gauge(dims)
    Om = synthetic.su3_field(dims, seed=99, eps=1.0)
    Up = np.empty_like(U)
    for x in range(V):
        for mu in range(4):
            y, _ = oracle.shift(dims, x, mu, +1)
            Up[x, mu] = Om[x] @ U[x, mu] @ Om[y].conj().T
    A = oracle.clover(U, dims, M0, CSW)
    Ap = oracle.clover(Up, dims, M0, CSW)
    W = np.einsum("st,xab->xsatb", np.eye(4), Om).reshape(V, 12, 12)
    assert rel(Ap, W @ A @ W.conj().transpose(0, 2, 1)) < 1e-14
    psi = synthetic.spinor(dims)[0].reshape(-1, 12)
    lhs = oracle.apply_D(Up, Ap, np.einsum("xij,xj->xi", W, psi), dims)
    rhs = np.einsum("xij,xj->xi", W, oracle.apply_D(U, A, psi, dims))
    assert rel(lhs, rhs) < 1e-14


# ----------------------------------------------------------- P5 structure

def test_clover_hermitian_commutes_with_gamma5():
    dims = (2, 4, 2, 2)
    U = synthetic.gauge(dims)
    A = oracle.clover(U, dims, M0, CSW)
    assert np.max(np.abs(A - A.conj().transpose(0, 2, 1))) < 1e-14
    G5 = np.kron(np.diag([1, 1, -1, -1]), np.eye(3))
    assert np.max(np.abs(A @ G5 - G5 @ A)) < 1e-14
    # the clover term is not trivially zero on a random field
    assert np.max(np.abs(A - (M0 + 4) * np.eye(12))) > 1e-2


def test_clover_abelian_closed_form():
    """U_mu(x) = exp(i a_mu(x)) I_3: every leaf of Eq. 1.12 is exp(i * flux)
    with the flux of the plaquette it traverses, so
    Q_munu - Q_numu = 2 i sum_leaves sin(theta_munu(leaf corner)),
    theta_munu(y) = a_mu(y) + a_nu(y+mu) - a_mu(y+nu) - a_nu(y)."""
    dims = (2, 4, 4, 2)
    V = int(np.prod(dims))
    rng = np.random.default_rng(5)
    a = rng.uniform(-1, 1, size=(V, 4))
    U = np.exp(1j * a)[:, :, None, None] * np.eye(3)[None, None]
    A = oracle.clover(U, dims, M0, CSW)
    ag = a.reshape(tuple(dims) + (4,))
    g = [oracle.gamma(mu) for mu in range(4)]
    expect = np.zeros((V, 12, 12), dtype=np.complex128)
    expect[:] = (M0 + 4) * np.eye(12)
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            sh = lambda F, ax, s: np.roll(F, -s, axis=ax)
            theta = ag[..., mu] + sh(ag[..., nu], mu, 1) - sh(ag[..., mu], nu, 1) - ag[..., nu]
            # leaves at corners x, x-mu, x-mu-nu, x-nu
            tot = (np.sin(theta) + np.sin(sh(theta, mu, -1)) + np.sin(sh(sh(theta, mu, -1), nu, -1))
                   + np.sin(sh(theta, nu, -1))).reshape(-1)
            expect -= (CSW / 32.0) * 2j * tot[:, None, None] * np.kron(g[mu] @ g[nu], np.eye(3))[None]
    assert rel(A, expect) < 1e-13


# ------------------------------------- P6 half-spinor (back-substitution) form

B = {  # gamma_mu = [[0, B_mu], [B_mu^H, 0]] in the chiral basis
    0: np.eye(2, dtype=np.complex128),
    1: np.diag([-1j, 1j]),
    2: np.array([[0, -1], [1, 0]], dtype=np.complex128),
    3: np.array([[0, -1j], [-1j, 0]], dtype=np.complex128),
}


def test_half_spinor_projection_identity():
    """(I - s gamma_mu) psi = (h, -s B^H h) with h = u - s B l (u, l = upper and
    lower spin pairs): the projected field has two independent spins, which is
    what the derivation after Algorithm 3 uses (lambda and chi carry 6 complex)."""
    rng = np.random.default_rng(1)
    for mu in range(4):
        g = oracle.gamma(mu)
        assert np.allclose(g[:2, 2:], B[mu]) and np.allclose(g[2:, :2], B[mu].conj().T)
        for s in (+1, -1):
            psi = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
            full = (np.eye(4) - s * g) @ psi
            h = psi[:2] - s * B[mu] @ psi[2:]
            assert np.allclose(full[:2], h)
            assert np.allclose(full[2:], -s * B[mu].conj().T @ h)


# --------------------------------------------------------- even-odd Schur

def test_even_odd_schur():
    dims = (2, 2, 2, 4)
    U = synthetic.gauge(dims)
    A = oracle.clover(U, dims, M0, CSW)
    eo = oracle.EvenOdd(U, A, dims)
    D = _dense.dense_D(U, dims, M0, CSW, A=A)
    idx = lambda s: (12 * s[:, None] + np.arange(12)[None]).reshape(-1)
    ie, io = idx(eo.even), idx(eo.odd)
    Dhat_dense = D[np.ix_(io, io)] - D[np.ix_(io, ie)] @ np.linalg.solve(D[np.ix_(ie, ie)], D[np.ix_(ie, io)])
    v = synthetic.spinor(dims, seed=5)[0].reshape(-1, 12)[eo.odd]
    assert rel(eo.Dhat(v).reshape(-1), Dhat_dense @ v.reshape(-1)) < 1e-13
    assert rel(eo.DhatH(v).reshape(-1), Dhat_dense.conj().T @ v.reshape(-1)) < 1e-13
    # det D = det A_ee * det Dhat
    s1, l1 = np.linalg.slogdet(D)
    s2, l2 = np.linalg.slogdet(D[np.ix_(ie, ie)])
    s3, l3 = np.linalg.slogdet(Dhat_dense)
    assert abs(l1 - (l2 + l3)) < 1e-9 and abs(s1 - s2 * s3) < 1e-9
    # Schur solve + reconstruction = full solve
    b = synthetic.spinor(dims, seed=6)[0].reshape(-1, 12)
    x_full = np.linalg.solve(D, b.reshape(-1)).reshape(-1, 12)
    x_o = np.linalg.solve(Dhat_dense, eo.prepare(b).reshape(-1)).reshape(-1, 12)
    assert rel(eo.reconstruct(b, x_o), x_full) < 1e-12


# ------------------------------------------------------------- P7 FGMRES

def _small_system(dims=(4, 4, 4, 4)):
    U = synthetic.gauge(dims)
    A = oracle.clover(U, dims, M0, CSW)
    op = lambda v: oracle.apply_D(U, A, v.reshape(-1, 12), dims).reshape(-1)
    b = synthetic.spinor(dims)[0].reshape(-1)
    return U, A, op, b


def test_fgmres_converges_true_residual_4x4():
    """4^4 lattice, m0 = -0.4, c_sw = 1, FGMRES(30) to 1e-10; solution checked
    against a dense direct solve."""
    dims = (4, 4, 4, 4)
    U, A, op, b = _small_system(dims)
    x, st = oracle.fgmres(op, b, m=30, tol=1e-10, max_restarts=200)
    assert st.converged
    assert np.linalg.norm(b - op(x)) < 1e-10 * np.linalg.norm(b)
    D = _dense.dense_D(U, dims, M0, CSW, A=A)
    assert rel(x, np.linalg.solve(D, b)) < 1e-8
    for c, k in enumerate(st.inner_steps[:-1]):
        assert k == 30  # full cycles
    # one application for each true residual + one per Arnoldi step (Algorithm 2)
    assert st.applies == len(st.true_residuals) + sum(st.inner_steps)


def test_fgmres_exact_inverse_one_step():
    dims = (2, 2, 2, 2)
    U, A, op, b = _small_system(dims)
    D = _dense.dense_D(U, dims, M0, CSW, A=A)
    Dinv = np.linalg.inv(D)
    x, st = oracle.fgmres(op, b, m=10, tol=1e-10, M=lambda j, v: Dinv @ v)
    assert st.inner_steps[0] == 1
    assert rel(x, Dinv @ b) < 1e-12


def test_fgmres_fixed_preconditioner_equals_gmres_and_min_residual():
    dims = (2, 2, 2, 2)
    U, A, op, b = _small_system(dims)
    m = 8
    rng = np.random.default_rng(2)
    Mi = np.eye(b.size) + 0.05 * (rng.normal(size=(b.size, b.size)) + 1j * rng.normal(size=(b.size, b.size)))
    xf, sf = oracle.fgmres(op, b, m=m, tol=1e-30, max_restarts=1, M=lambda j, v: Mi @ v)
    xg, sg = oracle.gmres_right(op, b, m=m, tol=1e-30, max_restarts=1, Minv=lambda v: Mi @ v)
    assert rel(xf, xg) < 1e-10
    # GMRES = minimal residual over x0 + K_m(A M^-1, r0) mapped by M^-1
    D = _dense.dense_D(U, dims, M0, CSW, A=A)
    AM = D @ Mi
    K = [b]
    for _ in range(m - 1):
        K.append(AM @ K[-1])
    K = np.stack(K, 1)
    Q_, _ = np.linalg.qr(K)
    c = np.linalg.lstsq(AM @ Q_, b, rcond=None)[0]
    assert rel(xf, Mi @ (Q_ @ c)) < 1e-8


def test_arnoldi_relation_and_orthonormality():
    dims = (2, 2, 2, 2)
    U, A, op, b = _small_system(dims)
    rec = []
    oracle.fgmres(op, b, m=12, tol=1e-30, max_restarts=1, record=rec)
    V, H, Z = rec[-1]
    Vm = np.stack(V, 1)
    # V_{m+1}: append the last normalised w
    k = H.shape[1]
    w_next = (np.stack([op(z) for z in Z], 1) - Vm @ H[:k, :k])[:, -1] / H[k, k - 1]
    Vk1 = np.concatenate([Vm, w_next[:, None]], 1)
    assert np.max(np.abs(Vk1.conj().T @ Vk1 - np.eye(k + 1))) < 1e-13
    AZ = np.stack([op(z) for z in Z], 1)
    assert rel(AZ, Vk1 @ H) < 1e-13


# ------------------------------------------------------------ P8 adjoint

def _L(U, phi, psi, dims, A_fixed):
    """Re <phi, D psi>; the self coupling is rebuilt from U unless A_fixed is given."""
    A = oracle.clover(U, dims, M0, CSW) if A_fixed is None else A_fixed
    return np.real(np.vdot(phi, oracle.apply_D(U, A, psi, dims)))


@pytest.mark.parametrize("with_clover", [False, True])
def test_link_force_finite_differences(with_clover):
    dims = (2, 2, 2, 4)
    V = int(np.prod(dims))
    U = synthetic.gauge(dims)
    psi = synthetic.spinor(dims, seed=synthetic.SEED_RHS)[0].reshape(-1, 12)
    phi = synthetic.spinor(dims, seed=synthetic.SEED_PHI)[0].reshape(-1, 12)
    A_fixed = None if with_clover else oracle.clover(U, dims, M0, CSW)
    G, F = oracle.force(U, phi, psi, dims, csw=CSW, with_clover=with_clover)
    # grad_psi = D^H phi (exact)
    rng = np.random.default_rng(8)

    def su3_dir(shape):
        X = rng.normal(size=shape + (3, 3)) + 1j * rng.normal(size=shape + (3, 3))
        X = 0.5 * (X - np.conj(np.swapaxes(X, -1, -2)))
        return X - np.trace(X, axis1=-2, axis2=-1)[..., None, None] / 3 * np.eye(3)

    def expm_ah(X):  # exp of anti-Hermitian via eigh of the Hermitian iX
        w, v = np.linalg.eigh(1j * X)
        return np.einsum("...ab,...b,...cb->...ac", v, np.exp(-1j * w), v.conj())

    h = 1e-6
    # single-link directions
    for _ in range(12):
        x, mu = rng.integers(V), rng.integers(4)
        X = su3_dir(())
        Up, Um = U.copy(), U.copy()
        Up[x, mu] = expm_ah(h * X) @ U[x, mu]
        Um[x, mu] = expm_ah(-h * X) @ U[x, mu]
        fd = (_L(Up, phi, psi, dims, A_fixed) - _L(Um, phi, psi, dims, A_fixed)) / (2 * h)
        an = np.real(np.sum(np.conj(F[x, mu]) * X))
        assert abs(fd - an) <= 1e-7 * max(1.0, abs(an))
    # one global direction field
    X = su3_dir((V, 4))
    Up = np.einsum("xmab,xmbc->xmac", expm_ah(h * X), U)
    Um = np.einsum("xmab,xmbc->xmac", expm_ah(-h * X), U)
    fd = (_L(Up, phi, psi, dims, A_fixed) - _L(Um, phi, psi, dims, A_fixed)) / (2 * h)
    an = np.real(np.sum(np.conj(F) * X))
    assert abs(fd - an) / abs(an) < 1e-7
    # G itself against real/imag finite differences on one entry
    x, mu, a, b_ = 3, 2, 1, 2
    for comp, unit in ((0, 1.0), (1, 1j)):
        Up, Um = U.copy(), U.copy()
        Up[x, mu, a, b_] += h * unit
        Um[x, mu, a, b_] -= h * unit
        fd = (_L(Up, phi, psi, dims, A_fixed) - _L(Um, phi, psi, dims, A_fixed)) / (2 * h)
        val = G[x, mu, a, b_].real if comp == 0 else G[x, mu, a, b_].imag
        assert abs(fd - val) < 1e-7 * max(1, abs(val))


def _table_5_1():
    path = os.path.join(os.path.dirname(__file__), "golden", "table_5_1_configurations.txt")
    rows = {}
    for ln in open(path):
        if ln.strip() and not ln.startswith("#"):
            f = ln.split()
            rows[f[0]] = (tuple(int(v) for v in f[1:5]), float(f[5]), float(f[6]), float(f[7]))
    return rows


def test_oracle_solves_the_tiny_configuration_of_table_5_1():
    """The thesis' tiny configuration (Table 5.1: 8^4, m0 = -0.1, c_sw = 1.0)
    with its tolerance (Section 5.3: 1e-10), on a synthetic gauge field (the
    thesis' configuration is not available): the oracle's FGMRES (Algorithm 2,
    M = I, restart 30) reaches the tolerance on the true residual."""
    dims, m0, csw, tol = _table_5_1()["tiny"]
    assert (dims, m0, csw, tol) == ((8, 8, 8, 8), -0.1, 1.0, 1e-10)
    U = synthetic.gauge(dims)
    A = oracle.clover(U, dims, m0, csw)
    b = synthetic.spinor(dims, nrhs=1)[0].reshape(-1)
    x, st = oracle.fgmres(lambda v: oracle.apply_D(U, A, v.reshape(-1, 12), dims).reshape(-1), b, m=30, tol=tol,
                   max_restarts=200)
    r = b - oracle.apply_D(U, A, x.reshape(-1, 12), dims).reshape(-1)
    assert np.linalg.norm(r) / np.linalg.norm(b) < tol


def test_c_sw_and_tolerance_defaults_follow_table_5_1():
    """c_sw = 1.0 in every configuration of Table 5.1 and the 1e-10 tolerance
    of Section 5.3 are the defaults of the benchmark and of dd_solve."""
    import ctypes
    rows = _table_5_1()
    assert {r[2] for r in rows.values()} == {1.0} and {r[3] for r in rows.values()} == {1e-10}
    import bench
    assert bench.CSW == 1.0
    import paper_2407_00041_gb300 as dd
    p = dd.binding.SolveParams()
    dd.lib.dd_solve_params_default(ctypes.byref(p))
    assert p.tol == 1e-10
