"""Independent numpy restatement of Eq. 1.11-1.13 as a dense matrix.

Used only to pin the C oracle on tiny lattices.  It shares nothing with the
oracle: neighbours come from numpy index arithmetic, Q_munu from rolled link
arrays, and D is assembled block by block with Kronecker products.
"""
from __future__ import annotations

import numpy as np

SIGMA = [
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
]


def gammas():
    """Euclidean chiral basis, index order T, Z, Y, X.

    gamma_k = [[0, -i sigma_k], [i sigma_k, 0]] with k = 1, 2, 3 for X, Y, Z
    and gamma_T = [[0, I], [I, 0]]."""
    z2, i2 = np.zeros((2, 2)), np.eye(2)
    g = {}
    for k, name in zip(range(3), "XYZ"):
        g[name] = np.block([[z2, -1j * SIGMA[k]], [1j * SIGMA[k], z2]])
    g["T"] = np.block([[z2, i2], [i2, z2]]).astype(np.complex128)
    return [g["T"], g["Z"], g["Y"], g["X"]]


def gamma5():
    gT, gZ, gY, gX = gammas()
    return gX @ gY @ gZ @ gT


def _grid(U, dims):
    return U.reshape(tuple(dims) + (4, 3, 3))


def Q_field(U, dims, mu, nu):
    """Q_munu(x) of Eq. 1.12 at every site, from rolled link arrays: [V, 3, 3]."""
    G = _grid(U, dims)
    Um, Un = G[..., mu, :, :], G[..., nu, :, :]

    def at(F, **shift):  # F(x + a*mu + b*nu)
        out = F
        for ax, s in shift.items():
            axis = mu if ax == "m" else nu
            out = np.roll(out, -s, axis=axis)
        return out

    H = lambda M: np.conj(np.swapaxes(M, -1, -2))
    mm = lambda *Ms: _chain(Ms)
    l1 = mm(Um, at(Un, m=1), H(at(Um, n=1)), H(Un))
    l2 = mm(Un, H(at(Um, m=-1, n=1)), H(at(Un, m=-1)), at(Um, m=-1))
    l3 = mm(H(at(Um, m=-1)), H(at(Un, m=-1, n=-1)), at(Um, m=-1, n=-1), at(Un, n=-1))
    l4 = mm(H(at(Un, n=-1)), at(Um, n=-1), at(Un, n=-1, m=1), H(Um))
    return (l1 + l2 + l3 + l4).reshape(-1, 3, 3)


def _chain(Ms):
    out = Ms[0]
    for M in Ms[1:]:
        out = np.einsum("...ab,...bc->...ac", out, M)
    return out


def clover_field(U, dims, m0, csw):
    g = gammas()
    V = int(np.prod(dims))
    A = np.zeros((V, 12, 12), dtype=np.complex128)
    A[:] = (m0 + 4.0) * np.eye(12)
    for mu in range(4):
        for nu in range(4):
            F = Q_field(U, dims, mu, nu) - Q_field(U, dims, nu, mu)
            GG = g[mu] @ g[nu]
            A -= (csw / 32.0) * np.einsum("st,xab->xsatb", GG, F).reshape(V, 12, 12)
    return A


def dense_D(U, dims, m0, csw, t_bc=-1, A=None):
    """D of Eq. 1.13 as a dense (12V x 12V) matrix, row/column index 12*site + comp."""
    dims = tuple(int(d) for d in dims)
    V = int(np.prod(dims))
    g = gammas()
    if A is None:
        A = clover_field(U, dims, m0, csw)
    Ul = U.reshape(V, 4, 3, 3)
    D = np.zeros((12 * V, 12 * V), dtype=np.complex128)
    coords = np.array(np.unravel_index(np.arange(V), dims)).T
    I4 = np.eye(4)
    for x in range(V):
        D[12 * x:12 * x + 12, 12 * x:12 * x + 12] += A[x]
        for mu in range(4):
            for step in (+1, -1):
                c = coords[x].copy()
                c[mu] += step
                sign = 1.0
                if c[mu] in (-1, dims[mu]):
                    c[mu] %= dims[mu]
                    if mu == 0:
                        sign = float(t_bc)
                y = int(np.ravel_multi_index(tuple(c), dims))
                if step == +1:
                    blk = np.kron(I4 - g[mu], Ul[x, mu])
                else:
                    blk = np.kron(I4 + g[mu], Ul[y, mu].conj().T)
                D[12 * x:12 * x + 12, 12 * y:12 * y + 12] += -0.5 * sign * blk
    return D
