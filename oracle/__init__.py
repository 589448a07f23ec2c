"""CPU oracle of the Wilson-clover path: a plain, slow FP64 restatement of the
thesis "Accelerating Lattice QCD Simulations using GPUs" (Matthaei, 2023).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library (``paper_2407_00041_gb300``) and never imports it.

Contents and the passage each part follows:
  * ``wilson_clover.c`` (loaded through ctypes): gamma matrices, Q_munu
    (Eq. 1.12), self coupling A(x) (Eq. 1.11 / 2.5), D (Eq. 1.13), D^H as the
    conjugate transpose of Eq. 1.13's terms, and the derivative of
    Re <phi, D psi> with respect to the links.
  * this module: the even-odd Schur complement (not in the thesis; defined
    from the block form of D), the su(3) force projection wrapper.
  * ``fgmres.py``: Algorithm 2 (FGMRES) and Algorithm 1 (right-preconditioned
    GMRES), Section 1.2.
  * ``sap.py``: the Schwarz alternating procedure named in Section 1.3 (red-black
    multiplicative Schwarz with minimal-residual block solves), the smoother
    and flexible preconditioner M_j.
  * ``amg.py``: the two-level AMG preconditioner of Section 1.3 (aggregation
    with a chirality split, P from orthonormalised test vectors, R = P^H,
    D_c = R D P, coarse-grid correction plus SAP post-smoothing, the setup
    phase).

Array conventions (same as ``synthetic``):
  dims = (nT, nZ, nY, nX); psi [V, 4, 3] (or [V, 12]); U [V, 4, 3, 3];
  self coupling A [V, 12, 12].
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

from .fgmres import fgmres, gmres_right  # noqa: F401
from . import amg, sap  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wilson_clover.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``wilson_clover.c`` into ``liboracle.so`` (gcc -O2, OpenMP over sites)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P, I, D, L = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
        sig = {
            "oracle_gamma": [I, P],
            "oracle_shift": [P, L, I, I, I, P],
            "oracle_Q": [P, P, L, I, I, P],
            "oracle_clover_site": [P, P, D, D, L, P],
            "oracle_clover_field": [P, P, D, D, P],
            "oracle_clover_sites": [P, P, D, D, P, L, P],
            "oracle_threads": [],
            "oracle_set_threads": [I],
            "oracle_apply_D": [P, I, P, P, P, P],
            "oracle_apply_D_sites": [P, I, P, P, P, P, L, P],
            "oracle_apply_DH": [P, I, P, P, P, P],
            "oracle_force_hop": [P, I, P, P, P, P],
            "oracle_force_clover": [P, P, D, P, P, P],
            "oracle_force_project": [L, P, P, P],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = None
        lib.oracle_shift.restype = L
        lib.oracle_threads.restype = I
        _lib = lib
    return _lib


def _dims(dims):
    return (ctypes.c_int * 4)(*[int(d) for d in dims])


def _c(a, dtype=np.complex128):
    return np.ascontiguousarray(a, dtype=dtype)


def volume(dims) -> int:
    return int(np.prod([int(d) for d in dims]))


def gamma(mu: int) -> np.ndarray:
    """gamma_mu (mu = 0..3 for T, Z, Y, X) in the oracle's chiral basis."""
    out = np.empty(16, dtype=np.complex128)
    _load().oracle_gamma(mu, out.ctypes.data)
    return out.reshape(4, 4)


def shift(dims, site: int, mu: int, step: int, t_bc: int = -1):
    """(neighbour site, boundary sign) of ``site + step*mu``."""
    sg = ctypes.c_double()
    s = _load().oracle_shift(_dims(dims), int(site), mu, step, t_bc, ctypes.byref(sg))
    return int(s), sg.value


def Q(U, dims, site: int, mu: int, nu: int) -> np.ndarray:
    """Q_munu(x) of Eq. 1.12 as a 3x3 matrix."""
    U = _c(U)
    out = np.empty(9, dtype=np.complex128)
    _load().oracle_Q(_dims(dims), U.ctypes.data, int(site), mu, nu, out.ctypes.data)
    return out.reshape(3, 3)


def clover(U, dims, m0: float, csw: float) -> np.ndarray:
    """Self coupling A(x) of Eq. 2.5 at every site: [V, 12, 12]."""
    U = _c(U)
    A = np.empty((volume(dims), 12, 12), dtype=np.complex128)
    _load().oracle_clover_field(_dims(dims), U.ctypes.data, m0, csw, A.ctypes.data)
    return A


def clover_sites(U, dims, m0: float, csw: float, sites) -> np.ndarray:
    """A(x) of Eq. 2.5 for the listed sites only: [len(sites), 12, 12]."""
    U = _c(U)
    s = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.empty((s.size, 12, 12), dtype=np.complex128)
    _load().oracle_clover_sites(_dims(dims), U.ctypes.data, m0, csw, s.ctypes.data, s.size, out.ctypes.data)
    return out


def threads() -> int:
    """OpenMP threads the oracle's site loops use."""
    return int(_load().oracle_threads())


def set_threads(n: int) -> None:
    """Threads of the oracle's later site loops (timing only; same results)."""
    _load().oracle_set_threads(int(n))


def apply_D(U, A, psi, dims, t_bc: int = -1) -> np.ndarray:
    """D psi per Eq. 1.13 (a = 1); psi of shape [V, ...] with 12 components per site."""
    U, A = _c(U), _c(A)
    p = _c(psi).reshape(-1, 12)
    out = np.empty_like(p)
    _load().oracle_apply_D(_dims(dims), t_bc, U.ctypes.data, A.ctypes.data, p.ctypes.data, out.ctypes.data)
    return out.reshape(np.shape(psi))


def apply_D_sites(U, A_sites, psi, dims, sites, t_bc: int = -1) -> np.ndarray:
    """(D psi)(x) for x in ``sites`` only; ``A_sites`` = self coupling of those sites."""
    U, A = _c(U), _c(A_sites)
    p = _c(psi).reshape(-1, 12)
    s = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.empty((s.size, 12), dtype=np.complex128)
    _load().oracle_apply_D_sites(_dims(dims), t_bc, U.ctypes.data, A.ctypes.data, p.ctypes.data,
                                 s.ctypes.data, s.size, out.ctypes.data)
    return out


def apply_DH(U, A, psi, dims, t_bc: int = -1) -> np.ndarray:
    """D^H psi: the conjugate transpose of Eq. 1.13's terms, applied by scatter."""
    U, A = _c(U), _c(A)
    p = _c(psi).reshape(-1, 12)
    out = np.empty_like(p)
    _load().oracle_apply_DH(_dims(dims), t_bc, U.ctypes.data, A.ctypes.data, p.ctypes.data, out.ctypes.data)
    return out.reshape(np.shape(psi))


# ---------------------------------------------------------------------------
# Even-odd (red-black) Schur complement.  Not in the thesis; defined from the
# block form of D.  Sites are split by parity (t+z+y+x) mod 2 (0 = even,
# 1 = odd).  With D = [[D_ee, D_eo], [D_oe, D_oo]] (D_ee = A_ee and
# D_oo = A_oo are the self coupling, site-diagonal):
#     Dhat = A_oo - D_oe A_ee^{-1} D_eo              (on odd sites)
#     bhat = b_o - D_oe A_ee^{-1} b_e
#     x_e  = A_ee^{-1} (b_e - D_eo x_o)
# D_eo and D_oe are taken as restrictions of the full apply of Eq. 1.13 to
# fields that vanish on the other parity; A_ee^{-1} is a dense 12x12 inverse
# per even site.
# ---------------------------------------------------------------------------

def parity(dims) -> np.ndarray:
    nT, nZ, nY, nX = (int(d) for d in dims)
    t, z, y, x = np.meshgrid(np.arange(nT), np.arange(nZ), np.arange(nY), np.arange(nX), indexing="ij")
    return ((t + z + y + x) % 2).reshape(-1)


def eo_sites(dims):
    """(even sites, odd sites), each in increasing lexicographic order."""
    p = parity(dims)
    return np.nonzero(p == 0)[0], np.nonzero(p == 1)[0]


class EvenOdd:
    """The even-odd Schur operator built from the full oracle apply."""

    def __init__(self, U, A, dims, t_bc: int = -1):
        self.U, self.A, self.dims, self.t_bc = _c(U), _c(A), tuple(dims), t_bc
        self.V = volume(dims)
        self.even, self.odd = eo_sites(dims)
        self.Ainv_e = np.linalg.inv(self.A[self.even])

    def _D_block(self, v_from, from_sites, to_sites):
        full = np.zeros((self.V, 12), dtype=np.complex128)
        full[from_sites] = v_from
        return apply_D(self.U, self.A, full, self.dims, self.t_bc)[to_sites]

    def D_eo(self, v_o):
        return self._D_block(v_o, self.odd, self.even)

    def D_oe(self, v_e):
        return self._D_block(v_e, self.even, self.odd)

    def Aee_inv(self, v_e):
        return np.einsum("sij,sj->si", self.Ainv_e, v_e)

    def A_oo(self, v_o):
        return np.einsum("sij,sj->si", self.A[self.odd], v_o)

    def Dhat(self, v_o):
        v_o = np.asarray(v_o).reshape(-1, 12)
        return self.A_oo(v_o) - self.D_oe(self.Aee_inv(self.D_eo(v_o)))

    def DhatH(self, v_o):
        """Conjugate transpose of Dhat: A_oo^H - D_eo^H A_ee^{-H} D_oe^H."""
        v_o = np.asarray(v_o).reshape(-1, 12)
        full = np.zeros((self.V, 12), dtype=np.complex128)
        full[self.odd] = v_o
        t_e = apply_DH(self.U, self.A, full, self.dims, self.t_bc)[self.even]  # D_oe^H v_o
        t_e = np.einsum("sji,sj->si", self.Ainv_e.conj(), t_e)  # A_ee^{-H}
        full = np.zeros((self.V, 12), dtype=np.complex128)
        full[self.even] = t_e
        u_o = apply_DH(self.U, self.A, full, self.dims, self.t_bc)[self.odd]  # D_eo^H t_e
        return np.einsum("sji,sj->si", self.A[self.odd].conj(), v_o) - u_o

    def prepare(self, b):
        b = np.asarray(b).reshape(-1, 12)
        return b[self.odd] - self.D_oe(self.Aee_inv(b[self.even]))

    def reconstruct(self, b, x_o):
        b = np.asarray(b).reshape(-1, 12)
        x = np.zeros((self.V, 12), dtype=np.complex128)
        x[self.odd] = x_o
        x[self.even] = self.Aee_inv(b[self.even] - self.D_eo(x_o))
        return x


# ---------------------------------------------------------------------------
# Link derivative of L = Re <phi, D psi>
# ---------------------------------------------------------------------------

def force(U, phi, psi, dims, csw: float = 0.0, t_bc: int = -1, with_clover: bool = True):
    """(G, F) for L = Re sum_x phi(x)^H (D psi)(x).

    G = dL/dRe U + i dL/dIm U per link ([V, 4, 3, 3]); F = P(G U^H) is its
    su(3) projection.  ``with_clover=False`` holds the self coupling fixed
    (only the hopping terms of Eq. 1.13 are differentiated); otherwise the
    self coupling is rebuilt from the links (Eq. 1.11, 1.12) and differentiated
    too.
    """
    U = _c(U)
    ph = _c(phi).reshape(-1, 12)
    ps = _c(psi).reshape(-1, 12)
    V = volume(dims)
    G = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    lib = _load()
    lib.oracle_force_hop(_dims(dims), t_bc, U.ctypes.data, ph.ctypes.data, ps.ctypes.data, G.ctypes.data)
    if with_clover and csw != 0.0:
        Gc = np.zeros_like(G)
        lib.oracle_force_clover(_dims(dims), U.ctypes.data, csw, ph.ctypes.data, ps.ctypes.data, Gc.ctypes.data)
        G += Gc
    F = np.empty_like(G)
    lib.oracle_force_project(V * 4, U.ctypes.data, G.ctypes.data, F.ctypes.data)
    return G, F


def su3_project(U, G):
    """P(G U^H) for arrays of links [..., 3, 3]."""
    U, G = _c(U), _c(G)
    F = np.empty_like(G)
    _load().oracle_force_project(U.size // 9, U.ctypes.data, G.ctypes.data, F.ctypes.data)
    return F
