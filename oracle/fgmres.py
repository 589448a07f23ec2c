"""FGMRES (Algorithm 2) and right-preconditioned GMRES (Algorithm 1), Section 1.2.

TEST INFRASTRUCTURE ONLY (part of the CPU oracle).

Both follow the algorithms step by step in numpy, in FP64:
  * restart loop: r = b - A x, beta = ||r||, v_1 = r / beta;
  * Arnoldi with modified Gram-Schmidt, h_ij = <w, v_i> = v_i^H w;
  * least squares y = argmin ||beta e_1 - H y|| via numpy's lstsq;
  * x <- x + Z y (FGMRES) or x <- x + M^{-1} V y (GMRES).

Readings where the thesis is silent:
  * termination: ||b - A x|| < tol * ||b - A x_0|| checked on the true
    residual at the start of each restart cycle, or ``max_restarts`` cycles;
  * inside a cycle the least-squares residual ||beta e_1 - H y|| is checked
    after every Arnoldi step and the cycle ends early once it is below
    tol * ||b - A x_0||;
  * the breakdown rule of the thesis: the cycle also ends when
    |h_{j+1,j}| < tol / 10.
"""
from __future__ import annotations

import numpy as np


class Stats:
    def __init__(self):
        self.applies = 0          # operator applications (residuals and Arnoldi steps)
        self.cycles = 0           # restart cycles run
        self.inner_steps = []     # Arnoldi steps per cycle
        self.true_residuals = []  # ||b - A x|| at the start of each cycle
        self.converged = False


def _lsq(H, beta, k):
    rhs = np.zeros(k + 1, dtype=np.complex128)
    rhs[0] = beta
    y = np.linalg.lstsq(H[: k + 1, :k], rhs, rcond=None)[0]
    res = np.linalg.norm(rhs - H[: k + 1, :k] @ y)
    return y, res


def _krylov(A, b, m, tol, max_restarts, x0, precond, flexible, record):
    b = np.asarray(b, dtype=np.complex128).reshape(-1)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128).reshape(-1)
    st = Stats()
    r0norm = None
    while True:
        r = b - A(x)                                   # residual of the cycle
        st.applies += 1
        beta = np.linalg.norm(r)
        st.true_residuals.append(beta)
        if r0norm is None:
            r0norm = beta
        if beta < tol * r0norm or beta == 0.0:
            st.converged = True
            break
        if st.cycles >= max_restarts:
            break
        st.cycles += 1
        V = [r / beta]                                 # first basis vector
        Z = []
        H = np.zeros((m + 1, m), dtype=np.complex128)  # Hessenberg matrix
        k = 0
        for j in range(m):                             # Arnoldi steps
            z = precond(j, V[j])                       # z_j = M_j^{-1} v_j
            Z.append(z)
            w = A(z)
            st.applies += 1
            for i in range(j + 1):                     # modified Gram-Schmidt
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            k = j + 1
            _, res = _lsq(H, beta, k)
            if record is not None:
                record.append((V[: j + 1], H[: j + 2, : j + 1].copy(), Z[:]))
            if res < tol * r0norm or abs(H[j + 1, j]) < tol / 10:
                break
            V.append(w / H[j + 1, j])                  # next basis vector
        st.inner_steps.append(k)
        y, _ = _lsq(H, beta, k)                        # least squares
        if flexible:
            x = x + np.stack(Z[:k], axis=1) @ y        # Algorithm 2: x + Z_m y
        else:
            x = x + precond(None, np.stack(V[:k], axis=1) @ y)  # Algorithm 1: x + M^{-1} V_m y
    return x, st


def fgmres(A, b, m=30, tol=1e-10, max_restarts=100, x0=None, M=None, record=None):
    """Algorithm 2.  ``A(v)`` applies the operator; ``M(j, v)`` applies
    M_j^{-1} (identity if None).  Returns (x, Stats)."""
    precond = (lambda j, v: v) if M is None else M
    return _krylov(A, b, m, tol, max_restarts, x0, precond, True, record)


def gmres_right(A, b, m=30, tol=1e-10, max_restarts=100, x0=None, Minv=None):
    """Algorithm 1 with a fixed right preconditioner ``Minv(v)`` (identity if None)."""
    f = (lambda v: v) if Minv is None else Minv
    return _krylov(A, b, m, tol, max_restarts, x0, lambda j, v: f(v), False, None)
