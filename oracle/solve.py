"""Conjugate gradients on the Dirichlet-condensed system (TEST INFRASTRUCTURE ONLY).

Dirichlet rows and columns with u = 0 are removed ("condensed stiffness
matrix", SM B.1 solver configuration) and K_II u_I = F_I is solved by plain
CG until ||K_II u_I - F_I|| / ||F_I|| <= tol (the paper's criterion).  The
sparse matrix-vector product is scipy's; the iteration is written out here.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def condense(K: sp.csr_matrix, F: np.ndarray, dirichlet: np.ndarray):
    interior = np.flatnonzero(~dirichlet)
    return K[interior][:, interior].tocsr(), F[interior], interior


def cg(A, b: np.ndarray, tol: float = 1e-10, maxit: int = 100000, x0=None):
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A @ x
    p = r.copy()
    rr = float(r @ r)
    nb = float(np.linalg.norm(b))
    if nb == 0.0:
        return x, 0, 0.0
    it = 0
    while it < maxit:
        if np.sqrt(rr) / nb <= tol:
            break
        Ap = A @ p
        alpha = rr / float(p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        rr_new = float(r @ r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    res = float(np.linalg.norm(b - A @ x)) / nb
    return x, it, res


def solve_dirichlet(K: sp.csr_matrix, F: np.ndarray, dirichlet: np.ndarray, tol: float = 1e-10, g=None):
    """Solve with u = g on the Dirichlet nodes (g = 0 when None)."""
    n = K.shape[0]
    u = np.zeros(n)
    if g is not None:
        u[dirichlet] = g[dirichlet]
    rhs = F - K @ u
    Kc, Fc, interior = condense(K, rhs, dirichlet)
    x, it, res = cg(Kc, Fc, tol=tol)
    u[interior] = x
    return u, it, res
