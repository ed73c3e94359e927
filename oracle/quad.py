"""FP64 oracle of plane-stress bilinear quadrilaterals (QUAD4) with the SIMP
material law of the SM's topology-optimisation benchmark.  TEST
INFRASTRUCTURE ONLY (tests, smoke, the bench's CPU baseline).

Written from the textbook definitions, not from the library's arithmetic:
  * shape functions on [0, 1]^2: N0 = (1-s)(1-t), N1 = s(1-t), N2 = st,
    N3 = (1-s)t, corners counter-clockwise;
  * 2 x 2 Gauss-Legendre points (numpy), weights 1/4;
  * K0_e = sum_q w_q |det J_q| B_q^T D B_q with the engineering-strain
    matrix B (rows e_xx, e_yy, g_xy) and the plane-stress
    D = 1/(1 - nu^2) [[1, nu, 0], [nu, 1, 0], [0, 0, (1 - nu)/2]] (E = 1);
  * SIMP (SM): E(rho) = E_min + rho^p (E_max - E_min), K = sum_e E(rho_e) K0_e;
  * compliance sensitivity (SM): dC/drho_e = -p rho_e^(p-1) (E_max - E_min)
    u_e^T K0_e u_e.
DoFs are interleaved: 2 node + component.
"""
from __future__ import annotations

import numpy as np

from . import CSR


def gauss2():
    x, w = np.polynomial.legendre.leggauss(2)
    s = (x + 1.0) / 2.0
    pts = [(a, b) for b in s for a in s]
    return pts, np.full(4, 0.25)


def shape_grad(s, t):
    """dN/ds and dN/dt of the four corners at (s, t)."""
    return np.array([[-(1 - t), -(1 - s)], [(1 - t), -s], [t, s], [-t, (1 - s)]])


def element_k0(Xe, nu):
    D = np.array([[1.0, nu, 0.0], [nu, 1.0, 0.0], [0.0, 0.0, (1.0 - nu) / 2.0]]) / (1.0 - nu * nu)
    K = np.zeros((8, 8))
    pts, w = gauss2()
    for (s, t), wq in zip(pts, w):
        dN = shape_grad(s, t)          # [4, 2] reference
        J = Xe.T @ dN                  # J[i, k] = d x_i / d ref_k
        g = dN @ np.linalg.inv(J)      # physical gradients [4, 2]
        B = np.zeros((3, 8))
        for a in range(4):
            B[0, 2 * a] = g[a, 0]
            B[1, 2 * a + 1] = g[a, 1]
            B[2, 2 * a] = g[a, 1]
            B[2, 2 * a + 1] = g[a, 0]
        K += wq * abs(np.linalg.det(J)) * (B.T @ D @ B)
    return K


def _dofs(cell):
    return np.array([[2 * v, 2 * v + 1] for v in cell]).ravel()


def assemble_simp(cells, coords, rho, E_min, E_max, penal, nu) -> CSR:
    """DoF-level CSR of K(rho) by scatter-add into a dictionary of keys."""
    cells = np.asarray(cells)
    X = np.asarray(coords, dtype=np.float64)
    dok = {}
    for e, cell in enumerate(cells):
        Ee = E_min + float(rho[e]) ** penal * (E_max - E_min)
        Ke = Ee * element_k0(X[cell], nu)
        dof = _dofs(cell)
        for a in range(8):
            for b in range(8):
                key = (int(dof[a]), int(dof[b]))
                dok[key] = dok.get(key, 0.0) + Ke[a, b]
    n = 2 * X.shape[0]
    keys = sorted(dok)
    rows = np.array([k[0] for k in keys], dtype=np.int64)
    rp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rp, rows + 1, 1)
    return CSR(np.cumsum(rp), np.array([k[1] for k in keys], dtype=np.int32), np.array([dok[k] for k in keys]))


def simp_sensitivity(cells, coords, rho, E_min, E_max, penal, nu, u):
    cells = np.asarray(cells)
    X = np.asarray(coords, dtype=np.float64)
    out = np.zeros(len(cells))
    for e, cell in enumerate(cells):
        ue = np.asarray(u)[_dofs(cell)]
        out[e] = -penal * float(rho[e]) ** (penal - 1) * (E_max - E_min) * (ue @ element_k0(X[cell], nu) @ ue)
    return out
