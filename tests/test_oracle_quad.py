"""Pins of the QUAD4 plane-stress / SIMP oracle.

Expected values: exact rational integration of the element stiffness on
rectangles, the three rigid-body modes (and nothing else) in the null space,
the constant-strain patch test, the SIMP scaling, and central differences
of the compliance for the closed-form sensitivity.
"""
from __future__ import annotations

from fractions import Fraction as Fr

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import meshgen as mg
from oracle import quad as Q


def _poly_mul(p, q):
    out = {}
    for (a, b), c in p.items():
        for (d, e), f in q.items():
            out[(a + d, b + e)] = out.get((a + d, b + e), 0) + c * f
    return out


def _exact_rect_k0(ax, by, nu):
    """int over [0, ax] x [0, by] of B^T D B with polynomial shape gradients, exactly."""
    # physical gradients of the bilinear corner functions in the reference variables s = x / ax, t = y / by:
    # dN/dx = (dN/ds) / ax, dN/dy = (dN/dt) / by; polynomials in (s, t) as {(i, j): coeff}
    dNds = [{(0, 0): -1, (0, 1): 1}, {(0, 0): 1, (0, 1): -1}, {(0, 1): 1}, {(0, 1): -1}]
    dNdt = [{(0, 0): -1, (1, 0): 1}, {(1, 0): -1}, {(1, 0): 1}, {(0, 0): 1, (1, 0): -1}]
    gx = [{k: Fr(v) / ax for k, v in p.items()} for p in dNds]
    gy = [{k: Fr(v) / by for k, v in p.items()} for p in dNdt]
    nu = Fr(nu)
    D = [[1 / (1 - nu * nu), nu / (1 - nu * nu), 0], [nu / (1 - nu * nu), 1 / (1 - nu * nu), 0],
         [0, 0, (1 - nu) / (2 * (1 - nu * nu))]]
    B = [[{} for _ in range(8)] for _ in range(3)]
    for a in range(4):
        B[0][2 * a] = gx[a]
        B[1][2 * a + 1] = gy[a]
        B[2][2 * a] = gy[a]
        B[2][2 * a + 1] = gx[a]
    K = [[Fr(0)] * 8 for _ in range(8)]
    for i in range(8):
        for j in range(8):
            poly = {}
            for r in range(3):
                for c in range(3):
                    if D[r][c] == 0:
                        continue
                    for k, v in _poly_mul(B[r][i], B[c][j]).items():
                        poly[k] = poly.get(k, 0) + D[r][c] * v
            # int_0^1 int_0^1 s^i t^j ds dt = 1 / ((i + 1)(j + 1)); area element ax * by
            K[i][j] = sum(v / ((k[0] + 1) * (k[1] + 1)) for k, v in poly.items()) * ax * by
    return K


@pytest.mark.parametrize("ax,by", [(Fr(1), Fr(1)), (Fr(3, 2), Fr(1, 2))])
def test_rectangle_element_matches_exact_integration(ax, by):
    X = np.array([[0, 0], [float(ax), 0], [float(ax), float(by)], [0, float(by)]])
    K = Q.element_k0(X, 0.3)
    want = np.array([[float(v) for v in row] for row in _exact_rect_k0(ax, by, Fr(3, 10))])
    assert np.allclose(K, want, rtol=0, atol=1e-14 * np.abs(want).max())


def _distorted(nx, ny, seed=2):
    m = mg.quad_grid(nx, ny)
    g = np.random.default_rng(seed)
    disp = g.uniform(-0.2 * m.h, 0.2 * m.h, size=m.coords.shape)
    disp[m.boundary] = 0
    m.coords = m.coords + disp
    return m


def test_rigid_body_modes_span_the_null_space():
    m = _distorted(3, 2)
    K = Q.assemble_simp(m.cells, m.coords, np.ones(m.n_elems), 0.0, 1.0, 3.0, 0.3).to_scipy().toarray()
    x, y = m.coords[:, 0], m.coords[:, 1]
    modes = [np.ravel(np.stack([np.ones_like(x), 0 * x], 1)), np.ravel(np.stack([0 * x, np.ones_like(x)], 1)),
             np.ravel(np.stack([-y, x], 1))]
    for r in modes:
        assert np.abs(K @ r).max() < 1e-12
    ev = np.linalg.eigvalsh(K)
    assert np.sum(ev < 1e-10 * ev.max()) == 3


def test_constant_strain_patch_test():
    m = _distorted(5, 4)
    K = Q.assemble_simp(m.cells, m.coords, np.ones(m.n_elems), 0.0, 2.0, 3.0, 0.3).to_scipy()
    A = np.array([[0.3, -0.2], [0.5, 0.1]])
    u = (m.coords @ A.T).ravel()
    f = K @ u
    interior = np.repeat(~m.boundary, 2)
    assert np.abs(f[interior]).max() < 1e-12


def test_simp_scaling():
    m = _distorted(3, 3)
    rho = np.random.default_rng(1).uniform(0.1, 1.0, m.n_elems)
    K1 = Q.assemble_simp(m.cells, m.coords, np.ones(m.n_elems), 70.0, 7000.0, 3.0, 0.3)
    K0 = Q.assemble_simp(m.cells, m.coords, np.ones(m.n_elems), 0.0, 1.0, 3.0, 0.3)
    assert np.allclose(K1.val, 7000.0 * K0.val, rtol=1e-14)
    Kr = Q.assemble_simp(m.cells, m.coords, rho, 70.0, 7000.0, 3.0, 0.3).to_scipy()
    Ksum = sum((70.0 + rho[e] ** 3 * 6930.0) * Q.assemble_simp(m.cells[e:e + 1], m.coords, [1.0], 0.0, 1.0, 3.0,
                                                                  0.3).to_scipy() for e in range(m.n_elems))
    assert abs(Kr - Ksum).max() < 1e-9 * abs(Kr).max()


def _compliance(cfg, rho):
    m = cfg["mesh"]
    K = Q.assemble_simp(m.cells, m.coords, rho, cfg["E_min"], cfg["E_max"], cfg["penal"], cfg["nu"]).to_scipy()
    free = ~cfg["dirichlet"]
    u = np.zeros(K.shape[0])
    u[free] = spla.spsolve(sp.csc_matrix(K[free][:, free]), cfg["F"][free])
    return float(cfg["F"] @ u), u


def test_sensitivity_matches_central_differences():
    cfg = mg.cantilever(12, 6, 12.0, 6.0)
    m = cfg["mesh"]
    rho = np.random.default_rng(3).uniform(0.3, 0.9, m.n_elems)
    C, u = _compliance(cfg, rho)
    dc = Q.simp_sensitivity(m.cells, m.coords, rho, cfg["E_min"], cfg["E_max"], cfg["penal"], cfg["nu"], u)
    assert np.all(dc <= 0.0)
    for e in (0, 17, 40, 71):
        h = 1e-6
        rp, rm = rho.copy(), rho.copy()
        rp[e] += h
        rm[e] -= h
        fd = (_compliance(cfg, rp)[0] - _compliance(cfg, rm)[0]) / (2 * h)
        assert abs(fd - dc[e]) <= 1e-6 * abs(dc[e]), (e, fd, dc[e])
