"""Pins of the oracle's residual of Eq. (res1), y = K x - F, and its loss.

Expected values come from exact rational assembly, the closed-form solution
of the structured Poisson system, polynomial reproduction and the sign
conventions of the definition; none re-derives y from the oracle itself.
"""
from __future__ import annotations

from fractions import Fraction as Fr

import numpy as np
import pytest

import meshgen as mg
import oracle as O
from oracle import exact as X
from test_oracle_pins import _dst_solution, _dyadic_tri_mesh, _jittered


def _exact_residual(cells, coords, kind, kap, c, x, f, geo=None):
    """Exact K x - F by rational scatter-add (element matrices by monomial
    integration, F with constant f)."""
    verts = [[Fr(float(v)) for v in p] for p in coords]
    N = len(coords)
    y = [Fr(0)] * N
    xs = [Fr(float(v)) for v in x]
    for cl in cells:
        cl = list(map(int, cl))
        V = [verts[k] for k in cl]
        Vg = V[:geo] if geo else V
        K = X.stiffness(Vg, kind, Fr(kap))
        M = X.mass(Vg, kind)
        Fe = X.load(Vg, kind, Fr(f))
        for a, ga in enumerate(cl):
            y[ga] += sum((K[a][b] + Fr(c) * M[a][b]) * xs[gb] for b, gb in enumerate(cl)) - Fe[a]
    return np.array([float(v) for v in y])


@pytest.mark.parametrize("case", ["p1_tri", "p2_tri", "p1_tet"])
def test_residual_matches_exact_rational_assembly(case):
    g = np.random.default_rng(41)
    if case == "p1_tri":
        cells, coords = _dyadic_tri_mesh(4, 2)
        el, kind, geo = O.P1_TRI, "p1", None
    elif case == "p2_tri":
        m = mg.p2_tri_grid(2)
        cells, coords, el, kind, geo = m.cells, m.coords, O.P2_TRI, "p2", 3
    else:
        m = mg.kuhn_tet_grid(2)
        cells, coords, el, kind, geo = m.cells, m.coords, O.P1_TET, "p1", None
    x = g.integers(-8, 9, size=len(coords)) / 8.0  # dyadic values
    kap, c, f = 1.25, 0.5, 0.75
    want = _exact_residual(cells, coords, kind, kap, c, x, f, geo)
    y, loss = O.residual(el, cells, coords, np.array([kap]), O.CONSTANT, c, x, np.array([f]), O.CONSTANT)
    assert np.allclose(y, want, rtol=0, atol=1e-14 * max(1.0, np.abs(want).max()))
    assert loss == pytest.approx(float(np.dot(want, want)), rel=1e-13)


def test_structured_poisson_discrete_solution_has_zero_residual():
    n = 64
    m = mg.tri_grid(n)
    U = _dst_solution(n)
    m1 = n + 1
    ii, jj = np.arange(m.n_nodes) % m1, np.arange(m.n_nodes) // m1
    u = np.zeros(m.n_nodes)
    inner = ~m.boundary
    u[inner] = U[jj[inner] - 1, ii[inner] - 1]
    y, loss = O.residual(O.P1_TRI, m.cells, m.coords, np.ones(m.n_elems * 3), O.PER_QP, 0.0, u, np.array([1.0]),
                         O.CONSTANT, dirichlet=m.boundary.astype(np.uint8))
    # interior rows of K u and F are 4 u_i - sum of 4 neighbours and h^2: y is rounding only
    scale = 8.0 * np.abs(u).max()
    assert np.all(y[m.boundary] == 0.0)
    assert np.abs(y).max() <= 1e-13 * scale
    assert loss <= (1e-13 * scale) ** 2 * m.n_nodes
    # a dropped load term would leave y = K u = F = h^2 on the interior
    y_nof, _ = O.residual(O.P1_TRI, m.cells, m.coords, np.ones(m.n_elems * 3), O.PER_QP, 0.0, u,
                          dirichlet=m.boundary.astype(np.uint8))
    assert np.allclose(y_nof[inner], 1.0 / n ** 2, rtol=1e-9, atol=0)


@pytest.mark.parametrize("el", [O.P1_TRI, O.P2_TRI, O.P1_TET])
def test_linear_field_leaves_minus_the_load(el):
    # K u_lin vanishes on interior rows (patch test), so y = -F there; with
    # f = 1 and the load's closed form on the structured grid for P1 triangles
    m = _jittered(el)
    a = np.array([0.3, -1.2, 0.7][: m.coords.shape[1]])
    ulin = m.coords @ a + 0.4
    y0, _ = O.residual(el, m.cells, m.coords, np.array([2.0]), O.CONSTANT, 0.0, ulin)
    assert np.abs(y0[~m.boundary]).max() < 1e-12
    fq = np.random.default_rng(5).uniform(-1, 1, m.n_nodes)
    y1, _ = O.residual(el, m.cells, m.coords, np.array([2.0]), O.CONSTANT, 0.0, ulin, fq, O.PER_NODE)
    # F = M fq for a nodal f: with kappa = 0, c = 1 and x = fq the matrix term is that same M fq
    yM, _ = O.residual(el, m.cells, m.coords, np.zeros(1), O.CONSTANT, 1.0, fq)
    assert np.allclose(y1[~m.boundary], -yM[~m.boundary], rtol=0, atol=1e-12)


def test_structured_load_sign_and_mask():
    n = 16
    m = mg.tri_grid(n)
    y, loss = O.residual(O.P1_TRI, m.cells, m.coords, np.ones(1), O.CONSTANT, 0.0, np.zeros(m.n_nodes),
                         np.array([1.0]), O.CONSTANT, dirichlet=m.boundary.astype(np.uint8))
    counts = np.bincount(m.cells.ravel(), minlength=m.n_nodes)
    want = np.where(m.boundary, 0.0, -counts / (6.0 * n * n))
    assert np.array_equal(y == 0, m.boundary)
    assert np.allclose(y, want, rtol=1e-15, atol=0)
    assert loss == pytest.approx(float(np.sum(want ** 2)), rel=1e-14)


def test_p2_quadratic_residual_vanishes():
    # u = x^2 + y^2 lies in P2 and -Laplace u = -4: the residual with f = -4 vanishes on interior rows
    m = mg.p2_tri_grid(6, jitter_seed=5)
    u = (m.coords ** 2).sum(axis=1)
    y, _ = O.residual(O.P2_TRI, m.cells, m.coords, np.array([1.0]), O.CONSTANT, 0.0, u, np.array([-4.0]), O.CONSTANT)
    assert np.abs(y[~m.boundary]).max() < 1e-12
