"""Pins of the oracle's boundary-facet terms (Neumann and Robin).

Expected values: the perimeter and surface area of the unit square and
cube, the closed-form edge and face mass matrices, exact rational
integration on dyadic edges, and exact reproduction of linear solutions of
Laplace's equation under Robin, Neumann and Dirichlet conditions.
"""
from __future__ import annotations

from fractions import Fraction as Fr

import numpy as np
import pytest
import scipy.sparse as sp

import meshgen as mg
import oracle as O
from oracle import solve as S


def _jittered(el, n, seed=3):
    if el == O.P1_TRI:
        return mg.jitter(mg.tri_grid(n), seed)
    m = mg.kuhn_tet_grid(n)
    g = np.random.default_rng(seed)
    disp = g.uniform(-0.15 * m.h, 0.15 * m.h, size=m.coords.shape)
    disp[m.boundary] = 0
    m.coords = m.coords + disp
    return m


def _dense(M, N):
    A = np.zeros((N, N))
    for (i, j), v in M.items():
        A[i, j] += v
    return A


@pytest.mark.parametrize("el,measure", [(O.P1_TRI, 4.0), (O.P1_TET, 6.0)])
def test_boundary_measure_and_load_sums(el, measure):
    m = _jittered(el, 6 if el == O.P1_TRI else 3)
    f = mg.boundary_facets(m)
    M, F = O.assemble_facets(el, f, m.coords, np.array([2.5]), O.CONSTANT, np.array([1.5]), O.CONSTANT)
    assert sum(M.values()) == pytest.approx(2.5 * measure, rel=1e-14)
    assert F.sum() == pytest.approx(1.5 * measure, rel=1e-14)
    assert np.all(F[~m.boundary] == 0.0)


def test_edge_closed_forms_on_the_structured_square():
    n = 8
    m = mg.tri_grid(n)
    f = mg.boundary_facets(m)
    h = 1.0 / n
    M, F = O.assemble_facets(O.P1_TRI, f, m.coords, np.array([3.0]), O.CONSTANT, np.array([2.0]), O.CONSTANT)
    A = _dense(M, m.n_nodes)
    for e in f:
        i, j = int(e[0]), int(e[1])
        assert A[i, j] == pytest.approx(3.0 * h / 6.0, rel=1e-14)  # alpha h / 6 per edge, one edge per pair
    b = np.flatnonzero(m.boundary)
    assert np.allclose(np.diag(A)[b], 2 * 3.0 * h / 3.0, rtol=1e-14)  # two edges of alpha h / 3 each
    assert np.allclose(F[b], 2.0 * h, rtol=1e-14)  # two half edges of g h / 2


def test_face_closed_form_on_one_triangle():
    # one tetrahedron with a face in the z = 0 plane of area 1/2 * 0.5 * 0.25
    X = np.array([[0, 0, 0], [0.5, 0, 0], [0, 0.25, 0], [0, 0, 0.75]], float)
    face = np.array([[0, 1, 2]])
    M, F = O.assemble_facets(O.P1_TET, face, X, np.array([1.0]), O.CONSTANT, np.array([1.0]), O.CONSTANT)
    area = 0.5 * 0.5 * 0.25
    A = _dense(M, 4)[:3, :3]
    want = area / 12.0 * np.array([[2, 1, 1], [1, 2, 1], [1, 1, 2]])
    assert np.allclose(A, want, rtol=1e-14, atol=0)
    assert np.allclose(F[:3], area / 3.0, rtol=1e-14)


def test_edge_matrix_exact_rational():
    # int_0^1 phi_a phi_b |e| dt with phi = (1 - t, t) on a dyadic edge, alpha linear along it (PER_QP
    # values of alpha = 1 + t): exact integrals of (1 - t)^2 (1 + t) etc. times |e| = 3/4
    X = np.array([[0.25, 0.5], [1.0, 0.5], [0.25, 1.0]])
    edge = np.array([[0, 1]])
    xq, _ = np.polynomial.legendre.leggauss(2)
    tq = (xq + 1) / 2
    M, _ = O.assemble_facets(O.P1_TRI, edge, X, 1.0 + tq, O.PER_QP)
    L = Fr(3, 4)
    # exact: int (1-t)^2 (1+t) = 5/12, int t(1-t)(1+t) = 1/4, int t^2 (1+t) = 7/12
    want = {(0, 0): L * Fr(5, 12), (0, 1): L * Fr(1, 4), (1, 0): L * Fr(1, 4), (1, 1): L * Fr(7, 12)}
    for k, v in want.items():
        assert M[k] == pytest.approx(float(v), rel=1e-15)


@pytest.mark.parametrize("el", [O.P1_TRI, O.P1_TET])
def test_nodal_load_is_boundary_mass_times_values(el):
    m = _jittered(el, 5 if el == O.P1_TRI else 3)
    f = mg.boundary_facets(m)
    gv = np.random.default_rng(4).uniform(-1, 1, m.n_nodes)
    M, _ = O.assemble_facets(el, f, m.coords, np.array([1.0]), O.CONSTANT)
    _, F = O.assemble_facets(el, f, m.coords, g=gv, g_layout=O.PER_NODE)
    assert np.allclose(F, _dense(M, m.n_nodes) @ gv, rtol=0, atol=1e-14)


def _outward_normal(el, P):
    """Axis-aligned outward normal of a facet of the unit square or cube."""
    c = P.mean(axis=0)
    d = P.shape[1]
    for k in range(d):
        if np.allclose(P[:, k], 0.0):
            n = np.zeros(d)
            n[k] = -1.0
            return n
        if np.allclose(P[:, k], 1.0):
            n = np.zeros(d)
            n[k] = 1.0
            return n
    raise AssertionError(("not a boundary facet", c))


def _facet_points(el, P):
    nf = P.shape[0]
    if nf == 2:
        xq, _ = np.polynomial.legendre.leggauss(2)
        return [P[0] + (t + 1) / 2 * (P[1] - P[0]) for t in xq]
    _, xq = O.quadrature(O.P1_TRI)
    return [P[0] + x[0] * (P[1] - P[0]) + x[1] * (P[2] - P[0]) for x in xq]


@pytest.mark.parametrize("el", [O.P1_TRI, O.P1_TET])
def test_linear_solution_reproduced_under_mixed_conditions(el):
    """u = a.x + b solves Laplace's equation: Dirichlet on the faces x_0 = 0,
    Neumann (g = du/dn) on the faces x_1 = 0 and x_1 = 1, Robin (g = du/dn +
    alpha u) on the rest; the P1 solution reproduces u to solver tolerance."""
    m = _jittered(el, 6 if el == O.P1_TRI else 3, seed=7)
    d = m.coords.shape[1]
    a = np.array([0.7, -1.3, 0.4][:d])
    u = m.coords @ a + 0.25
    alpha = 1.7
    facets = mg.boundary_facets(m)
    rob, neu = [], []
    for fv in facets:
        n = _outward_normal(el, m.coords[fv])
        if n[0] == -1.0:
            continue  # Dirichlet side
        (neu if abs(n[1]) == 1.0 else rob).append(fv)
    rob, neu = np.array(rob), np.array(neu)
    nq = 2 if el == O.P1_TRI else 3

    def gvals(fs, with_alpha):
        out = []
        for fv in fs:
            P = m.coords[fv]
            n = _outward_normal(el, P)
            for x in _facet_points(el, P):
                out.append(a @ n + (alpha * (x @ a + 0.25) if with_alpha else 0.0))
        return np.array(out)

    K = O.assemble_bilinear(el, m.cells, m.coords, np.array([1.0]), O.CONSTANT, 0.0).to_scipy().tolil()
    Mr, Fr_ = O.assemble_facets(el, rob, m.coords, np.array([alpha]), O.CONSTANT, gvals(rob, True), O.PER_QP)
    _, Fn = O.assemble_facets(el, neu, m.coords, g=gvals(neu, False), g_layout=O.PER_QP)
    for (i, j), v in Mr.items():
        K[i, j] += v
    K = sp.csr_matrix(K)
    F = Fr_ + Fn
    dirichlet = np.isclose(m.coords[:, 0], 0.0)
    uh, it, res = S.solve_dirichlet(K, F, dirichlet, tol=1e-13, g=u)
    assert np.abs(uh - u).max() < 1e-10
    assert len(rob) > 0 and len(neu) > 0 and nq in (2, 3)
