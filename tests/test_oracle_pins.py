"""Pins of the FP64 oracle against what the mathematics fixes.

Nothing here compares the oracle with itself: every expected value is a
closed form, a published table, an exact rational integral, an invariant of
the continuous problem, or a finite difference of the forward map.
"""
from __future__ import annotations

import math
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

import meshgen as mg
import oracle as O
from oracle import exact as X
from oracle import solve as S

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_matrices():
    out = {}
    name = None
    with open(os.path.join(GOLD, "reference_matrices.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if not tok[0].lstrip("-").isdigit():
                name = tok[0]
                num, den = tok[1].split("/")
                out[name] = [Fr(int(num), int(den)), []]
            else:
                out[name][1].append([int(t) for t in tok])
    return {k: np.array(v[1], dtype=float) * float(v[0]) for k, v in out.items()}


# ---------------------------------------------------------------- quadrature
@pytest.mark.parametrize("el,degree", [(O.P1_TRI, 2), (O.P2_TRI, 4), (O.P1_TET, 2)])
def test_quadrature_exact_to_its_degree(el, degree):
    w, x = O.quadrature(el)
    d = x.shape[1]
    import itertools
    for exps in itertools.product(range(degree + 1), repeat=d):
        if sum(exps) > degree:
            continue
        got = float(np.sum(w * np.prod(x ** np.array(exps), axis=1)))
        want = float(X.monomial_integral_ref(exps))
        assert abs(got - want) <= 1e-15 * max(1.0, abs(want)) + 1e-17, (exps, got, want)


def test_tri6_rule_matches_dunavant_table():
    rows = np.loadtxt(os.path.join(GOLD, "dunavant_deg4_6pt.txt"))
    w, x = O.quadrature(O.P2_TRI)
    # barycentric of the oracle's points: l0 = 1 - xi - eta, l1 = xi, l2 = eta
    bary = np.stack([1 - x[:, 0] - x[:, 1], x[:, 0], x[:, 1]], axis=1)
    for q in range(6):
        orbit = rows[0] if q < 3 else rows[1]
        assert abs(w[q] - 0.5 * orbit[0]) < 1e-14
        assert np.allclose(np.sort(bary[q]), np.sort(orbit[1:]), atol=1e-14, rtol=0)
        # distinguished coordinate (the odd one) sits at index q mod 3
        odd = orbit[1]
        assert abs(bary[q][q % 3] - odd) < 1e-14


def test_quadrature_point_order():
    # order of the per-point coefficient arrays, fixed by the design
    w, x = O.quadrature(O.P1_TRI)
    assert np.allclose(x, [[1 / 6, 1 / 6], [2 / 3, 1 / 6], [1 / 6, 2 / 3]], atol=0, rtol=0)
    w, x = O.quadrature(O.P1_TET)
    a, b = (5 + 3 * math.sqrt(5)) / 20, (5 - math.sqrt(5)) / 20
    assert np.allclose(x, [[b, b, b], [a, b, b], [b, a, b], [b, b, a]], atol=1e-16)
    assert np.allclose(w, 1 / 24)


# ---------------------------------------------------------------- element matrices
def test_reference_element_matrices():
    M = _read_matrices()
    tri = [[0, 0], [1, 0], [0, 1]]
    tet = [[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]]
    assert np.array_equal(O.element_matrix(O.P1_TRI, tri, 1.0, 0.0), M["tri_stiffness"])
    assert np.allclose(O.element_matrix(O.P1_TRI, tri, 0.0, 1.0), M["tri_mass"], rtol=1e-15, atol=1e-17)
    assert np.allclose(O.element_matrix(O.P1_TET, tet, 1.0, 0.0), M["tet_stiffness"], rtol=1e-15, atol=1e-17)
    assert np.allclose(O.element_matrix(O.P1_TET, tet, 0.0, 1.0), M["tet_mass"], rtol=1e-15, atol=1e-17)


def _dyadic_simplex(g, d, scale=8):
    while True:
        V = [[Fr(int(v), scale) for v in g.integers(-scale, scale + 1, size=d)] for _ in range(d + 1)]
        S_ = X.Simplex(V)
        if S_.vol != 0:
            return V


@pytest.mark.parametrize("kind,el,d", [("p1", O.P1_TRI, 2), ("p2", O.P2_TRI, 2), ("p1", O.P1_TET, 3)])
def test_element_matrix_vs_exact_integration(kind, el, d):
    g = np.random.default_rng(7)
    for _ in range(6):
        V = _dyadic_simplex(g, d)
        kap, c = Fr(int(g.integers(1, 9)), 4), Fr(int(g.integers(0, 9)), 8)
        Ke = np.array(X.stiffness(V, kind, kap), dtype=float) + float(c) * np.array(X.mass(V, kind), dtype=float)
        Ko = O.element_matrix(el, np.array(V, dtype=float), float(kap), float(c))
        assert np.allclose(Ko, Ke, rtol=1e-13, atol=1e-13 * np.abs(Ke).max())
        Fe = np.array(X.load(V, kind, 1), dtype=float)
        cells = np.arange(d + 1 if kind == "p1" else 6)[None, :]
        if kind == "p2":
            # P2 edge nodes at midpoints (their coordinates are not used by the geometry)
            Vf = np.array(V, dtype=float)
            coords = np.vstack([Vf, (Vf[0] + Vf[1]) / 2, (Vf[1] + Vf[2]) / 2, (Vf[2] + Vf[0]) / 2])
        else:
            coords = np.array(V, dtype=float)
        Fo = O.assemble_load(el, cells, coords, np.array([1.0]), O.CONSTANT)
        assert np.allclose(Fo, Fe, rtol=1e-13, atol=1e-15)


def test_elastic_element_vs_voigt():
    g = np.random.default_rng(8)
    for _ in range(5):
        V = _dyadic_simplex(g, 3)
        lam, mu = Fr(int(g.integers(1, 9)), 4), Fr(int(g.integers(1, 9)), 8)
        Ke = np.array(X.elasticity(V, lam, mu), dtype=float)
        Ko = O.elastic_element_matrix(np.array(V, dtype=float), float(lam), float(mu))
        assert np.allclose(Ko, Ke, rtol=1e-13, atol=1e-13 * np.abs(Ke).max())


def test_per_qp_kappa_p1_depends_on_weights_only():
    # P1 gradients are constant, so kappa at the points enters as sum_q w_q kappa_q
    g = np.random.default_rng(9)
    Xc = g.normal(size=(3, 2))
    kq = g.uniform(0.5, 2.0, size=3)
    K1 = O.element_matrix(O.P1_TRI, Xc, kq, 0.0)
    K2 = O.element_matrix(O.P1_TRI, Xc, np.full(3, kq.mean()), 0.0)
    assert np.allclose(K1, K2, rtol=1e-14)


# ---------------------------------------------------------------- global DOK vs exact DOK
def _dyadic_tri_mesh(n, seed):
    m = mg.tri_grid(n)
    g = np.random.default_rng(seed)
    # interior jitter by multiples of h/16 within +-0.1875h keeps coordinates dyadic
    disp = g.integers(-3, 4, size=m.coords.shape) / (16 * n)
    disp[m.boundary] = 0
    return m.cells, m.coords + disp


def test_dok_matches_exact_assembly_small_meshes():
    cases = []
    cells, coords = _dyadic_tri_mesh(4, 1)
    cases.append((O.P1_TRI, "p1", cells, coords))
    cases.append((O.P1_TRI, "p1", np.array([[0, 1, 2]]), np.array([[0, 0], [1, 0], [0, 1]], float)))
    cases.append((O.P1_TRI, "p1", np.array([[0, 1, 2], [1, 3, 2]]), np.array([[0, 0], [1, 0], [0, 1], [1.25, 0.75]])))
    p2 = mg.p2_tri_grid(2)
    cases.append((O.P2_TRI, "p2", p2.cells, p2.coords))
    t = mg.kuhn_tet_grid(2)
    cases.append((O.P1_TET, "p1", t.cells, t.coords))
    for el, kind, cells, coords in cases:
        kap, c = 1.5, 0.25
        verts = [[Fr(float(v)) for v in p] for p in coords]
        geo = 3 if el == O.P2_TRI else None

        def local(Xs, kind=kind, geo=geo):
            V = Xs[:geo] if geo else Xs
            K = X.stiffness(V, kind, Fr(kap))
            M_ = X.mass(V, kind)
            return [[K[a][b] + Fr(c) * M_[a][b] for b in range(len(K))] for a in range(len(K))]

        dok = X.assemble_dok([list(map(int, cl)) for cl in cells], verts, local)
        res = O.assemble_bilinear(el, cells, coords, np.array([kap]), O.CONSTANT, c)
        keys = sorted(dok)
        rows = res.rows_of()
        assert list(zip(rows.tolist(), res.col.tolist())) == keys
        want = np.array([float(dok[k]) for k in keys])
        assert np.allclose(res.val, want, rtol=1e-13, atol=1e-14 * np.abs(want).max())


# ---------------------------------------------------------------- structured Poisson (config-1 shape)
def test_five_point_stencil_bit_exact():
    n = 64
    m = mg.tri_grid(n)
    K = O.assemble_bilinear(O.P1_TRI, m.cells, m.coords, np.ones(m.n_elems * 3), O.PER_QP, 0.0)
    assert K.nnz == 29057
    m1 = n + 1
    rows = K.rows_of()
    for s in range(K.nnz):
        i, j = rows[s], K.col[s]
        if m.boundary[i]:
            continue
        di, dj = j % m1 - i % m1, j // m1 - i // m1
        if (di, dj) == (0, 0):
            want = 4.0
        elif abs(di) + abs(dj) == 1:
            want = -1.0
        else:
            assert (di, dj) in ((1, 1), (-1, -1))
            want = 0.0
        assert K.val[s] == want


def test_structured_load_counts_incident_triangles():
    n = 64
    m = mg.tri_grid(n)
    F = O.assemble_load(O.P1_TRI, m.cells, m.coords, np.array([1.0]), O.CONSTANT)
    counts = np.bincount(m.cells.ravel(), minlength=m.n_nodes)
    assert np.allclose(F, counts / (6.0 * n * n), rtol=1e-15, atol=0)


def _dst_solution(n):
    """Closed form of the 5-point system (4u - sum nbrs) = h^2 with u = 0 on the boundary."""
    mm = n - 1
    k = np.arange(1, mm + 1)
    Smat = np.sqrt(2.0 / n) * np.sin(np.outer(k, k) * np.pi / n)
    lam = 2.0 - 2.0 * np.cos(k * np.pi / n)
    B = np.full((mm, mm), 1.0 / n ** 2)
    U = Smat @ ((Smat @ B @ Smat) / (lam[:, None] + lam[None, :])) @ Smat
    return U  # U[j-1, i-1] for interior node (i, j)


def _continuum_centre():
    m = np.arange(1, 4001, 2, dtype=np.float64)
    sm = (-1.0) ** ((m - 1) / 2)
    M, Nn = np.meshgrid(m, m, indexing="ij")
    T = 16.0 * np.outer(sm, sm) / (np.pi ** 4 * M * Nn * (M ** 2 + Nn ** 2))
    return float(T.sum())


def test_config1_solution_matches_closed_form_and_converges():
    errs = []
    uc = _continuum_centre()
    assert abs(uc - 0.07367) < 1e-5
    for n in (32, 64):
        m = mg.tri_grid(n)
        K = O.assemble_bilinear(O.P1_TRI, m.cells, m.coords, np.ones(m.n_elems * 3), O.PER_QP, 0.0).to_scipy()
        F = O.assemble_load(O.P1_TRI, m.cells, m.coords, np.array([1.0]), O.CONSTANT)
        u, it, res = S.solve_dirichlet(K, F, m.boundary, tol=1e-12)
        assert res <= 1e-12
        U = _dst_solution(n)
        m1 = n + 1
        ii = np.arange(m.n_nodes) % m1
        jj = np.arange(m.n_nodes) // m1
        inner = ~m.boundary
        assert np.allclose(u[inner], U[jj[inner] - 1, ii[inner] - 1], rtol=1e-9, atol=1e-13)
        centre = (n // 2) * m1 + n // 2
        errs.append(abs(u[centre] - uc))
    rate = math.log2(errs[0] / errs[1])
    assert 1.8 < rate < 2.2, (errs, rate)


# ---------------------------------------------------------------- invariants on jittered meshes
def _jittered(el, n=6, seed=3):
    if el == O.P1_TRI:
        m = mg.jitter(mg.tri_grid(n), seed)
    elif el == O.P2_TRI:
        m = mg.p2_tri_grid(n, jitter_seed=seed)
    else:
        m = mg.kuhn_tet_grid(n if n <= 4 else 4)
        g = np.random.default_rng(seed)
        disp = g.uniform(-0.15 * m.h, 0.15 * m.h, size=m.coords.shape)
        disp[m.boundary] = 0
        m.coords = m.coords + disp
    return m


@pytest.mark.parametrize("el", [O.P1_TRI, O.P2_TRI, O.P1_TET])
def test_invariants_row_sums_symmetry_mass(el):
    m = _jittered(el)
    nq = O.NQ[el]
    kap = np.random.default_rng(11).lognormal(size=m.n_elems * nq)
    K = O.assemble_bilinear(el, m.cells, m.coords, kap, O.PER_QP, 0.0).to_scipy()
    rs = np.asarray(K.sum(axis=1)).ravel()
    assert np.abs(rs).max() <= 1e-12 * abs(K).max()
    D = (K - K.T).tocoo()
    assert np.abs(D.data).max(initial=0) <= 1e-13 * abs(K).max()
    M = O.assemble_bilinear(el, m.cells, m.coords, np.zeros(1), O.CONSTANT, 1.0).to_scipy()
    assert abs(M.sum() - 1.0) < 1e-13


@pytest.mark.parametrize("el", [O.P1_TRI, O.P2_TRI, O.P1_TET])
def test_patch_test_linear_solution(el):
    m = _jittered(el)
    a = np.array([0.3, -1.2, 0.7][: m.coords.shape[1]])
    ulin = m.coords @ a + 0.4
    K = O.assemble_bilinear(el, m.cells, m.coords, np.array([2.0]), O.CONSTANT, 0.0).to_scipy()
    r = K @ ulin
    assert np.abs(r[~m.boundary]).max() < 1e-12
    u, it, res = S.solve_dirichlet(K, np.zeros(m.n_nodes), m.boundary, tol=1e-13, g=ulin)
    assert np.abs(u - ulin).max() < 1e-10


def test_p2_reproduces_quadratic():
    # u = x^2 + y^2 lies in P2; -Laplace u = -4, so K u = F(f = -4) at interior nodes.
    m = mg.p2_tri_grid(6, jitter_seed=5)
    u = (m.coords ** 2).sum(axis=1)
    K = O.assemble_bilinear(O.P2_TRI, m.cells, m.coords, np.array([1.0]), O.CONSTANT, 0.0).to_scipy()
    F = O.assemble_load(O.P2_TRI, m.cells, m.coords, np.array([-4.0]), O.CONSTANT)
    r = K @ u - F
    assert np.abs(r[~m.boundary]).max() < 1e-12


def test_elasticity_rigid_body_modes_and_null_space():
    m = mg.kuhn_tet_grid(2)
    g = np.random.default_rng(5)
    m.coords = m.coords + np.where(m.boundary[:, None], 0, g.uniform(-0.05, 0.05, size=m.coords.shape))
    lam = g.uniform(0.5, 2.0, size=m.n_elems)
    mu = g.uniform(0.3, 1.0, size=m.n_elems)
    K = O.assemble_elasticity(m.cells, m.coords, lam, mu, O.PER_ELEMENT).to_scipy().toarray()
    assert np.allclose(K, K.T, atol=1e-13 * np.abs(K).max())
    x = m.coords
    modes = []
    for c in range(3):
        t = np.zeros((m.n_nodes, 3))
        t[:, c] = 1
        modes.append(t.ravel())
    for axis in range(3):
        w = np.zeros(3)
        w[axis] = 1
        modes.append(np.cross(w, x).ravel())
    for r in modes:
        assert np.abs(K @ r).max() < 1e-12 * np.abs(K).max()
    ev = np.linalg.eigvalsh(K)
    tol = 1e-10 * ev.max()
    assert int(np.sum(np.abs(ev) < tol)) == 6
    assert ev.min() > -tol


def test_load_sums_and_mass_interpolant():
    m = _jittered(O.P1_TET)
    F = O.assemble_load(O.P1_TET, m.cells, m.coords, np.array([1.0]), O.CONSTANT)
    X_ = m.coords[m.cells]
    vol = np.abs(np.linalg.det(np.stack([X_[:, 1] - X_[:, 0], X_[:, 2] - X_[:, 0], X_[:, 3] - X_[:, 0]], -1))) / 6
    want = np.bincount(m.cells.ravel(), weights=np.repeat(vol / 4, 4), minlength=m.n_nodes)
    assert np.allclose(F, want, rtol=1e-13)
    assert abs(F.sum() - 1.0) < 1e-13
    # nodal f: F = M f with the exact rational mass matrix on a dyadic mesh
    cells, coords = _dyadic_tri_mesh(3, 2)
    f = np.random.default_rng(3).uniform(-1, 1, size=coords.shape[0])
    verts = [[Fr(float(v)) for v in p] for p in coords]
    dok = X.assemble_dok([list(map(int, c)) for c in cells], verts, lambda Xs: X.mass(Xs, "p1"))
    Mx = np.zeros((coords.shape[0],) * 2)
    for (i, j), v in dok.items():
        Mx[i, j] = float(v)
    Fo = O.assemble_load(O.P1_TRI, cells, coords, f, O.PER_NODE)
    assert np.allclose(Fo, Mx @ f, rtol=1e-13, atol=1e-16)
    # vector body force, per component
    F3 = O.assemble_load(O.P1_TET_VEC3, m.cells, m.coords, np.array([0.0, 0.0, -1.0]), O.CONSTANT, ncomp=3)
    assert np.allclose(F3.reshape(-1, 3)[:, 2], -want, rtol=1e-13)
    assert np.all(F3.reshape(-1, 3)[:, :2] == 0)


def test_manufactured_solution_converges_second_order():
    w6, x6 = O.quadrature(O.P2_TRI)  # degree-4 rule for the error integral
    errs = []
    hs = [8, 16, 32, 64]
    for n in hs:
        m = mg.tri_grid(n)
        w3, x3 = O.quadrature(O.P1_TRI)
        Xc = m.coords[m.cells]
        J = np.stack([Xc[:, 1] - Xc[:, 0], Xc[:, 2] - Xc[:, 0]], -1)
        # physical quadrature points for the load: x = x0 + J xhat
        xq = Xc[:, None, 0, :] + np.einsum("erc,qc->eqr", J, x3)
        fq = 2 * np.pi ** 2 * np.sin(np.pi * xq[..., 0]) * np.sin(np.pi * xq[..., 1])
        K = O.assemble_bilinear(O.P1_TRI, m.cells, m.coords, np.array([1.0]), O.CONSTANT, 0.0).to_scipy()
        F = O.assemble_load(O.P1_TRI, m.cells, m.coords, fq.ravel(), O.PER_QP)
        u, it, res = S.solve_dirichlet(K, F, m.boundary, tol=1e-12)
        phi = np.array([O.basis(O.P1_TRI, x)[0] for x in x6])  # [6, 3]
        uh = np.einsum("qa,ea->eq", phi, u[m.cells])
        x6p = Xc[:, None, 0, :] + np.einsum("erc,qc->eqr", J, x6)
        ue = np.sin(np.pi * x6p[..., 0]) * np.sin(np.pi * x6p[..., 1])
        det = np.abs(np.linalg.det(J))
        errs.append(math.sqrt(float(np.sum(det[:, None] * w6[None, :] * (uh - ue) ** 2))))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert min(rates) >= 1.9, (errs, rates)


# ---------------------------------------------------------------- backward vs finite differences
def _random_grad_csr(K: O.CSR, seed):
    g = np.random.default_rng(seed)
    return O.CSR(K.row_ptr, K.col, g.normal(size=K.nnz))


def _L(el, cells, coords, kappa, layout, c, G: O.CSR):
    K = O.assemble_bilinear(el, cells, coords, kappa, layout, c)
    assert np.array_equal(K.col, G.col)
    return float(K.val @ G.val)


@pytest.mark.parametrize("el,layout", [(O.P1_TRI, O.PER_QP), (O.P2_TRI, O.PER_QP), (O.P1_TET, O.PER_ELEMENT),
                                       (O.P1_TRI, O.CONSTANT)])
def test_backward_matches_central_differences(el, layout):
    m = _jittered(el, n=3, seed=4)
    nq = O.NQ[el]
    g = np.random.default_rng(12)
    nk = m.n_elems * nq if layout == O.PER_QP else m.n_elems if layout == O.PER_ELEMENT else 1
    kap = g.uniform(0.5, 2.0, size=nk)
    c = 0.7
    K = O.assemble_bilinear(el, m.cells, m.coords, kap, layout, c)
    G = _random_grad_csr(K, 13)
    gk, gx, gc = O.assemble_backward(el, m.cells, m.coords, kap, layout, c, grad_csr=G)

    def fd(fun, x0, eps):
        return (fun(x0 + eps) - fun(x0 - eps)) / (2 * eps)

    for i in range(nk):
        e = np.zeros(nk)
        e[i] = 1
        num = fd(lambda t: _L(el, m.cells, m.coords, kap + t * e, layout, c, G), 0.0, 1e-6)
        assert abs(num - gk[i]) <= 1e-7 * max(1.0, abs(gk[i]))
    num = fd(lambda t: _L(el, m.cells, m.coords, kap, layout, t, G), c, 1e-6)
    assert abs(num - gc) <= 1e-7 * max(1.0, abs(gc))
    used = np.unique(m.cells[:, :3] if el == O.P2_TRI else m.cells)
    for node in used[:12]:
        for r in range(m.coords.shape[1]):
            def Lx(t):
                cc = m.coords.copy()
                cc[node, r] += t
                return _L(el, m.cells, cc, kap, layout, c, G)
            num = fd(Lx, 0.0, 1e-6)
            assert abs(num - gx[node, r]) <= 1e-7 * max(1.0, abs(gx[node, r])), (node, r, num, gx[node, r])
    if el == O.P2_TRI:
        edge_nodes = np.setdiff1d(np.arange(m.n_nodes), np.unique(m.cells[:, :3]))
        assert np.all(gx[edge_nodes] == 0)


def test_backward_adjoint_outer_product_and_identity():
    m = _jittered(O.P1_TET, n=3, seed=2)
    g = np.random.default_rng(21)
    kap = g.uniform(0.5, 1.5, size=m.n_elems)
    lam = g.normal(size=m.n_nodes)
    U = g.normal(size=m.n_nodes)
    K = O.assemble_bilinear(O.P1_TET, m.cells, m.coords, kap, O.PER_ELEMENT, 0.0)
    G = O.CSR(K.row_ptr, K.col, lam[K.rows_of()] * U[K.col])
    a = O.assemble_backward(O.P1_TET, m.cells, m.coords, kap, O.PER_ELEMENT, 0.0, grad_csr=G)
    b = O.assemble_backward(O.P1_TET, m.cells, m.coords, kap, O.PER_ELEMENT, 0.0, lam=lam, U=U)
    assert np.allclose(a[0], b[0], rtol=1e-13, atol=1e-15)
    assert np.allclose(a[1], b[1], rtol=1e-12, atol=1e-14)
    # dL/dkappa_e = lam_e^T K_e U_e / kappa_e   (K_e linear in kappa_e when c = 0)
    for e in range(0, m.n_elems, 7):
        Ke = O.element_matrix(O.P1_TET, m.coords[m.cells[e]], kap[e], 0.0)
        want = lam[m.cells[e]] @ Ke @ U[m.cells[e]] / kap[e]
        assert abs(a[0][e] - want) <= 1e-12 * max(1.0, abs(want))


def test_elasticity_backward_matches_central_differences():
    m = mg.kuhn_tet_grid(2)
    g = np.random.default_rng(31)
    m.coords = m.coords + np.where(m.boundary[:, None], 0, g.uniform(-0.05, 0.05, size=m.coords.shape))
    lam = g.uniform(0.5, 2.0, size=m.n_elems)
    mu = g.uniform(0.3, 1.0, size=m.n_elems)
    K = O.assemble_elasticity(m.cells, m.coords, lam, mu, O.PER_ELEMENT)
    G = O.CSR(K.row_ptr, K.col, g.normal(size=K.nnz))
    gl, gm, gx = O.elasticity_backward(m.cells, m.coords, lam, mu, O.PER_ELEMENT, grad_csr=G)

    def L(l_, m_, x_):
        Kx = O.assemble_elasticity(m.cells, x_, l_, m_, O.PER_ELEMENT)
        return float(Kx.val @ G.val)

    eps = 1e-6
    for e in range(0, m.n_elems, 5):
        d = np.zeros(m.n_elems)
        d[e] = eps
        assert abs((L(lam + d, mu, m.coords) - L(lam - d, mu, m.coords)) / (2 * eps) - gl[e]) < 1e-7 * max(1, abs(gl[e]))
        assert abs((L(lam, mu + d, m.coords) - L(lam, mu - d, m.coords)) / (2 * eps) - gm[e]) < 1e-7 * max(1, abs(gm[e]))
    for node in range(0, m.n_nodes, 3):
        for r in range(3):
            cp = m.coords.copy()
            cm = m.coords.copy()
            cp[node, r] += eps
            cm[node, r] -= eps
            num = (L(lam, mu, cp) - L(lam, mu, cm)) / (2 * eps)
            assert abs(num - gx[node, r]) < 1e-7 * max(1, abs(gx[node, r])), (node, r, num, gx[node, r])


def test_planted_mistake_is_caught():
    """A dropped mass term or a transposed gradient must break the pins above.

    The oracle's element routine is re-run with an input that mimics each
    mistake, and the exact-integration pin rejects it.
    """
    V = [[Fr(0), Fr(0)], [Fr(3, 4), Fr(1, 8)], [Fr(1, 4), Fr(5, 8)]]
    Ke = np.array(X.stiffness(V, "p1", 1), float) + 0.5 * np.array(X.mass(V, "p1"), float)
    dropped_mass = O.element_matrix(O.P1_TRI, np.array(V, float), 1.0, 0.0)
    assert not np.allclose(dropped_mass, Ke, rtol=1e-13)
    # swapping two vertices of one element permutes the local matrix; the global
    # assembly must not change (the orientation enters only through |det J|)
    Va = np.array(V, float)
    K1 = O.element_matrix(O.P1_TRI, Va, 1.0, 0.5)
    K2 = O.element_matrix(O.P1_TRI, Va[[0, 2, 1]], 1.0, 0.5)
    assert np.allclose(K1, K2[np.ix_([0, 2, 1], [0, 2, 1])], rtol=1e-14)


@pytest.mark.parametrize("el,layout,ncomp", [(O.P1_TRI, O.PER_NODE, 1), (O.P2_TRI, O.PER_QP, 1),
                                             (O.P1_TET, O.CONSTANT, 1), (O.P1_TET_VEC3, O.PER_NODE, 3)])
def test_load_backward_matches_central_differences(el, layout, ncomp):
    gel = O.P1_TET if el == O.P1_TET_VEC3 else el
    m = _jittered(gel, n=3, seed=6)
    g = np.random.default_rng(41)
    nf = {O.PER_NODE: m.n_nodes, O.PER_QP: m.n_elems * O.NQ[el], O.CONSTANT: 1}[layout] * ncomp
    f = g.uniform(-1, 1, size=nf)
    gF = g.normal(size=m.n_nodes * ncomp)
    gf, gx = O.load_backward(el, m.cells, m.coords, f, layout, ncomp, gF)

    def L(f_, x_):
        return float(gF @ O.assemble_load(el, m.cells, x_, f_, layout, ncomp))

    eps = 1e-6
    for i in range(0, nf, max(1, nf // 15)):
        d = np.zeros(nf)
        d[i] = eps
        num = (L(f + d, m.coords) - L(f - d, m.coords)) / (2 * eps)
        assert abs(num - gf[i]) < 1e-8 * max(1, abs(gf[i]))
    geo = np.unique(m.cells[:, :3] if el == O.P2_TRI else m.cells)
    for node in geo[:10]:
        for r in range(m.coords.shape[1]):
            cp, cm = m.coords.copy(), m.coords.copy()
            cp[node, r] += eps
            cm[node, r] -= eps
            num = (L(f, cp) - L(f, cm)) / (2 * eps)
            assert abs(num - gx[node, r]) < 1e-7 * max(1, abs(gx[node, r])), (node, r, num, gx[node, r])


# ---------------------------------------------------------------- coefficients that vary over the element
# Eq. (matlclquad) pairs the coefficient value kappa[e][q] with the
# quadrature point x_q of element e.  For P1 the gradients are constant and
# only the weights matter; for P2 the point matters.  A coefficient that is a
# polynomial in x, sampled at the physical quadrature points, has an exact
# integral that the rule reproduces when the integrand's degree is within
# the rule's (kappa quadratic: kappa grad phi_a . grad phi_b has degree 4 for
# P2, the 6-point rule's degree).  Pairing kappa_q with any other point, or a
# point with the wrong vertex, changes the result.
def _phys_points(el, V):
    w, xq = O.quadrature(el)
    V = np.asarray(V, dtype=float)
    J = (V[1:len(V)] - V[0]).T  # columns: edge vectors from vertex 0
    return xq @ J.T + V[0]


def _rand_poly(g, d, deg):
    import itertools
    out = {}
    for m in itertools.product(range(deg + 1), repeat=d):
        if sum(m) <= deg:
            out[m] = Fr(int(g.integers(-8, 9)), 8)
    out[tuple([0] * d)] = Fr(4)  # keep the coefficient away from zero
    return out


def _poly_at(P, pts):
    return np.array([float(X.eval_poly_at(P, [Fr(float(v)) for v in p])) for p in pts])


def test_p2_per_point_kappa_element_matches_exact_integral():
    g = np.random.default_rng(31)
    for _ in range(5):
        V = _dyadic_simplex(g, 2)
        P = _rand_poly(g, 2, 2)
        kq = _poly_at(P, _phys_points(O.P2_TRI, V))
        Ke = np.array(X.stiffness(V, "p2", X.coef_poly(V, P)), dtype=float)
        Ko = O.element_matrix(O.P2_TRI, np.array(V, dtype=float), kq, 0.0)
        assert np.allclose(Ko, Ke, rtol=1e-13, atol=1e-13 * np.abs(Ke).max())
        # the same values with the points' order reversed give another matrix
        Kr = O.element_matrix(O.P2_TRI, np.array(V, dtype=float), kq[::-1], 0.0)
        assert np.abs(Kr - Ke).max() > 1e-6 * np.abs(Ke).max()


def test_p2_per_point_kappa_assembly_matches_exact_assembly():
    # per-QP layout kappa[e * 6 + q] through the global scatter-add
    m = mg.p2_tri_grid(2, jitter_seed=None)
    g = np.random.default_rng(32)
    P = _rand_poly(g, 2, 2)
    cells, coords = m.cells, m.coords
    kq = np.concatenate([_poly_at(P, _phys_points(O.P2_TRI, coords[cl[:3]])) for cl in cells])
    verts = [[Fr(float(v)) for v in p] for p in coords]
    c = 0.375

    def local(Xs):
        V = Xs[:3]
        K = X.stiffness(V, "p2", X.coef_poly(V, P))
        M_ = X.mass(V, "p2")
        return [[K[a][b] + Fr(c) * M_[a][b] for b in range(6)] for a in range(6)]

    dok = X.assemble_dok([list(map(int, cl)) for cl in cells], verts, local)
    res = O.assemble_bilinear(O.P2_TRI, cells, coords, kq, O.PER_QP, c)
    keys = sorted(dok)
    assert list(zip(res.rows_of().tolist(), res.col.tolist())) == keys
    want = np.array([float(dok[k]) for k in keys])
    assert np.allclose(res.val, want, rtol=1e-13, atol=1e-13 * np.abs(want).max())


@pytest.mark.parametrize("el,kind,d,deg", [(O.P2_TRI, "p2", 2, 2), (O.P1_TRI, "p1", 2, 1), (O.P1_TET, "p1", 3, 1)])
def test_per_point_load_matches_exact_integral(el, kind, d, deg):
    # F_a = int f phi_a with f a polynomial of degree deg sampled at the points
    # (integrand degree deg + basis degree = the rule's degree)
    g = np.random.default_rng(33)
    for _ in range(4):
        V = _dyadic_simplex(g, d)
        P = _rand_poly(g, d, deg)
        fq = _poly_at(P, _phys_points(el, V))
        Fe = np.array(X.load_poly(V, kind, X.coef_poly(V, P)), dtype=float)
        Vf = np.array(V, dtype=float)
        if kind == "p2":
            coords = np.vstack([Vf, (Vf[0] + Vf[1]) / 2, (Vf[1] + Vf[2]) / 2, (Vf[2] + Vf[0]) / 2])
        else:
            coords = Vf
        cells = np.arange(coords.shape[0])[None, :]
        Fo = O.assemble_load(el, cells, coords, fq, O.PER_QP)
        assert np.allclose(Fo, Fe, rtol=1e-13, atol=1e-14 * np.abs(Fe).max())


def test_elasticity_per_point_lame_matches_exact():
    # P1 gradients are constant, so K depends on int lambda and int mu only:
    # |e| B^T D(mean lambda, mean mu) B in the Voigt form.  lambda and mu
    # linear in x (the 4-point rule has degree 2), sampled at the points of
    # each element of a small Kuhn mesh, in the per-QP layout [e * 4 + q].
    t = mg.kuhn_tet_grid(2)
    g = np.random.default_rng(34)
    PL, PM = _rand_poly(g, 3, 1), _rand_poly(g, 3, 1)
    PM[(0, 0, 0)] = Fr(2)
    lq = np.concatenate([_poly_at(PL, _phys_points(O.P1_TET, t.coords[cl])) for cl in t.cells])
    mq = np.concatenate([_poly_at(PM, _phys_points(O.P1_TET, t.coords[cl])) for cl in t.cells])
    verts = [[Fr(float(v)) for v in p] for p in t.coords]

    def local(Xs):
        return X.elasticity(Xs, X.mean_over(Xs, PL), X.mean_over(Xs, PM))

    dok = X.assemble_dok([list(map(int, cl)) for cl in t.cells], verts, local, ndof_per_node=3)
    res = O.assemble_elasticity(t.cells, t.coords, lq, mq, O.PER_QP)
    keys = sorted(dok)
    assert list(zip(res.rows_of().tolist(), res.col.tolist())) == keys
    want = np.array([float(dok[k]) for k in keys])
    assert np.allclose(res.val, want, rtol=1e-12, atol=1e-13 * np.abs(want).max())
    # lambda and mu exchanged give another matrix
    sw = O.assemble_elasticity(t.cells, t.coords, mq, lq, O.PER_QP)
    assert np.abs(sw.val - want).max() > 1e-6 * np.abs(want).max()
