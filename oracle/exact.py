"""Exact rational element matrices (TEST INFRASTRUCTURE ONLY).

An independent route to the local matrices of Eq. (matlclquad): no
quadrature, no reference element and no Jacobian inverse in floating point.
Basis functions are polynomials in the barycentric coordinates l_i of the
physical simplex; their gradients follow from the chain rule
grad(phi) = sum_j (d phi / d l_j) grad(l_j), with grad(l_j) read off the
exact inverse of the vertex matrix [[1 ...], [x ...], [y ...]].  Products are
integrated exactly with the simplex monomial formula

    int_T prod_i l_i^{a_i} = d! |T| prod_i a_i! / (sum_i a_i + d)!

Elasticity is formed as B^T D B with the Voigt strain vector
(e_xx, e_yy, e_zz, g_yz, g_xz, g_xy) and Hooke's matrix D(lambda, mu),
a different formulation from the index form used in the C++ oracle.

Coordinates must be given as Fractions (or integers) for exact results.
"""
from __future__ import annotations

from fractions import Fraction as Fr
from math import factorial


def _inv(M):
    n = len(M)
    A = [[Fr(v) for v in row] + [Fr(int(i == j)) for j in range(n)] for i, row in enumerate(M)]
    for c in range(n):
        p = next(r for r in range(c, n) if A[r][c] != 0)
        A[c], A[p] = A[p], A[c]
        piv = A[c][c]
        A[c] = [v / piv for v in A[c]]
        for r in range(n):
            if r != c and A[r][c] != 0:
                f = A[r][c]
                A[r] = [vr - f * vc for vr, vc in zip(A[r], A[c])]
    return [row[n:] for row in A]


def _det(M):
    n = len(M)
    if n == 1:
        return Fr(M[0][0])
    s = Fr(0)
    for j in range(n):
        minor = [row[:j] + row[j + 1:] for row in M[1:]]
        s += (-1) ** j * Fr(M[0][j]) * _det(minor)
    return s


class Simplex:
    def __init__(self, verts):
        self.v = [[Fr(c) for c in p] for p in verts]
        self.d = len(self.v[0])
        assert len(self.v) == self.d + 1
        T = [[Fr(1)] * (self.d + 1)] + [[self.v[k][r] for k in range(self.d + 1)] for r in range(self.d)]
        Ti = _inv(T)
        # l = Ti @ [1, x, y(, z)]  ->  grad l_i = Ti[i][1:]
        self.grad_l = [Ti[i][1:] for i in range(self.d + 1)]
        self.vol = abs(_det([[self.v[k + 1][r] - self.v[0][r] for k in range(self.d)] for r in range(self.d)])) / factorial(self.d)

    def integrate(self, poly):
        """poly: dict {exponent tuple (len d+1): coefficient}."""
        d = self.d
        s = Fr(0)
        for a, c in poly.items():
            num = 1
            for ai in a:
                num *= factorial(ai)
            s += c * Fr(factorial(d) * num, factorial(sum(a) + d))
        return s * self.vol


def _mul(p, q):
    out = {}
    for a, ca in p.items():
        for b, cb in q.items():
            k = tuple(x + y for x, y in zip(a, b))
            out[k] = out.get(k, 0) + ca * cb
    return out


def _add(p, q, s=1):
    out = dict(p)
    for k, v in q.items():
        out[k] = out.get(k, 0) + s * v
    return out


def _diff(p, j):
    out = {}
    for a, c in p.items():
        if a[j] > 0:
            k = list(a)
            k[j] -= 1
            k = tuple(k)
            out[k] = out.get(k, 0) + c * a[j]
    return out


def _lam(i, n):
    return {tuple(int(k == i) for k in range(n)): Fr(1)}


def _one(n):
    return {tuple([0] * n): Fr(1)}


def basis_polys(kind: str, d: int):
    """Barycentric polynomial basis: 'p1' (any d) or 'p2' (triangles)."""
    n = d + 1
    if kind == "p1":
        return [_lam(i, n) for i in range(n)]
    assert kind == "p2" and d == 2
    L = [_lam(i, 3) for i in range(3)]
    verts = [_add(_mul(L[i], {k: 2 * v for k, v in L[i].items()}), L[i], -1) for i in range(3)]
    edges = [{k: 4 * v for k, v in _mul(L[a], L[b]).items()} for a, b in ((0, 1), (1, 2), (2, 0))]
    return verts + edges


def _grad_terms(S: Simplex, p):
    """grad p as a list over spatial r of polynomials."""
    n = S.d + 1
    out = []
    for r in range(S.d):
        acc = {}
        for j in range(n):
            dj = _diff(p, j)
            g = S.grad_l[j][r]
            if g != 0 and dj:
                acc = _add(acc, {k: v * g for k, v in dj.items()})
        out.append(acc)
    return out


def stiffness(verts, kind="p1", kappa=1):
    """K_ab = int kappa grad phi_a . grad phi_b.  kappa is a constant, or a
    polynomial in the barycentric coordinates of the simplex (a dict, see
    ``coef_poly``) for a coefficient that varies over the element."""
    S = Simplex(verts)
    B = basis_polys(kind, S.d)
    G = [_grad_terms(S, b) for b in B]
    k = len(B)
    kp = kappa if isinstance(kappa, dict) else {tuple([0] * (S.d + 1)): Fr(kappa)}
    K = [[Fr(0)] * k for _ in range(k)]
    for a in range(k):
        for b in range(k):
            s = Fr(0)
            for r in range(S.d):
                s += S.integrate(_mul(kp, _mul(G[a][r], G[b][r])))
            K[a][b] = s
    return K


def coef_poly(verts, coeffs):
    """A polynomial coefficient c(x) = sum_m coeffs[m] * x^m (m an exponent
    tuple over the spatial coordinates) written in the barycentric
    coordinates of the simplex, using x_r = sum_i l_i v_i[r]."""
    n = len(verts)
    xs = [{tuple(int(k == i) for k in range(n)): Fr(verts[i][r]) for i in range(n)} for r in range(len(verts[0]))]
    out = {}
    for m, c in coeffs.items():
        term = {tuple([0] * n): Fr(c)}
        for r, e in enumerate(m):
            for _ in range(e):
                term = _mul(term, xs[r])
        out = _add(out, term)
    return out


def eval_poly_at(coeffs, x):
    """sum_m coeffs[m] * x^m at a point given as Fractions."""
    s = Fr(0)
    for m, c in coeffs.items():
        t = Fr(c)
        for r, e in enumerate(m):
            t *= Fr(x[r]) ** e
        s += t
    return s


def load_poly(verts, kind, f_bary):
    """F_a = int f phi_a for f given as a barycentric polynomial."""
    S = Simplex(verts)
    return [S.integrate(_mul(f_bary, p)) for p in basis_polys(kind, S.d)]


def mean_over(verts, coeffs):
    """(1/|T|) int_T c(x) for a spatial polynomial c."""
    S = Simplex(verts)
    return S.integrate(coef_poly(verts, coeffs)) / S.vol


def mass(verts, kind="p1"):
    S = Simplex(verts)
    B = basis_polys(kind, S.d)
    k = len(B)
    return [[S.integrate(_mul(B[a], B[b])) for b in range(k)] for a in range(k)]


def load(verts, kind="p1", f=1):
    """F_a = f * int phi_a (constant f)."""
    S = Simplex(verts)
    return [Fr(f) * S.integrate(p) for p in basis_polys(kind, S.d)]


def elasticity(verts, lam, mu):
    """P1 tetrahedron, V * B^T D B with Voigt strains; DoF index 3a + i."""
    S = Simplex(verts)
    assert S.d == 3
    g = S.grad_l
    lam, mu = Fr(lam), Fr(mu)
    D = [[lam + 2 * mu, lam, lam, 0, 0, 0],
         [lam, lam + 2 * mu, lam, 0, 0, 0],
         [lam, lam, lam + 2 * mu, 0, 0, 0],
         [0, 0, 0, mu, 0, 0],
         [0, 0, 0, 0, mu, 0],
         [0, 0, 0, 0, 0, mu]]
    Bm = [[Fr(0)] * 12 for _ in range(6)]
    for a in range(4):
        gx, gy, gz = g[a]
        c = 3 * a
        Bm[0][c + 0] = gx
        Bm[1][c + 1] = gy
        Bm[2][c + 2] = gz
        Bm[3][c + 1] = gz
        Bm[3][c + 2] = gy
        Bm[4][c + 0] = gz
        Bm[4][c + 2] = gx
        Bm[5][c + 0] = gy
        Bm[5][c + 1] = gx
    DB = [[sum(D[i][k] * Bm[k][j] for k in range(6)) for j in range(12)] for i in range(6)]
    return [[S.vol * sum(Bm[k][i] * DB[k][j] for k in range(6)) for j in range(12)] for i in range(12)]


def monomial_integral_ref(exps):
    """Exact integral of prod x_s^{e_s} over the reference simplex."""
    d = len(exps)
    num = 1
    for e in exps:
        num *= factorial(e)
    return Fr(num, factorial(sum(exps) + d))


def assemble_dok(cells, verts, local_fn, ndof_per_node=1):
    """Exact scatter-add of local matrices into a dict {(row, col): Fraction}."""
    dok = {}
    for cell in cells:
        X = [verts[v] for v in cell]
        K = local_fn(X)
        dofs = [ndof_per_node * v + i for v in cell for i in range(ndof_per_node)]
        for a, ga in enumerate(dofs):
            for b, gb in enumerate(dofs):
                dok[(ga, gb)] = dok.get((ga, gb), Fr(0)) + K[a][b]
    return dok
