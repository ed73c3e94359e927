"""FP64 CPU oracle for Galerkin assembly (TEST INFRASTRUCTURE ONLY).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never calls it, and it
shares no code, header or constant with the GPU library.

* ``tg_oracle.cpp`` — the C++ scatter-add into a dictionary of keys (DOK),
  Eq. (scatter_add) with local matrices from Eq. (matlclquad); the load
  vector; analytic gradients; vector P1 elasticity (Hooke's law, SM B.1).
* ``exact.py`` — exact rational element matrices by monomial integration
  (independent of quadrature), used to pin the C++ oracle on tiny meshes.
* ``solve.py`` — conjugate gradients on the Dirichlet-condensed system.
* ``residual()`` — the residual vector of Eq. (res1), K x - F, from the
  assembled oracle matrix and load vector.
* ``reaction_load()``, ``semilinear_residual()`` — the semilinear reaction
  term of the method of lines by quadrature, and the residual with it.
* ``assemble_facets()`` — the Neumann and Robin boundary terms by
  scatter-add over boundary facets (edge: Gauss-Legendre; face: the
  triangle rule).

Parity of every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants, exact integration and finite differences.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tg_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libtg_oracle.so")

P1_TRI, P2_TRI, P1_TET, P1_TET_VEC3 = 0, 1, 2, 3
PER_ELEMENT, PER_QP, PER_NODE, CONSTANT = 0, 1, 2, 3
NV = {P1_TRI: 3, P2_TRI: 6, P1_TET: 4, P1_TET_VEC3: 4}
DIM = {P1_TRI: 2, P2_TRI: 2, P1_TET: 3, P1_TET_VEC3: 3}
NQ = {P1_TRI: 3, P2_TRI: 6, P1_TET: 4, P1_TET_VEC3: 4}


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (FP64, no contraction, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
                        _SRC, "-o", tmp], check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        d, i64, i32, vp = C.c_double, C.c_int64, C.c_int, C.c_void_p
        L.orc_quadrature.restype = i32
        L.orc_quadrature.argtypes = [i32, vp, vp]
        L.orc_basis.argtypes = [i32, vp, vp, vp]
        L.orc_element_matrix.argtypes = [i32, vp, vp, d, vp]
        L.orc_elastic_element_matrix.argtypes = [vp, vp, vp, vp]
        L.orc_assemble_bilinear.restype = vp
        L.orc_assemble_bilinear.argtypes = [i32, i64, i64, vp, vp, vp, i32, d, vp]
        L.orc_assemble_elasticity.restype = vp
        L.orc_assemble_elasticity.argtypes = [i64, i64, vp, vp, vp, vp, i32, vp]
        L.orc_csr_nrows.restype = i64
        L.orc_csr_nrows.argtypes = [vp]
        L.orc_csr_nnz.restype = i64
        L.orc_csr_nnz.argtypes = [vp]
        L.orc_csr_export.argtypes = [vp, vp, vp, vp]
        L.orc_csr_free.argtypes = [vp]
        L.orc_assemble_load.argtypes = [i32, i64, i64, vp, vp, vp, i32, i32, vp]
        L.orc_assemble_backward.restype = i32
        L.orc_assemble_backward.argtypes = [i32, i64, i64, vp, vp, vp, i32, d, vp, vp, vp, vp, vp, vp, vp, vp]
        L.orc_load_backward.restype = i32
        L.orc_load_backward.argtypes = [i32, i64, i64, vp, vp, vp, i32, i32, vp, vp, vp]
        L.orc_elasticity_backward.restype = i32
        L.orc_elasticity_backward.argtypes = [i64, i64, vp, vp, vp, vp, i32, vp, vp, vp, vp, vp, vp, vp, vp]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


class CSR:
    """CSR export of the oracle's DOK (int64 row pointers, int32 columns)."""

    def __init__(self, row_ptr, col, val):
        self.row_ptr, self.col, self.val = row_ptr, col, val

    @property
    def nnz(self):
        return int(self.col.shape[0])

    @property
    def n_rows(self):
        return int(self.row_ptr.shape[0] - 1)

    def to_scipy(self, n_cols=None):
        import scipy.sparse as sp
        n = self.n_rows
        return sp.csr_matrix((self.val, self.col, self.row_ptr), shape=(n, n_cols or n))

    def rows_of(self):
        return np.repeat(np.arange(self.n_rows), np.diff(self.row_ptr))


def _export(h) -> CSR:
    L = lib()
    n = L.orc_csr_nrows(h)
    nnz = L.orc_csr_nnz(h)
    rp = np.empty(n + 1, np.int64)
    col = np.empty(nnz, np.int32)
    val = np.empty(nnz, np.float64)
    L.orc_csr_export(h, _p(rp), _p(col), _p(val))
    L.orc_csr_free(h)
    return CSR(rp, col, val)


def quadrature(el: int):
    w = np.zeros(8)
    x = np.zeros(24)
    nq = lib().orc_quadrature(el, _p(w), _p(x))
    d = DIM[el]
    return w[:nq].copy(), x[: nq * d].reshape(nq, d).copy()


def basis(el: int, x):
    x = _f64(x)
    phi = np.zeros(6)
    dphi = np.zeros(18)
    lib().orc_basis(el, _p(x), _p(phi), _p(dphi))
    nv = NV[el]
    return phi[:nv].copy(), dphi[: nv * DIM[el]].reshape(nv, DIM[el]).copy()


def element_matrix(el: int, X, kq, c: float = 0.0):
    X = _f64(X)
    kq = _f64(np.broadcast_to(np.asarray(kq, dtype=np.float64), (NQ[el],)))
    nv = NV[el]
    K = np.zeros(nv * nv)
    lib().orc_element_matrix(el, _p(X), _p(kq), float(c), _p(K))
    return K.reshape(nv, nv)


def elastic_element_matrix(X, lam, mu):
    X = _f64(X)
    lq = _f64(np.broadcast_to(np.asarray(lam, dtype=np.float64), (4,)))
    mq = _f64(np.broadcast_to(np.asarray(mu, dtype=np.float64), (4,)))
    K = np.zeros(144)
    lib().orc_elastic_element_matrix(_p(X), _p(lq), _p(mq), _p(K))
    return K.reshape(12, 12)


def assemble_bilinear(el, cells, coords, kappa, kappa_layout, c=0.0, row_mask=None) -> CSR:
    cells = _i32(cells)
    coords = _f64(coords)
    kappa = _f64(np.atleast_1d(kappa))
    mask = None if row_mask is None else np.ascontiguousarray(row_mask, dtype=np.uint8)
    h = lib().orc_assemble_bilinear(el, cells.shape[0], coords.shape[0], _p(cells), _p(coords), _p(kappa),
                                    kappa_layout, float(c), _p(mask))
    return _export(h)


def assemble_elasticity(cells, coords, lam, mu, layout, row_mask=None) -> CSR:
    cells = _i32(cells)
    coords = _f64(coords)
    lam = _f64(np.atleast_1d(lam))
    mu = _f64(np.atleast_1d(mu))
    mask = None if row_mask is None else np.ascontiguousarray(row_mask, dtype=np.uint8)
    h = lib().orc_assemble_elasticity(cells.shape[0], coords.shape[0], _p(cells), _p(coords), _p(lam), _p(mu),
                                      layout, _p(mask))
    return _export(h)


def assemble_load(el, cells, coords, f, f_layout, ncomp=1):
    cells = _i32(cells)
    coords = _f64(coords)
    f = _f64(np.atleast_1d(f))
    N = coords.shape[0]
    F = np.zeros(N * ncomp)
    lib().orc_assemble_load(el, cells.shape[0], N, _p(cells), _p(coords), _p(f), f_layout, ncomp, _p(F))
    return F


def assemble_backward(el, cells, coords, kappa, kappa_layout, c, grad_csr: CSR | None = None, lam=None, U=None):
    """Returns (grad_kappa, grad_coords [N, d], grad_c)."""
    cells = _i32(cells)
    coords = _f64(coords)
    kappa = _f64(np.atleast_1d(kappa))
    E, N = cells.shape[0], coords.shape[0]
    nq = NQ[el]
    nk = E * nq if kappa_layout == PER_QP else E if kappa_layout == PER_ELEMENT else 1
    gk = np.zeros(nk)
    gx = np.zeros(N * DIM[el])
    gc = np.zeros(1)
    if grad_csr is not None:
        rp, col, val = grad_csr.row_ptr, grad_csr.col, _f64(grad_csr.val)
        lam_p = U_p = None
    else:
        rp = col = val = None
        lam_p, U_p = _f64(lam), _f64(U)
    lib().orc_assemble_backward(el, E, N, _p(cells), _p(coords), _p(kappa), kappa_layout, float(c), _p(rp), _p(col),
                                _p(val), _p(lam_p), _p(U_p), _p(gk), _p(gx), _p(gc))
    return gk, gx.reshape(N, DIM[el]), float(gc[0])


def elasticity_backward(cells, coords, lam, mu, layout, grad_csr: CSR | None = None, lam_adj=None, U=None):
    """Returns (grad_lam, grad_mu, grad_coords [N, 3])."""
    cells = _i32(cells)
    coords = _f64(coords)
    lam = _f64(np.atleast_1d(lam))
    mu = _f64(np.atleast_1d(mu))
    E, N = cells.shape[0], coords.shape[0]
    nc = E * 4 if layout == PER_QP else E
    gl = np.zeros(nc)
    gm = np.zeros(nc)
    gx = np.zeros(N * 3)
    if grad_csr is not None:
        rp, col, val = grad_csr.row_ptr, grad_csr.col, _f64(grad_csr.val)
        la = Up = None
    else:
        rp = col = val = None
        la, Up = _f64(lam_adj), _f64(U)
    lib().orc_elasticity_backward(E, N, _p(cells), _p(coords), _p(lam), _p(mu), layout, _p(rp), _p(col), _p(val),
                                  _p(la), _p(Up), _p(gl), _p(gm), _p(gx))
    return gl, gm, gx.reshape(N, 3)


def load_backward(el, cells, coords, f, f_layout, ncomp, gF):
    """Returns (grad_f, grad_coords [N, d]) of L = gF . F."""
    cells = _i32(cells)
    coords = _f64(coords)
    f = _f64(np.atleast_1d(f))
    gF = _f64(gF)
    E, N = cells.shape[0], coords.shape[0]
    nq = NQ[el]
    nf = E * nq * ncomp if f_layout == PER_QP else N * ncomp if f_layout == PER_NODE else ncomp
    gf = np.zeros(nf)
    d = DIM[el]
    gx = np.zeros(N * d)
    lib().orc_load_backward(el, E, N, _p(cells), _p(coords), _p(f), f_layout, ncomp, _p(gF), _p(gf), _p(gx))
    return gf, gx.reshape(N, d)


def residual(el, cells, coords, kappa, kappa_layout, c, x, f=None, f_layout=PER_NODE, dirichlet=None):
    """Residual of Eq. (res1): y = K(kappa, c) x - F(f) with K and F assembled
    by scatter-add (F omitted when f is None), y = 0 on the rows where
    dirichlet != 0 (the rows the reduced system drops), and the loss
    sum_i y_i^2.  Returns (y, loss)."""
    K = assemble_bilinear(el, cells, coords, kappa, kappa_layout, c).to_scipy()
    y = K @ _f64(x)
    if f is not None:
        y = y - assemble_load(el, cells, coords, f, f_layout)
    if dirichlet is not None:
        y[np.asarray(dirichlet) != 0] = 0.0
    return y, float(np.dot(y, y))


def _facet_rule(nf):
    """Quadrature on the reference facet: (points in facet barycentric-free
    coordinates, weights); the edge [0, 1] with 2 Gauss-Legendre points
    (weights sum to 1), or the reference triangle's rule (sum 1/2)."""
    if nf == 2:
        x, w = np.polynomial.legendre.leggauss(2)
        return ((x + 1.0) / 2.0)[:, None], w / 2.0
    w, x = quadrature(P1_TRI)
    return x, w


def _facet_basis(nf, xq):
    if nf == 2:
        return np.array([1.0 - xq[0], xq[0]])
    return np.array([1.0 - xq[0] - xq[1], xq[0], xq[1]])


def assemble_facets(el, facets, coords, alpha=None, alpha_layout=CONSTANT, g=None, g_layout=CONSTANT):
    """Boundary terms of the Robin condition kappa du/dn + alpha u = g and
    the Neumann condition kappa du/dn = g, facet by facet in input order:
      M[(g_a, g_b)] += sum_q w_q |J_f| alpha_q phi_a phi_b,
      F[g_a]        += sum_q w_q |J_f| g_q phi_a,
    |J_f| = edge length (triangles) or twice the face area (tetrahedra).
    alpha layouts PER_ELEMENT (per facet), PER_QP, CONSTANT; g layouts
    PER_NODE (facet interpolant), PER_QP, CONSTANT.  Returns (dict of matrix
    entries, F [N])."""
    facets = np.asarray(facets)
    X = _f64(coords)
    nf = facets.shape[1]
    assert nf == DIM[el]
    xq, wq = _facet_rule(nf)
    nq = len(wq)
    M = {}
    F = np.zeros(X.shape[0])
    for f, fv in enumerate(facets):
        P = X[fv]
        if nf == 2:
            J = float(np.linalg.norm(P[1] - P[0]))
        else:
            J = float(np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0])))
        for q in range(nq):
            phi = _facet_basis(nf, xq[q])
            if alpha is not None:
                a_ = np.atleast_1d(alpha)
                aq = a_[f * nq + q] if alpha_layout == PER_QP else a_[f] if alpha_layout == PER_ELEMENT else a_[0]
                for a in range(nf):
                    for b in range(nf):
                        key = (int(fv[a]), int(fv[b]))
                        M[key] = M.get(key, 0.0) + wq[q] * J * aq * phi[a] * phi[b]
            if g is not None:
                g_ = np.atleast_1d(g)
                if g_layout == PER_NODE:
                    gq = float(phi @ g_[fv])
                elif g_layout == PER_QP:
                    gq = g_[f * nq + q]
                else:
                    gq = g_[0]
                for a in range(nf):
                    F[fv[a]] += wq[q] * J * gq * phi[a]
    return M, F


def _abs_det(el, cells, X):
    """|det J_e| of every element from its geometric vertices."""
    if DIM[el] == 2:
        a, b, c = X[cells[:, 0]], X[cells[:, 1]], X[cells[:, 2]]
        e1, e2 = b - a, c - a
        return np.abs(e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0])
    a = X[cells[:, 0]]
    J = np.stack([X[cells[:, k]] - a for k in (1, 2, 3)], axis=2)
    return np.abs(np.linalg.det(J))


def reaction_load(el, cells, coords, x, reaction, x_react=None):
    """Reaction term of a semilinear form, element by element with the
    element's quadrature rule:
      N[g(a)] += |det J_e| sum_q w_q s_q phi_a(x_q),  u_q = sum_b phi_b(x_q) x[g(b)],
    s_q = r(u_q) with r(u) = sum_k reaction[k] u^k; with x_react, s_q =
    r'(ur_q) u_q (ur_q interpolating x_react): the Jacobian at x_react
    applied to x."""
    cells = np.asarray(cells, dtype=np.int64)
    X = _f64(coords)
    x = _f64(x)
    r = [float(v) for v in reaction]
    w, xq = quadrature(el)
    adet = _abs_det(el, cells, X)
    out = np.zeros(X.shape[0])
    nv = NV[el]
    for q in range(len(w)):
        phi, _ = basis(el, xq[q])
        u = sum(phi[b] * x[cells[:, b]] for b in range(nv))
        if x_react is None:
            s = r[0] + r[1] * u + r[2] * u ** 2 + r[3] * u ** 3
        else:
            xr = _f64(x_react)
            ur = sum(phi[b] * xr[cells[:, b]] for b in range(nv))
            s = (r[1] + 2 * r[2] * ur + 3 * r[3] * ur ** 2) * u
        for a in range(nv):
            np.add.at(out, cells[:, a], adet * w[q] * s * phi[a])
    return out


def semilinear_residual(el, cells, coords, kappa, kappa_layout, c, x, reaction, f=None, f_layout=PER_NODE,
                        dirichlet=None, x_react=None):
    """y = K x + N - F (N from reaction_load), y = 0 on Dirichlet rows;
    returns (y, sum y^2)."""
    y, _ = residual(el, cells, coords, kappa, kappa_layout, c, x, f, f_layout)
    y = y + reaction_load(el, cells, coords, x, reaction, x_react)
    if dirichlet is not None:
        y[np.asarray(dirichlet) != 0] = 0.0
    return y, float(np.dot(y, y))
