"""GPU parity of the boundary-facet terms (Neumann and Robin) against the
FP64 oracle, added onto the element assembly."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import meshgen as mg
import oracle as O
from gpu_helpers import TOL, dev, host_as, jittered_tet, jittered_tri, relfro

pytestmark = pytest.mark.gpu

DTYPES = [torch.float64, torch.float32]


@pytest.fixture(scope="module")
def tg():
    import paper_2602_05052_gb300 as tg
    return tg


def _mesh(el):
    return jittered_tri(40) if el == mg.P1_TRI else jittered_tet(8)


def _coef(layout, nf_count, nq, N, seed):
    g = np.random.default_rng(seed)
    if layout == mg.PER_QP:
        return g.uniform(0.5, 2.0, nf_count * nq)
    if layout == mg.PER_ELEMENT:
        return g.uniform(0.5, 2.0, nf_count)
    if layout == mg.PER_NODE:
        return g.uniform(-1.0, 1.0, N)
    return np.array([g.uniform(0.5, 2.0)])


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("gl", [mg.PER_NODE, mg.PER_QP, mg.CONSTANT])
@pytest.mark.parametrize("al", [mg.PER_ELEMENT, mg.PER_QP, mg.CONSTANT])
@pytest.mark.parametrize("el", [mg.P1_TRI, mg.P1_TET])
def test_facets_match_oracle(tg, el, al, gl, dtype):
    m = _mesh(el)
    fac = mg.boundary_facets(m)
    nq = 2 if el == mg.P1_TRI else 3
    alpha = _coef(al, len(fac), nq, m.n_nodes, seed=80 + al)
    gv = _coef(gl, len(fac), nq, m.n_nodes, seed=90 + gl)
    k = np.random.default_rng(5).uniform(0.5, 2.0, m.n_elems)
    f = np.random.default_rng(6).uniform(-1, 1, m.n_nodes)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, el)
    fc = tg.tg_build_facets(p, dev(fac, torch.int32))
    assert fc.n_facets == len(fac) and fc.n_boundary_nodes == int(m.boundary.sum())
    X = dev(m.coords, dtype)
    vals = tg.tg_assemble_bilinear(p, X, dev(k, dtype), mg.PER_ELEMENT, 0.3)
    F = tg.tg_assemble_load(p, X, dev(f, dtype), mg.PER_NODE)
    tg.tg_assemble_facets(fc, X, dev(alpha, dtype), al, dev(gv, dtype), gl, vals, F)
    xs = host_as(m.coords, dtype)
    K = O.assemble_bilinear(el, m.cells, xs, host_as(k, dtype), O.PER_ELEMENT, 0.3)
    Mb, Fb = O.assemble_facets(el, fac, xs, host_as(alpha, dtype), al, host_as(gv, dtype), gl)
    want = K.val.copy()
    rows = K.rows_of()
    slot = {(int(r), int(c)): s for s, (r, c) in enumerate(zip(rows, K.col))}
    for key, v in Mb.items():
        want[slot[key]] += v
    Fw = O.assemble_load(el, m.cells, xs, host_as(f, dtype), O.PER_NODE) + Fb
    assert relfro(vals.cpu().numpy(), want) <= TOL[dtype]
    assert relfro(F.cpu().numpy(), Fw) <= TOL[dtype]
    # the boundary terms alone, against the oracle's
    zero = torch.zeros_like(vals)
    zF = torch.zeros_like(F)
    tg.tg_assemble_facets(fc, X, dev(alpha, dtype), al, dev(gv, dtype), gl, zero, zF)
    bw = np.zeros(K.nnz)
    for key, v in Mb.items():
        bw[slot[key]] += v
    assert relfro(zero.cpu().numpy(), bw) <= TOL[dtype]
    assert relfro(zF.cpu().numpy(), Fb) <= TOL[dtype]
    assert tg.tg_get_device_status(p) == (0, -1)


def test_facets_are_deterministic(tg):
    m = jittered_tri(64)
    fac = mg.boundary_facets(m)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TRI)
    fc = tg.tg_build_facets(p, dev(fac, torch.int32))
    X = dev(m.coords, torch.float32)
    al = dev(np.random.default_rng(1).uniform(0.5, 2, len(fac) * 2), torch.float32)
    gv = dev(np.random.default_rng(2).uniform(-1, 1, m.n_nodes), torch.float32)
    base = torch.randn(p.nnz, device="cuda")
    baseF = torch.randn(m.n_nodes, device="cuda")
    outs = []
    for _ in range(3):
        v, F = base.clone(), baseF.clone()
        tg.tg_assemble_facets(fc, X, al, mg.PER_QP, gv, mg.PER_NODE, v, F)
        outs.append((v, F))
    assert all(torch.equal(a[0], outs[0][0]) and torch.equal(a[1], outs[0][1]) for a in outs)


@pytest.mark.parametrize("el", [mg.P1_TRI, mg.P1_TET])
def test_robin_solution_reproduces_linear_field(tg, el):
    """Robin on the whole boundary, Laplace's equation, u = a.x + b: the
    GPU assembly (elements + facets) and CG reproduce u."""
    m = jittered_tri(24, hilbert=False) if el == mg.P1_TRI else jittered_tet(5)
    d = m.coords.shape[1]
    a = np.array([0.7, -1.3, 0.4][:d])
    alpha = 1.7
    fac = mg.boundary_facets(m)
    pts, gq = [], []
    for fv in fac:
        P = m.coords[fv]
        n = np.zeros(d)
        for k2 in range(d):
            if np.allclose(P[:, k2], 0.0):
                n[k2] = -1.0
            elif np.allclose(P[:, k2], 1.0):
                n[k2] = 1.0
        if len(fv) == 2:
            xq, _ = np.polynomial.legendre.leggauss(2)
            xs = [P[0] + (t + 1) / 2 * (P[1] - P[0]) for t in xq]
        else:
            _, xq = O.quadrature(O.P1_TRI)
            xs = [P[0] + x[0] * (P[1] - P[0]) + x[1] * (P[2] - P[0]) for x in xq]
        for x in xs:
            gq.append(a @ n + alpha * (x @ a + 0.25))
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, el)
    fc = tg.tg_build_facets(p, dev(fac, torch.int32))
    X = dev(m.coords, torch.float64)
    vals = tg.tg_assemble_bilinear(p, X, dev([1.0], torch.float64), mg.CONSTANT, 0.0)
    F = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
    tg.tg_assemble_facets(fc, X, dev([alpha], torch.float64), mg.CONSTANT, dev(np.array(gq), torch.float64),
                          mg.PER_QP, vals, F)
    u, it, rel = tg.tg_cg_solve(p, vals, F, rtol=1e-13)
    assert np.abs(u.cpu().numpy() - (m.coords @ a + 0.25)).max() < 1e-9


def test_facet_build_errors(tg):
    m = jittered_tri(6)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TRI)
    for bad, code in (([[0, m.n_nodes]], "INDEX_RANGE"), ([[3, 3]], "DEGENERATE"), ([[0, m.n_nodes - 1]], "INVALID")):
        with pytest.raises(tg.TGError) as e:
            tg.tg_build_facets(p, dev(np.array(bad), torch.int32))
        assert code in str(e.value)
    m2 = mg.p2_tri_grid(3)
    p2 = tg.tg_build_pattern(dev(m2.cells, torch.int32), m2.n_nodes, mg.P2_TRI)
    with pytest.raises(tg.TGError):
        tg.tg_build_facets(p2, dev(np.array([[0, 1]]), torch.int32))
    # an empty facet set is valid and does nothing
    fc = tg.tg_build_facets(p, torch.empty((0, 2), dtype=torch.int32, device="cuda"))
    v = torch.ones(p.nnz, dtype=torch.float64, device="cuda")
    tg.tg_assemble_facets(fc, dev(m.coords, torch.float64), dev([1.0], torch.float64), mg.CONSTANT, vals=v)
    assert torch.equal(v, torch.ones_like(v))


def test_degenerate_facet_is_flagged(tg):
    cells = np.array([[0, 1, 2]])
    X = np.array([[0, 0], [1, 0], [0, 1]], float)
    p = tg.tg_build_pattern(dev(cells, torch.int32), 3, mg.P1_TRI)
    fc = tg.tg_build_facets(p, dev(np.array([[0, 1], [1, 2]]), torch.int32))
    Xd = X.copy()
    Xd[2] = Xd[1]  # edge (1, 2) has zero length
    v = torch.zeros(p.nnz, dtype=torch.float64, device="cuda")
    tg.tg_assemble_facets(fc, dev(Xd, torch.float64), dev([1.0], torch.float64), mg.CONSTANT, vals=v)
    assert tg.tg_get_device_status(p) == (3, 1)
