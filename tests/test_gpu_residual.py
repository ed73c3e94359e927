"""GPU parity of the matrix-free residual y = K x - F of Eq. (res1) (and its
loss and reverse mode) against the FP64 oracle."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import meshgen as mg
import oracle as O
from gpu_helpers import LOSS_TOL, TOL, coef, dev, host_as, jittered_tri, mesh_for, rel_scalar, relfro

pytestmark = pytest.mark.gpu

DTYPES = [torch.float64, torch.float32]


@pytest.fixture(scope="module")
def tg():
    import paper_2602_05052_gb300 as tg
    return tg


def _inputs(m, el, layout, fl, seed):
    g = np.random.default_rng(seed)
    k = coef(layout, m.n_elems, mg.NQ[el], seed=seed + 1)
    x = g.uniform(-1, 1, m.n_nodes)
    if fl is None:
        f = None
    elif fl == mg.PER_NODE:
        f = g.uniform(-1, 1, m.n_nodes)
    elif fl == mg.PER_QP:
        f = g.uniform(-1, 1, m.n_elems * mg.NQ[el])
    else:
        f = np.array([0.7])
    return k, x, f


def _check(tg, p, m, el, layout, c, k, x, f, fl, dtype, dirichlet=None):
    dd = dev(dirichlet.astype(np.uint8), torch.uint8) if dirichlet is not None else None
    y, loss = tg.tg_residual(p, dev(m.coords, dtype), dev(k, dtype), layout, c, dev(x, dtype),
                             dev(f, dtype) if f is not None else None, fl if fl is not None else mg.PER_NODE, dd)
    want, wl = O.residual(el, m.cells, host_as(m.coords, dtype), host_as(k, dtype), layout, c, host_as(x, dtype),
                          host_as(f, dtype) if f is not None else None, fl if fl is not None else O.PER_NODE,
                          dirichlet)
    assert relfro(y.cpu().numpy(), want) <= TOL[dtype]
    assert rel_scalar(loss.item(), wl) <= LOSS_TOL[dtype]
    assert tg.tg_get_device_status(p) == (0, -1)
    return y, loss


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("fl", [None, mg.PER_NODE, mg.PER_QP, mg.CONSTANT])
@pytest.mark.parametrize("layout", [mg.PER_QP, mg.PER_ELEMENT, mg.CONSTANT])
@pytest.mark.parametrize("el", [mg.P1_TRI, mg.P1_TET])
def test_residual_p1_matches_oracle(tg, el, layout, fl, dtype):
    m = mesh_for(el)
    k, x, f = _inputs(m, el, layout, fl, seed=60 + el)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, el)
    assert p.n_blocks > 0
    _check(tg, p, m, el, layout, 0.6, k, x, f, fl, dtype, dirichlet=m.boundary)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("layout", [mg.PER_QP, mg.CONSTANT])
def test_residual_p2_matches_oracle(tg, layout, dtype):
    m = mesh_for(mg.P2_TRI)
    k, x, _ = _inputs(m, mg.P2_TRI, layout, None, seed=70)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P2_TRI)
    _check(tg, p, m, mg.P2_TRI, layout, 0.4, k, x, None, None, dtype)
    _check(tg, p, m, mg.P2_TRI, layout, 0.4, k, x, None, None, dtype, dirichlet=m.boundary)


@pytest.mark.parametrize("dtype", DTYPES)
def test_residual_is_bitwise_deterministic(tg, dtype):
    m = jittered_tri(64)
    k, x, f = _inputs(m, mg.P1_TRI, mg.PER_QP, mg.PER_NODE, seed=71)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TRI)
    args = (dev(m.coords, dtype), dev(k, dtype), mg.PER_QP, 1.0, dev(x, dtype), dev(f, dtype), mg.PER_NODE)
    y0, l0 = tg.tg_residual(p, *args)
    for _ in range(3):
        y1, l1 = tg.tg_residual(p, *args)
        assert torch.equal(y0, y1) and torch.equal(l0, l1)


def test_residual_without_row_blocks(tg):
    """A random numbering of a 90,601-node mesh leaves the pattern without
    row blocks: the two-pass kernels serve the call, with the same bits as
    the row-block kernel on the same elements (only the node numbering
    differs)."""
    m = jittered_tri(300)
    g = np.random.default_rng(72)
    relabel = g.permutation(m.n_nodes)
    cells = relabel[m.cells]
    X = np.empty_like(m.coords)
    X[relabel] = m.coords
    k, x, f = _inputs(m, mg.P1_TRI, mg.PER_QP, mg.PER_NODE, seed=73)
    xr, fr = np.empty_like(x), np.empty_like(f)
    xr[relabel], fr[relabel] = x, f
    dirichlet = np.zeros(m.n_nodes, bool)
    dirichlet[relabel[m.boundary]] = True
    p = tg.tg_build_pattern(dev(cells, torch.int32), m.n_nodes, mg.P1_TRI)
    assert p.n_blocks == 0
    for dt in DTYPES:
        y, loss = tg.tg_residual(p, dev(X, dt), dev(k, dt), mg.PER_QP, 0.2, dev(xr, dt), dev(fr, dt), mg.PER_NODE,
                                 dev(dirichlet.astype(np.uint8), torch.uint8))
        want, wl = O.residual(mg.P1_TRI, cells, host_as(X, dt), host_as(k, dt), O.PER_QP, 0.2, host_as(xr, dt),
                              host_as(fr, dt), O.PER_NODE, dirichlet)
        assert relfro(y.cpu().numpy(), want) <= TOL[dt] and rel_scalar(loss.item(), wl) <= LOSS_TOL[dt]
        q = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TRI)
        assert q.n_blocks > 0
        yb, lb = tg.tg_residual(q, dev(m.coords, dt), dev(k, dt), mg.PER_QP, 0.2, dev(x, dt), dev(f, dt),
                                mg.PER_NODE, dev(m.boundary.astype(np.uint8), torch.uint8))
        assert torch.equal(y[torch.as_tensor(relabel, device="cuda")], yb)


def test_reverse_mode_and_gradcheck(tg):
    from paper_2602_05052_gb300 import autograd as A
    m = jittered_tri(6)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TRI)
    g = np.random.default_rng(74)
    mask = dev(m.boundary.astype(np.uint8), torch.uint8)
    coords = dev(m.coords, torch.float64).requires_grad_(True)
    k = dev(g.uniform(0.5, 2, m.n_elems * 3), torch.float64).requires_grad_(True)
    x = dev(g.uniform(-1, 1, m.n_nodes), torch.float64).requires_grad_(True)
    f = dev(g.uniform(-1, 1, m.n_nodes), torch.float64).requires_grad_(True)
    fn = lambda c_, k_, x_, f_: A.residual(p, c_, k_, mg.PER_QP, 0.3, x_, f_, mg.PER_NODE, mask)
    assert torch.autograd.gradcheck(fn, (coords, k, x, f), eps=1e-6, atol=1e-8)
    # dL/dx of L = ||y||^2 is 2 K (masked y): the oracle's matrix applied to the oracle's residual
    y = fn(coords, k, x, f)
    (y * y).sum().backward()
    yo, _ = O.residual(mg.P1_TRI, m.cells, m.coords, k.detach().cpu().numpy(), O.PER_QP, 0.3,
                       x.detach().cpu().numpy(), f.detach().cpu().numpy(), O.PER_NODE, m.boundary)
    K = O.assemble_bilinear(mg.P1_TRI, m.cells, m.coords, k.detach().cpu().numpy(), O.PER_QP, 0.3).to_scipy()
    assert relfro(x.grad.cpu().numpy(), 2 * (K @ yo)) <= 1e-12


def test_solve_assembled_gradient_in_f(tg):
    from paper_2602_05052_gb300 import autograd as A
    m = jittered_tri(5)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TRI)
    mask = dev(m.boundary.astype(np.uint8), torch.uint8)
    g = np.random.default_rng(75)
    coords = dev(m.coords, torch.float64)
    k = dev(g.uniform(0.5, 2, m.n_elems), torch.float64)
    f = dev(g.uniform(-1, 1, m.n_nodes), torch.float64).requires_grad_(True)
    fn = lambda f_: A.solve_assembled(p, coords, k, mg.PER_ELEMENT, f_, mg.PER_NODE, mask, rtol=1e-14)
    assert torch.autograd.gradcheck(fn, (f,), eps=1e-6, atol=1e-8)


def test_residual_diffusion2d_full_size(tg):
    """The 1024^2 workload in FP32 against the oracle on every row."""
    cfg = mg.diffusion2d(1024)
    m = cfg["mesh"]
    g = np.random.default_rng(76)
    x = g.uniform(-1, 1, m.n_nodes)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TRI)
    _check(tg, p, m, mg.P1_TRI, mg.PER_QP, cfg["c"], cfg["kappa"], x, cfg["f"], mg.PER_NODE, torch.float32,
           dirichlet=m.boundary)


def test_edge_cases(tg):
    # isolated nodes only: y = 0 and loss = 0
    p = tg.tg_build_pattern(torch.empty((0, 3), dtype=torch.int32, device="cuda"), 5, mg.P1_TRI)
    y, loss = tg.tg_residual(p, dev(np.zeros((5, 2)), torch.float64), dev([1.0], torch.float64), mg.CONSTANT, 1.0,
                             dev(np.ones(5), torch.float64))
    assert torch.equal(y, torch.zeros_like(y)) and loss.item() == 0.0
    # one element and isolated nodes beside it
    cells = np.array([[0, 2, 4]])
    X = np.array([[0, 0], [5, 5], [1, 0], [6, 6], [0, 1]], float)
    p = tg.tg_build_pattern(dev(cells, torch.int32), 5, mg.P1_TRI)
    x = np.array([0.5, 9.0, -1.0, 9.0, 2.0])
    y, loss = tg.tg_residual(p, dev(X, torch.float64), dev([1.5], torch.float64), mg.CONSTANT, 0.25,
                             dev(x, torch.float64), dev([1.0], torch.float64), mg.CONSTANT)
    want, wl = O.residual(mg.P1_TRI, cells, X, np.array([1.5]), O.CONSTANT, 0.25, x, np.array([1.0]), O.CONSTANT)
    assert np.allclose(y.cpu().numpy(), want, rtol=1e-14, atol=1e-15) and abs(loss.item() - wl) <= 1e-13 * wl
    assert y[1].item() == 0.0 and y[3].item() == 0.0
    # a degenerate element is flagged
    Xd = X.copy()
    Xd[4] = [2, 0]
    tg.tg_residual(p, dev(Xd, torch.float64), dev([1.0], torch.float64), mg.CONSTANT, 0.0, dev(x, torch.float64))
    assert tg.tg_get_device_status(p) == (3, 0)


def test_invalid_arguments(tg):
    m = jittered_tri(4)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TRI)
    X, k = dev(m.coords, torch.float64), dev([1.0], torch.float64)
    x = dev(np.ones(m.n_nodes), torch.float64)
    with pytest.raises(tg.TGError):
        tg.tg_residual(p, X, k, mg.CONSTANT, 0.0, x, y=x)  # x and y alias
    with pytest.raises(tg.TGError):
        tg.tg_residual(p, X, k, mg.PER_NODE, 0.0, x)  # no nodal kappa
    m2 = mesh_for(mg.P2_TRI)
    p2 = tg.tg_build_pattern(dev(m2.cells, torch.int32), m2.n_nodes, mg.P2_TRI)
    with pytest.raises(tg.TGError):
        tg.tg_residual(p2, dev(m2.coords, torch.float64), k, mg.CONSTANT, 0.0, dev(np.ones(m2.n_nodes), torch.float64),
                       f=k, f_layout=mg.CONSTANT)  # load term on P2
