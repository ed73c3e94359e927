"""GPU parity of the semilinear residual (reaction term of the method of
lines and its Jacobian action) against the FP64 oracle."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import meshgen as mg
import oracle as O
from gpu_helpers import LOSS_TOL, TOL, dev, host_as, jittered_tri, mesh_for, rel_scalar, relfro

pytestmark = pytest.mark.gpu

DTYPES = [torch.float64, torch.float32]
R = [0.2, -0.9, 0.35, 1.1]


@pytest.fixture(scope="module")
def tg():
    import paper_2602_05052_gb300 as tg
    return tg


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("jac", [False, True])
@pytest.mark.parametrize("el", [mg.P1_TRI, mg.P2_TRI, mg.P1_TET])
def test_semilinear_matches_oracle(tg, el, jac, dtype):
    m = mesh_for(el)
    g = np.random.default_rng(100 + el)
    k = g.uniform(0.5, 2, m.n_elems * mg.NQ[el])
    x = g.uniform(-1, 1, m.n_nodes)
    xr = g.uniform(-1, 1, m.n_nodes) if jac else None
    f = g.uniform(-1, 1, m.n_nodes) if el != mg.P2_TRI else None
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, el)
    y, loss = tg.tg_semilinear_residual(p, dev(m.coords, dtype), dev(k, dtype), mg.PER_QP, 0.5, dev(x, dtype), R,
                                        dev(f, dtype) if f is not None else None, mg.PER_NODE,
                                        x_react=dev(xr, dtype) if jac else None,
                                        dirichlet=dev(m.boundary.astype(np.uint8), torch.uint8))
    want, wl = O.semilinear_residual(el, m.cells, host_as(m.coords, dtype), host_as(k, dtype), O.PER_QP, 0.5,
                                     host_as(x, dtype), R, host_as(f, dtype) if f is not None else None, O.PER_NODE,
                                     m.boundary, host_as(xr, dtype) if jac else None)
    assert relfro(y.cpu().numpy(), want) <= TOL[dtype]
    assert rel_scalar(loss.item(), wl) <= LOSS_TOL[dtype]
    assert tg.tg_get_device_status(p) == (0, -1)


@pytest.mark.parametrize("el", [mg.P1_TRI, mg.P2_TRI, mg.P1_TET])
def test_reaction_points_match_oracle_interpolation(tg, el):
    m = mesh_for(el)
    x = np.random.default_rng(104).uniform(-1, 1, m.n_nodes)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, el)
    rq = tg.tg_reaction_points(p, dev(x, torch.float64), R).cpu().numpy().reshape(m.n_elems, -1)
    w, xq = O.quadrature(el)
    for q in range(len(w)):
        phi, _ = O.basis(el, xq[q])
        u = sum(phi[b] * x[m.cells[:, b]] for b in range(m.cells.shape[1]))
        want = R[0] + R[1] * u + R[2] * u ** 2 + R[3] * u ** 3
        assert np.allclose(rq[:, q], want, rtol=1e-13, atol=1e-14)


def test_semilinear_without_row_blocks_equals_blocks(tg):
    m = jittered_tri(300)
    g = np.random.default_rng(101)
    relabel = g.permutation(m.n_nodes)
    cells = relabel[m.cells]
    X = np.empty_like(m.coords)
    X[relabel] = m.coords
    x = g.uniform(-1, 1, m.n_nodes)
    xr_ = np.empty_like(x)
    xr_[relabel] = x
    k = g.uniform(0.5, 2, m.n_elems * 3)
    p = tg.tg_build_pattern(dev(cells, torch.int32), m.n_nodes, mg.P1_TRI)
    q = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TRI)
    assert p.n_blocks == 0 and q.n_blocks > 0
    for dt in DTYPES:
        y, _ = tg.tg_semilinear_residual(p, dev(X, dt), dev(k, dt), mg.PER_QP, 0.5, dev(xr_, dt), R, loss=False)
        yb, _ = tg.tg_semilinear_residual(q, dev(m.coords, dt), dev(k, dt), mg.PER_QP, 0.5, dev(x, dt), R,
                                          loss=False)
        assert torch.equal(y[torch.as_tensor(relabel, device="cuda")], yb)


def test_semilinear_reverse_mode(tg):
    from paper_2602_05052_gb300 import autograd as A
    m = jittered_tri(6)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TRI)
    g = np.random.default_rng(102)
    mask = dev(m.boundary.astype(np.uint8), torch.uint8)
    coords = dev(m.coords, torch.float64)
    k = dev(g.uniform(0.5, 2, m.n_elems * 3), torch.float64).requires_grad_(True)
    x = dev(g.uniform(-1, 1, m.n_nodes), torch.float64).requires_grad_(True)
    f = dev(g.uniform(-1, 1, m.n_nodes), torch.float64).requires_grad_(True)
    fn = lambda k_, x_, f_: A.residual(p, coords, k_, mg.PER_QP, 0.3, x_, f_, mg.PER_NODE, mask, reaction=R)
    assert torch.autograd.gradcheck(fn, (k, x, f), eps=1e-6, atol=1e-8)
    # coordinates too (the reaction's |det J| term through the per-point load backward)
    c2 = coords.clone().requires_grad_(True)
    fc = lambda c_: A.residual(p, c_, k.detach(), mg.PER_QP, 0.3, x.detach(), f.detach(), mg.PER_NODE, mask,
                               reaction=R)
    assert torch.autograd.gradcheck(fc, (c2,), eps=1e-6, atol=1e-8)


def test_allen_cahn_step_residual(tg):
    """Backward Euler for du/dt = div(a^2 grad u) - eps^2 (u^3 - u): one call
    against the step's terms from the oracle."""
    cfg = mg.diffusion2d(256)
    m = cfg["mesh"]
    g = np.random.default_rng(103)
    U0, U1 = g.uniform(-1, 1, m.n_nodes), g.uniform(-1, 1, m.n_nodes)
    a2, dt, e2 = 0.01, 1e-3, 0.3
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TRI)
    X = dev(m.coords, torch.float64)
    r = [0.0, -e2, 0.0, e2]
    y, _ = tg.tg_semilinear_residual(p, X, dev([a2], torch.float64), mg.CONSTANT, 1.0 / dt, dev(U1, torch.float64), r,
                                     dev(U0 / dt, torch.float64), mg.PER_NODE,
                                     dirichlet=dev(m.boundary.astype(np.uint8), torch.uint8))
    M = O.assemble_bilinear(mg.P1_TRI, m.cells, m.coords, np.zeros(1), O.CONSTANT, 1.0).to_scipy()
    K = O.assemble_bilinear(mg.P1_TRI, m.cells, m.coords, np.array([1.0]), O.CONSTANT, 0.0).to_scipy()
    want = (M @ (U1 - U0)) / dt + a2 * (K @ U1) + O.reaction_load(mg.P1_TRI, m.cells, m.coords, U1, r)
    want[m.boundary] = 0.0
    assert relfro(y.cpu().numpy(), want) <= 1e-12
