"""GPU parity of the reverse-mode assembly against the oracle's analytic
gradients and against finite differences (differentiable 3D Poisson)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import meshgen as mg
import oracle as O
from gpu_helpers import TOL, coef, dev, host_as, jittered_tet, mesh_for, relfro

pytestmark = pytest.mark.gpu

ELS = [mg.P1_TRI, mg.P2_TRI, mg.P1_TET]
DTYPES = [torch.float64, torch.float32]
# the gradients meet the same relative Frobenius bounds as the assembled
# values: 1e-12 in FP64, 2e-6 in FP32 against the FP64 oracle fed the
# FP32-rounded inputs (measured on GB300: at most about 6e-7)
GTOL = TOL


@pytest.fixture(scope="module")
def tg():
    import paper_2602_05052_gb300 as tg
    return tg


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("layout", [mg.PER_QP, mg.PER_ELEMENT, mg.CONSTANT])
@pytest.mark.parametrize("el", ELS)
def test_backward_matches_oracle(tg, el, layout, dtype, fused):
    m = mesh_for(el)
    k = coef(layout, m.n_elems, mg.NQ[el], seed=50 + el)
    c = 0.6
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, el)
    g = np.random.default_rng(51)
    xs, ks = host_as(m.coords, dtype), host_as(k, dtype)
    if fused:
        lam, U = host_as(g.normal(size=m.n_nodes), dtype), host_as(g.normal(size=m.n_nodes), dtype)
        gk, gx, gc = tg.tg_assemble_backward(p, dev(m.coords, dtype), dev(k, dtype), layout, c, lam=dev(lam, dtype),
                                             U=dev(U, dtype))
        rk, rx, rc = O.assemble_backward(el, m.cells, xs, ks, layout, c, lam=lam, U=U)
    else:
        ref = O.assemble_bilinear(el, m.cells, xs, ks, layout, c)
        gv = host_as(g.normal(size=p.nnz), dtype)
        gk, gx, gc = tg.tg_assemble_backward(p, dev(m.coords, dtype), dev(k, dtype), layout, c, grad_vals=dev(gv, dtype))
        rk, rx, rc = O.assemble_backward(el, m.cells, xs, ks, layout, c, grad_csr=O.CSR(ref.row_ptr, ref.col, gv))
    assert relfro(gk.cpu().numpy(), rk) <= GTOL[dtype]
    assert relfro(gx.cpu().numpy(), rx) <= GTOL[dtype]
    assert relfro(gc.cpu().numpy(), [rc]) <= GTOL[dtype]
    assert tg.tg_get_device_status(p) == (0, -1)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("layout", [mg.PER_NODE, mg.PER_QP, mg.CONSTANT])
@pytest.mark.parametrize("el", ELS + [mg.P1_TET_VEC3])
def test_load_backward_matches_oracle(tg, el, layout, dtype):
    m = mesh_for(el)
    ncomp = 3 if el == mg.P1_TET_VEC3 else 1
    g = np.random.default_rng(60 + el)
    nf = {mg.PER_NODE: m.n_nodes, mg.PER_QP: m.n_elems * mg.NQ[el], mg.CONSTANT: 1}[layout] * ncomp
    f = host_as(g.uniform(-1, 1, size=nf), dtype)
    gF = host_as(g.normal(size=m.n_nodes * ncomp), dtype)
    xs = host_as(m.coords, dtype)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, el)
    gf, gx = tg.tg_assemble_load_backward(p, dev(m.coords, dtype), dev(f, dtype), layout, ncomp, dev(gF, dtype))
    rf, rx = O.load_backward(el, m.cells, xs, f, layout, ncomp, gF)
    assert relfro(gf.cpu().numpy(), rf) <= GTOL[dtype]
    assert relfro(gx.cpu().numpy(), rx) <= GTOL[dtype]
    # accumulate adds to what is there
    gf2, gx2 = gf.clone(), gx.clone()
    tg.tg_assemble_load_backward(p, dev(m.coords, dtype), dev(f, dtype), layout, ncomp, dev(gF, dtype), grad_f=gf2,
                                 grad_coords=gx2, accumulate=True)
    assert torch.allclose(gf2, 2 * gf) and torch.allclose(gx2, 2 * gx)


@pytest.mark.parametrize("dtype", DTYPES)
def test_backward_is_bitwise_deterministic(tg, dtype):
    m = mesh_for(mg.P1_TRI, "large")
    k = coef(mg.PER_QP, m.n_elems, 3, seed=5)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TRI)
    gv = dev(np.random.default_rng(2).normal(size=p.nnz), dtype)
    x, kk = dev(m.coords, dtype), dev(k, dtype)
    first = [t.clone() for t in tg.tg_assemble_backward(p, x, kk, mg.PER_QP, 1.0, grad_vals=gv)]
    for _ in range(9):
        again = tg.tg_assemble_backward(p, x, kk, mg.PER_QP, 1.0, grad_vals=gv)
        for a, b in zip(first, again):
            assert torch.equal(a, b)


def test_autograd_gradcheck(tg):
    from paper_2602_05052_gb300 import autograd as A
    m = mg.jitter(mg.tri_grid(3), 4)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TRI)
    x = dev(m.coords, torch.float64).requires_grad_(True)
    k = dev(np.random.default_rng(1).uniform(0.5, 2, size=m.n_elems * 3), torch.float64).requires_grad_(True)
    f = dev(np.random.default_rng(2).uniform(-1, 1, size=m.n_nodes), torch.float64).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda x_, k_: A.assemble(p, x_, k_, mg.PER_QP, 0.3), (x, k), eps=1e-6, atol=1e-8)
    assert torch.autograd.gradcheck(lambda x_, f_: A.load(p, x_, f_, mg.PER_NODE), (x, f), eps=1e-6, atol=1e-8)
    mask = dev(m.boundary.astype(np.uint8), torch.uint8)
    vals = A.assemble(p, x, k, mg.PER_QP, 0.0).detach().requires_grad_(True)
    F = A.load(p, x, f, mg.PER_NODE).detach().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda v_, F_: A.solve(p, v_, F_, mask, rtol=1e-14), (vals, F), eps=1e-6,
                                    atol=1e-7)


def _poisson3d_loss(tg, A, p, coords, kappa, f, mask, u_t, rtol=1e-13):
    u = A.solve_assembled(p, coords, kappa, mg.PER_ELEMENT, f, mg.CONSTANT, mask, rtol=rtol)
    return ((u - u_t) ** 2).sum()


def test_differentiable3d_full_size_finite_differences(tg):
    """48^3 Kuhn mesh: dL/dkappa and dL/dcoords of L = ||u - u_target||^2
    (forward assembly + CG, adjoint CG + backward assembly) against central
    differences along 16 random directions each."""
    from paper_2602_05052_gb300 import autograd as A
    cfg = mg.differentiable3d(48)
    m = cfg["mesh"]
    assert m.n_elems == 663552
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TET)
    mask = dev(m.boundary.astype(np.uint8), torch.uint8)
    x0 = dev(m.coords, torch.float64)
    f = dev([1.0], torch.float64)
    with torch.no_grad():
        u_t = A.solve_assembled(p, x0, dev(cfg["kappa_star"], torch.float64), mg.PER_ELEMENT, f, mg.CONSTANT, mask,
                                rtol=1e-13)
    k0 = dev(cfg["kappa"], torch.float64)
    k = k0.clone().requires_grad_(True)
    x = x0.clone().requires_grad_(True)
    L = _poisson3d_loss(tg, A, p, x, k, f, mask, u_t)
    L.backward()
    gk, gx = k.grad.clone(), x.grad.clone()
    dk = mg.fd_directions(16, m.n_elems, seed=55)
    dxs = mg.fd_directions(16, m.n_nodes * 3, seed=56).reshape(16, m.n_nodes, 3)
    dxs[:, m.boundary, :] = 0  # keep the domain fixed
    with torch.no_grad():
        for i in range(16):
            d = dev(dk[i], torch.float64)
            eps = 1e-2
            num = (_poisson3d_loss(tg, A, p, x0, k0 + eps * d, f, mask, u_t)
                   - _poisson3d_loss(tg, A, p, x0, k0 - eps * d, f, mask, u_t)).item() / (2 * eps)
            ana = float((gk * d).sum())
            assert abs(num - ana) <= 1e-6 * max(abs(ana), 1e-12 * float(L)), (i, num, ana)
            dx = dev(dxs[i], torch.float64)
            eps = 1e-3
            num = (_poisson3d_loss(tg, A, p, x0 + eps * dx, k0, f, mask, u_t)
                   - _poisson3d_loss(tg, A, p, x0 - eps * dx, k0, f, mask, u_t)).item() / (2 * eps)
            ana = float((gx * dx).sum())
            assert abs(num - ana) <= 1e-6 * max(abs(ana), 1e-12 * float(L)), (i, num, ana)


def test_differentiable3d_small_matches_oracle_gradient(tg):
    """Same pipeline on 12^3 against the oracle: assembly, CG, adjoint CG,
    analytic backward, all on the CPU."""
    from oracle import solve as S
    from paper_2602_05052_gb300 import autograd as A
    cfg = mg.differentiable3d(12)
    m = cfg["mesh"]
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TET)
    mask = dev(m.boundary.astype(np.uint8), torch.uint8)
    f1 = np.array([1.0])
    # oracle pipeline
    Ks = O.assemble_bilinear(O.P1_TET, m.cells, m.coords, cfg["kappa_star"], O.PER_ELEMENT, 0.0).to_scipy()
    F = O.assemble_load(O.P1_TET, m.cells, m.coords, f1, O.CONSTANT)
    ut, _, _ = S.solve_dirichlet(Ks, F, m.boundary, tol=1e-14)
    Kc = O.assemble_bilinear(O.P1_TET, m.cells, m.coords, cfg["kappa"], O.PER_ELEMENT, 0.0)
    u, _, _ = S.solve_dirichlet(Kc.to_scipy(), F, m.boundary, tol=1e-14)
    lam, _, _ = S.solve_dirichlet(Kc.to_scipy(), 2 * (u - ut), m.boundary, tol=1e-14)
    rk, rx, _ = O.assemble_backward(O.P1_TET, m.cells, m.coords, cfg["kappa"], O.PER_ELEMENT, 0.0, lam=-lam, U=u)
    _, rx2 = O.load_backward(O.P1_TET, m.cells, m.coords, f1, O.CONSTANT, 1, lam)
    # GPU pipeline
    k = dev(cfg["kappa"], torch.float64).requires_grad_(True)
    x = dev(m.coords, torch.float64).requires_grad_(True)
    u_t = dev(ut, torch.float64)
    L = _poisson3d_loss(tg, A, p, x, k, dev(f1, torch.float64), mask, u_t, rtol=1e-14)
    L.backward()
    assert relfro(k.grad.cpu().numpy(), rk) <= 1e-9
    assert relfro(x.grad.cpu().numpy(), rx + rx2) <= 1e-9


# ---------------------------------------------------------------- vector P1 elasticity
@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("layout", [mg.PER_ELEMENT, mg.PER_QP])
def test_elasticity_backward_matches_oracle(tg, layout, dtype, fused):
    m = jittered_tet(6)  # 343 nodes, 1,296 tetrahedra
    lam = coef(layout, m.n_elems, 4, seed=71, lo=0.5, hi=2.0)
    mu = coef(layout, m.n_elems, 4, seed=72, lo=0.3, hi=1.0)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TET_VEC3)
    xs, ls, ms = host_as(m.coords, dtype), host_as(lam, dtype), host_as(mu, dtype)
    g = np.random.default_rng(73)
    args = (p, dev(m.coords, dtype), dev(lam, dtype), dev(mu, dtype), layout)
    if fused:
        la = host_as(g.normal(size=3 * m.n_nodes), dtype)
        U = host_as(g.normal(size=3 * m.n_nodes), dtype)
        kw = dict(lam_adj=dev(la, dtype), U=dev(U, dtype))
        want = O.elasticity_backward(m.cells, xs, ls, ms, layout, lam_adj=la, U=U)
    else:
        ref = O.assemble_elasticity(m.cells, xs, ls, ms, layout)
        gv = host_as(g.normal(size=ref.nnz), dtype)
        kw = dict(grad_vals=dev(gv, dtype))
        want = O.elasticity_backward(m.cells, xs, ls, ms, layout, grad_csr=O.CSR(ref.row_ptr, ref.col, gv))
    got = tg.tg_assemble_elasticity_backward(*args, **kw)
    for a, b in zip(got, want):
        assert relfro(a.cpu().numpy().reshape(-1), np.asarray(b).reshape(-1)) <= GTOL[dtype]
    again = tg.tg_assemble_elasticity_backward(*args, **kw)
    assert all(torch.equal(a, b) for a, b in zip(got, again))
    assert tg.tg_get_device_status(p) == (0, -1)


def _fan_tets(m=20, seed=75):
    """2m tetrahedra around the z axis: a centre node, an apex above and one
    below, a ring of m nodes; the centre node has m + 2 neighbours, so its
    row is longer than 16 and the pattern gets no row blocks."""
    g = np.random.default_rng(seed)
    ang = 2 * np.pi * np.arange(m) / m
    ring = np.stack([np.cos(ang), np.sin(ang), g.uniform(-0.1, 0.1, m)], 1)
    coords = np.vstack([[0.0, 0.0, 0.0], [0.0, 0.0, 1.0], [0.0, 0.0, -1.0], ring])
    cells = []
    for i in range(m):
        a, b = 3 + i, 3 + (i + 1) % m
        cells += [[0, a, b, 1], [0, b, a, 2]]
    return np.asarray(cells, dtype=np.int32), coords


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("dtype", DTYPES)
def test_elasticity_backward_without_row_blocks(tg, dtype, fused):
    """The two-pass elasticity backward (every pattern without row blocks)."""
    cells, coords = _fan_tets()
    n, E = coords.shape[0], cells.shape[0]
    g = np.random.default_rng(76)
    lam, mu = g.uniform(0.5, 2.0, E), g.uniform(0.3, 1.0, E)
    p = tg.tg_build_pattern(dev(cells, torch.int32), n, mg.P1_TET_VEC3)
    assert p.n_blocks == 0
    xs, ls, ms = host_as(coords, dtype), host_as(lam, dtype), host_as(mu, dtype)
    args = (p, dev(coords, dtype), dev(lam, dtype), dev(mu, dtype), mg.PER_ELEMENT)
    if fused:
        la, U = host_as(g.normal(size=3 * n), dtype), host_as(g.normal(size=3 * n), dtype)
        kw = dict(lam_adj=dev(la, dtype), U=dev(U, dtype))
        want = O.elasticity_backward(cells, xs, ls, ms, mg.PER_ELEMENT, lam_adj=la, U=U)
    else:
        ref = O.assemble_elasticity(cells, xs, ls, ms, mg.PER_ELEMENT)
        gv = host_as(g.normal(size=ref.nnz), dtype)
        kw = dict(grad_vals=dev(gv, dtype))
        want = O.elasticity_backward(cells, xs, ls, ms, mg.PER_ELEMENT, grad_csr=O.CSR(ref.row_ptr, ref.col, gv))
    got = tg.tg_assemble_elasticity_backward(*args, **kw)
    for a, b in zip(got, want):
        assert relfro(a.cpu().numpy().reshape(-1), np.asarray(b).reshape(-1)) <= GTOL[dtype]
    again = tg.tg_assemble_elasticity_backward(*args, **kw)
    assert all(torch.equal(a, b) for a, b in zip(got, again))
    assert tg.tg_get_device_status(p) == (0, -1)


def test_elasticity_backward_central_differences(tg):
    """FP64: directional derivatives of L = <W, K(lam, mu, x)> against central
    differences of the GPU forward."""
    m = mesh_for(mg.P1_TET_VEC3)
    g = np.random.default_rng(74)
    lam = g.uniform(0.5, 2.0, m.n_elems)
    mu = g.uniform(0.3, 1.0, m.n_elems)
    dt = torch.float64
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TET_VEC3)
    gv = dev(g.normal(size=p.nnz), dt)
    x, l, u = dev(m.coords, dt), dev(lam, dt), dev(mu, dt)
    gl, gm, gx = tg.tg_assemble_elasticity_backward(p, x, l, u, mg.PER_ELEMENT, grad_vals=gv)

    def L(xx, ll, uu):
        return float(torch.dot(tg.tg_assemble_elasticity(p, xx, ll, uu, mg.PER_ELEMENT), gv))

    for k in range(3):
        dx = dev(g.normal(size=m.coords.shape) * 0.05 * m.h, dt)
        dl = dev(g.normal(size=m.n_elems), dt)
        du = dev(g.normal(size=m.n_elems), dt)
        eps = 1e-4
        fd = (L(x + eps * dx, l + eps * dl, u + eps * du) - L(x - eps * dx, l - eps * dl, u - eps * du)) / (2 * eps)
        an = float((gx * dx).sum() + (gl * dl).sum() + (gm * du).sum())
        assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)), (k, fd, an)


def test_backward_diffusion2d_full_size(tg):
    """The benchmark's backward on the 1024^2 workload in FP32 (the launch
    configuration bench.py times) against the oracle's analytic gradients
    of every element and node."""
    cfg = mg.diffusion2d(1024)
    m = cfg["mesh"]
    dtype = torch.float32
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TRI)
    xs, ks = host_as(m.coords, dtype), host_as(cfg["kappa"], dtype)
    gv = host_as(np.random.default_rng(1).normal(size=p.nnz), dtype)
    gk, gx, gc = tg.tg_assemble_backward(p, dev(m.coords, dtype), dev(cfg["kappa"], dtype), mg.PER_QP, cfg["c"],
                                         grad_vals=dev(gv, dtype))
    ref = O.assemble_bilinear(mg.P1_TRI, m.cells, xs, ks, O.PER_QP, cfg["c"])
    rk, rx, rc = O.assemble_backward(mg.P1_TRI, m.cells, xs, ks, O.PER_QP, cfg["c"],
                                     grad_csr=O.CSR(ref.row_ptr, ref.col, gv))
    assert relfro(gk.cpu().numpy().ravel(), rk) <= GTOL[dtype]
    assert relfro(gx.cpu().numpy(), rx) <= GTOL[dtype]
    assert relfro(gc.cpu().numpy(), [rc]) <= GTOL[dtype]
    assert tg.tg_get_device_status(p) == (0, -1)
