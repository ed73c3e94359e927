"""Batched persistent assembly (bitwise equal to per-instance launches, and to
the oracle within tolerance), its CUDA-graph capture and autotuner, and the
CG solve of the structured Poisson problem against its closed form."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import meshgen as mg
import oracle as O
from gpu_helpers import TOL, dev, host_as, relfro

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tg():
    import paper_2602_05052_gb300 as tg
    return tg


def _instances(sizes, dtype):
    insts = mg.batched_p2(len(sizes), seed=4, sizes=sizes)
    out = []
    for k in insts:
        m = k["mesh"]
        out.append(dict(mesh=m, x=dev(m.coords, dtype), kappa=dev(k["kappa"], dtype), kappa_np=k["kappa"]))
    return out


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_batch_bitwise_equals_single_launches(tg, dtype):
    sizes = [1, 2, 3, 5, 8, 13, 21, 34, 7, 4, 30, 17]
    insts = _instances(sizes, dtype)
    pats = [tg.tg_build_pattern(dev(i["mesh"].cells, torch.int32), i["mesh"].n_nodes, mg.P2_TRI) for i in insts]
    b = tg.tg_batch_create(pats)
    cs = [0.1 * j for j in range(len(insts))]
    out = [torch.full((p.nnz,), float("nan"), dtype=dtype, device="cuda") for p in pats]
    for sched in [(128, 512, 0), (64, 64, 2), (256, 2048, 0)]:
        tg.tg_batch_set_schedule(b, *sched)
        tg.tg_batch_assemble(b, [i["x"] for i in insts], [i["kappa"] for i in insts], mg.PER_QP, cs, out)
        for j, (i, p) in enumerate(zip(insts, pats)):
            single = tg.tg_assemble_bilinear(p, i["x"], i["kappa"], mg.PER_QP, cs[j])
            assert torch.equal(out[j], single), (sched, j)
    for j in (0, 5, 10):
        m = insts[j]["mesh"]
        ref = O.assemble_bilinear(O.P2_TRI, m.cells, host_as(m.coords, dtype), host_as(insts[j]["kappa_np"], dtype),
                                  O.PER_QP, cs[j])
        assert relfro(out[j].cpu().numpy(), ref.val) <= TOL[dtype]



def test_batched_p2_full_size(tg):
    """The 256-instance batched P2 workload as the benchmark runs it (FP32,
    autotuned schedule, one launch): bitwise equal to 256 single launches,
    and eight instances across the size range within the FP32 tolerance of
    the oracle."""
    insts = mg.batched_p2(256, seed=4)
    pats, xs, ks = [], [], []
    for k in insts:
        m = k["mesh"]
        pats.append(tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P2_TRI))
        xs.append(dev(m.coords, torch.float32))
        ks.append(dev(k["kappa"], torch.float32))
    b = tg.tg_batch_create(pats)
    cs = [0.0] * len(pats)
    out = [torch.full((p.nnz,), float("nan"), dtype=torch.float32, device="cuda") for p in pats]
    tg.tg_batch_autotune(b, xs, ks, mg.PER_QP, cs, out, reps=2)
    tg.tg_batch_assemble(b, xs, ks, mg.PER_QP, cs, out)
    for j, p in enumerate(pats):
        assert torch.equal(out[j], tg.tg_assemble_bilinear(p, xs[j], ks[j], mg.PER_QP, 0.0)), j
    order = np.argsort([k["mesh"].n_elems for k in insts])
    for j in order[:: len(order) // 8][:8]:
        m = insts[j]["mesh"]
        ref = O.assemble_bilinear(O.P2_TRI, m.cells, host_as(m.coords, torch.float32),
                                  host_as(insts[j]["kappa"], torch.float32), O.PER_QP, 0.0)
        assert relfro(out[j].cpu().numpy(), ref.val) <= TOL[torch.float32], j


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("el", [mg.P1_TRI, mg.P1_TET])
def test_batch_p1_bitwise_equals_single_launches(tg, dtype, el):
    """The batch runs each instance's row blocks with the single-instance
    block body, so its results are bitwise equal to single launches."""
    meshes = []
    for k, n in enumerate([3, 17, 40] if el == mg.P1_TRI else [2, 5, 9]):
        m = mg.jitter(mg.tri_grid(n), 50 + k) if el == mg.P1_TRI else mg.kuhn_tet_grid(n)
        meshes.append(m)
    nq = 3 if el == mg.P1_TRI else 4
    pats = [tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, el) for m in meshes]
    xs = [dev(m.coords, dtype) for m in meshes]
    ks = [dev(mg.lognormal((m.n_elems, nq), 60 + k), dtype) for k, m in enumerate(meshes)]
    cs = [0.0, 0.5, 2.0]
    b = tg.tg_batch_create(pats)
    out = [torch.full((p.nnz,), float("nan"), dtype=dtype, device="cuda") for p in pats]
    tg.tg_batch_assemble(b, xs, ks, mg.PER_QP, cs, out)
    for j, p in enumerate(pats):
        single = tg.tg_assemble_bilinear(p, xs[j], ks[j], mg.PER_QP, cs[j])
        assert torch.equal(out[j], single), j

def test_batch_graph_capture_and_autotune(tg):
    dtype = torch.float32
    sizes = mg.batch_sizes(48, seed=9)
    insts = _instances(sizes, dtype)
    pats = [tg.tg_build_pattern(dev(i["mesh"].cells, torch.int32), i["mesh"].n_nodes, mg.P2_TRI) for i in insts]
    b = tg.tg_batch_create(pats)
    xs, ks = [i["x"] for i in insts], [i["kappa"] for i in insts]
    cs = [0.0] * len(insts)
    out = [torch.empty(p.nnz, dtype=dtype, device="cuda") for p in pats]
    ms = tg.tg_batch_autotune(b, xs, ks, mg.PER_QP, cs, out, reps=2)
    assert ms > 0
    t, r, c = b.schedule()
    assert t in (64, 128, 256) and r % t == 0
    want = [torch.empty_like(o) for o in out]
    tg.tg_batch_assemble(b, xs, ks, mg.PER_QP, cs, want)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    for o in out:
        o.fill_(float("nan"))
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        tg.tg_batch_assemble(b, xs, ks, mg.PER_QP, cs, out, stream=s)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    for o, w in zip(out, want):
        assert torch.equal(o, w)


def test_batch_many_instances_spanning_launch_chunks(tg):
    # more instances than one launch's parameter table holds
    dtype = torch.float32
    sizes = [1 + (j % 4) for j in range(300)]
    insts = _instances(sizes, dtype)
    pats = [tg.tg_build_pattern(dev(i["mesh"].cells, torch.int32), i["mesh"].n_nodes, mg.P2_TRI) for i in insts]
    b = tg.tg_batch_create(pats)
    out = [torch.empty(p.nnz, dtype=dtype, device="cuda") for p in pats]
    cs = [1.0] * len(insts)
    tg.tg_batch_assemble(b, [i["x"] for i in insts], [i["kappa"] for i in insts], mg.PER_QP, cs, out)
    for j in (0, 255, 256, 299):
        single = tg.tg_assemble_bilinear(pats[j], insts[j]["x"], insts[j]["kappa"], mg.PER_QP, 1.0)
        assert torch.equal(out[j], single)


def test_cg_poisson_structured_matches_closed_form(tg):
    from test_oracle_pins import _dst_solution
    n = 64
    m = mg.tri_grid(n)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TRI)
    x = dev(m.coords, torch.float64)
    one = dev([1.0], torch.float64)
    vals = tg.tg_assemble_bilinear(p, x, one, mg.CONSTANT, 0.0)
    F = tg.tg_assemble_load(p, x, one, mg.CONSTANT)
    mask = dev(m.boundary.astype(np.uint8), torch.uint8)
    u, it, rel = tg.tg_cg_solve(p, vals, F, mask, rtol=1e-10)
    assert rel <= 1e-10 and 0 < it < 1000
    U = _dst_solution(n)
    ii = np.arange(m.n_nodes) % (n + 1)
    jj = np.arange(m.n_nodes) // (n + 1)
    un = u.cpu().numpy()
    inner = ~m.boundary
    assert np.all(un[m.boundary] == 0)
    assert np.allclose(un[inner], U[jj[inner] - 1, ii[inner] - 1], rtol=1e-8, atol=1e-12)
    # true residual of the condensed system
    r = tg.tg_spmv(p, vals, u).cpu().numpy() - F.cpu().numpy()
    assert np.linalg.norm(r[inner]) / np.linalg.norm(F.cpu().numpy()[inner]) <= 1e-9


def _cg_system(tg, kind, dtype):
    """Seeded SPD systems for the CG equality checks: a jittered 300x300 P1
    triangle grid (90,601 rows, more than the 2*SM*256 rows of one pass of
    the partial-dot grid), a 30^3 P1 tetrahedral grid, a 10^3 P1
    elasticity grid (3 DoFs per node, one clamped face) and a 640x640 P1
    triangle grid (410,881 rows, which tg_cg_solve runs as graph-captured
    launches)."""
    rng = np.random.default_rng(41)
    if kind == "elastic":
        m = mg.kuhn_tet_grid(10)
        p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TET_VEC3)
        lam = dev(rng.uniform(0.5, 2.0, m.n_elems), dtype)
        mu = dev(rng.uniform(0.3, 1.0, m.n_elems), dtype)
        vals = tg.tg_assemble_elasticity(p, dev(m.coords, dtype), lam, mu, mg.PER_ELEMENT)
        clamp = np.repeat(m.coords[:, 0] == 0.0, 3).astype(np.uint8)
        return p, vals, dev(rng.uniform(-1, 1, p.n_rows), dtype), dev(clamp, torch.uint8)
    if kind == "big":  # 410,881 rows: past the one-launch loop's four rows per thread
        m = mg.tri_grid(640)
    else:
        m = mg.jitter(mg.tri_grid(300), 5) if kind == "tri" else mg.kuhn_tet_grid(30)
    el = mg.P1_TET if kind == "tet" else mg.P1_TRI
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, el)
    k = mg.lognormal((m.n_elems,), 42)
    vals = tg.tg_assemble_bilinear(p, dev(m.coords, dtype), dev(k, dtype), mg.PER_ELEMENT, 0.1)
    return p, vals, dev(rng.uniform(-1, 1, m.n_nodes), dtype), dev(m.boundary.astype(np.uint8), torch.uint8)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("kind", ["tri", "tet", "elastic", "big"])
def test_cg_one_launch_equals_launch_per_kernel_loop(tg, kind, dtype):
    """tg_cg_solve runs its iterations in one cooperative launch (on the
    largest system: 8-iteration CUDA graphs); tg_cg_solve_noalloc keeps one
    launch per kernel.  Same iterates bit for bit: at convergence, and when
    maxit (not a multiple of the check period of 8) stops the loop first."""
    p, vals, F, mask = _cg_system(tg, kind, dtype)
    rtol = 1e-9 if dtype == torch.float64 else 1e-4
    full = None
    for maxit in (100000, 37):
        x1, it1, rel1 = tg.tg_cg_solve(p, vals, F, mask, rtol=rtol, maxit=maxit)
        x2, it2, rel2 = tg.tg_cg_solve_noalloc(p, vals, F, mask, rtol=rtol, maxit=maxit)
        assert (it1, rel1) == (it2, rel2)
        assert torch.equal(x1, x2)
        if full is None:
            full = it1
            assert 0 < it1 < maxit and rel1 <= rtol
        else:
            assert it1 == min(37, full)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_cg_initial_guess_and_zero_load(tg, dtype):
    """A nonzero initial guess: both forms give the same iterates bit for bit
    and the true residual of the condensed system meets the tolerance.  A
    zero load: the solution of K_II x_I = 0 is x = 0 whatever the guess, with
    no iteration and relres 0."""
    m = mg.jitter(mg.tri_grid(40), 7)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TRI)
    k = np.random.default_rng(8).uniform(0.5, 2.0, m.n_elems)
    vals = tg.tg_assemble_bilinear(p, dev(m.coords, dtype), dev(k, dtype), mg.PER_ELEMENT, 0.1)
    F = dev(np.random.default_rng(9).uniform(-1, 1, m.n_nodes), dtype)
    mask = dev(m.boundary.astype(np.uint8), torch.uint8)
    x0 = dev(np.random.default_rng(10).normal(size=m.n_nodes), dtype)
    rtol = 1e-10 if dtype == torch.float64 else 1e-4
    x1, it1, rel1 = tg.tg_cg_solve(p, vals, F, mask, x=x0.clone(), rtol=rtol)
    x2, it2, rel2 = tg.tg_cg_solve_noalloc(p, vals, F, mask, x=x0.clone(), rtol=rtol)
    assert (it1, rel1) == (it2, rel2) and torch.equal(x1, x2)
    assert 0 < it1 and rel1 <= rtol
    xs = x1.double().cpu().numpy()
    inner = ~m.boundary
    assert np.all(xs[m.boundary] == 0)
    r = tg.tg_spmv(p, vals.double(), x1.double()).cpu().numpy() - F.double().cpu().numpy()
    assert np.linalg.norm(r[inner]) / np.linalg.norm(F.double().cpu().numpy()[inner]) <= 100 * rtol
    zero = torch.zeros_like(F)
    for solve in (tg.tg_cg_solve, tg.tg_cg_solve_noalloc):
        x, it, rel = solve(p, vals, zero, mask, x=x0.clone(), rtol=rtol)
        assert it == 0 and rel == 0.0
        assert torch.count_nonzero(x).item() == 0


def test_spmv_and_outer_match_scipy(tg):
    m = mg.jitter(mg.tri_grid(30), 3)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TRI)
    k = np.random.default_rng(3).uniform(0.5, 2, size=m.n_elems * 3)
    vals = tg.tg_assemble_bilinear(p, dev(m.coords, torch.float64), dev(k, torch.float64), mg.PER_QP, 0.2)
    ref = O.assemble_bilinear(O.P1_TRI, m.cells, m.coords, k, O.PER_QP, 0.2)
    xv = np.random.default_rng(4).normal(size=m.n_nodes)
    y = tg.tg_spmv(p, vals, dev(xv, torch.float64)).cpu().numpy()
    assert relfro(y, ref.to_scipy() @ xv) <= 1e-13
    lam = np.random.default_rng(5).normal(size=m.n_nodes)
    o = tg.tg_csr_outer(p, dev(lam, torch.float64), dev(xv, torch.float64), alpha=-2.0).cpu().numpy()
    assert np.array_equal(o, -2.0 * lam[ref.rows_of()] * xv[ref.col])


def test_manufactured_solution_converges_on_the_gpu(tg):
    """u = sin(pi x) sin(pi y), -Laplace u = 2 pi^2 u, u = 0 on the boundary:
    GPU system assembly (f at the quadrature points) and GPU CG; the L2 error
    (degree-4 rule, on the host) falls at second order, as the oracle's
    pinned pipeline does."""
    import math
    w6, x6 = O.quadrature(O.P2_TRI)
    w3, x3 = O.quadrature(O.P1_TRI)
    errs = []
    for n in (16, 32, 64, 128):
        m = mg.jitter(mg.tri_grid(n), 9)
        Xc = m.coords[m.cells]
        J = np.stack([Xc[:, 1] - Xc[:, 0], Xc[:, 2] - Xc[:, 0]], -1)
        xq = Xc[:, None, 0, :] + np.einsum("erc,qc->eqr", J, x3)
        fq = 2 * np.pi ** 2 * np.sin(np.pi * xq[..., 0]) * np.sin(np.pi * xq[..., 1])
        p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TRI)
        vals, F = tg.tg_assemble_system(p, dev(m.coords, torch.float64), dev([1.0], torch.float64), mg.CONSTANT, 0.0,
                                        dev(fq.ravel(), torch.float64), mg.PER_QP)
        u, it, rel = tg.tg_cg_solve(p, vals, F, dev(m.boundary.astype(np.uint8), torch.uint8), rtol=1e-12)
        u = u.cpu().numpy()
        phi = np.array([O.basis(O.P1_TRI, x)[0] for x in x6])
        uh = np.einsum("qa,ea->eq", phi, u[m.cells])
        x6p = Xc[:, None, 0, :] + np.einsum("erc,qc->eqr", J, x6)
        ue = np.sin(np.pi * x6p[..., 0]) * np.sin(np.pi * x6p[..., 1])
        det = np.abs(np.linalg.det(J))
        errs.append(math.sqrt(float(np.sum(det[:, None] * w6[None, :] * (uh - ue) ** 2))))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert min(rates) >= 1.85, (errs, rates)
