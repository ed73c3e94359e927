"""GPU parity of the plane-stress QUAD4 / SIMP assembly and the compliance
sensitivity against the FP64 oracle."""
from __future__ import annotations

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla
import torch

import meshgen as mg
from gpu_helpers import TOL, dev, host_as, relfro
from oracle import quad as Q

pytestmark = pytest.mark.gpu

DTYPES = [torch.float64, torch.float32]
LAW = dict(e_min=70.0, e_max=70000.0, penal=3.0, nu=0.3)


@pytest.fixture(scope="module")
def tg():
    import paper_2602_05052_gb300 as tg
    return tg


def _distorted(nx, ny, seed=2):
    m = mg.quad_grid(nx, ny, 2.0, 1.0)
    g = np.random.default_rng(seed)
    disp = g.uniform(-0.2 * m.h, 0.2 * m.h, size=m.coords.shape)
    disp[m.boundary] = 0
    m.coords = m.coords + disp
    return m


def test_dof_pattern_bit_exact(tg):
    m = _distorted(7, 5)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.Q1_QUAD_VEC2)
    ref = Q.assemble_simp(m.cells, m.coords, np.ones(m.n_elems), 0.0, 1.0, 3.0, 0.3)
    assert p.n_rows == 2 * m.n_nodes and p.nnz == ref.nnz
    assert np.array_equal(p.row_ptr.cpu().numpy().astype(np.int64), ref.row_ptr)
    assert np.array_equal(p.col_idx.cpu().numpy(), ref.col)


@pytest.mark.parametrize("dtype", DTYPES)
def test_simp_assembly_and_sensitivity_match_oracle(tg, dtype):
    m = _distorted(9, 6)
    g = np.random.default_rng(4)
    rho = g.uniform(0.1, 1.0, m.n_elems)
    u = g.uniform(-1, 1, 2 * m.n_nodes)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.Q1_QUAD_VEC2)
    X, r = dev(m.coords, dtype), dev(rho, dtype)
    vals = tg.tg_assemble_simp(p, X, r, **LAW)
    ref = Q.assemble_simp(m.cells, host_as(m.coords, dtype), host_as(rho, dtype), LAW["e_min"], LAW["e_max"],
                          LAW["penal"], LAW["nu"])
    assert relfro(vals.cpu().numpy(), ref.val) <= TOL[dtype]
    dc = tg.tg_simp_sensitivity(p, X, r, **LAW, u=dev(u, dtype))
    want = Q.simp_sensitivity(m.cells, host_as(m.coords, dtype), host_as(rho, dtype), LAW["e_min"], LAW["e_max"],
                              LAW["penal"], LAW["nu"], host_as(u, dtype))
    assert relfro(dc.cpu().numpy(), want) <= TOL[dtype]
    again = tg.tg_assemble_simp(p, X, r, **LAW)
    assert torch.equal(vals, again)
    assert tg.tg_get_device_status(p) == (0, -1)


def test_cantilever_compliance_and_sensitivity(tg):
    """The SM's 60 x 30 cantilever at uniform density 0.5 in FP64: GPU
    assembly, masked CG and sensitivity against the oracle with a direct
    solve."""
    cfg = mg.cantilever()
    m = cfg["mesh"]
    law = {k: cfg[k] for k in ("E_min", "E_max", "penal", "nu")}
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.Q1_QUAD_VEC2)
    X, rho = dev(m.coords, torch.float64), dev(cfg["rho"], torch.float64)
    vals = tg.tg_assemble_simp(p, X, rho, law["E_min"], law["E_max"], law["penal"], law["nu"])
    F = dev(cfg["F"], torch.float64)
    mask = dev(cfg["dirichlet"].astype(np.uint8), torch.uint8)
    u, it, rel = tg.tg_cg_solve(p, vals, F, mask, rtol=1e-13, maxit=200000)
    assert rel <= 1e-13
    K = Q.assemble_simp(m.cells, m.coords, cfg["rho"], law["E_min"], law["E_max"], law["penal"], law["nu"]).to_scipy()
    free = ~cfg["dirichlet"]
    uo = np.zeros(2 * m.n_nodes)
    uo[free] = spla.spsolve(sp.csc_matrix(K[free][:, free]), cfg["F"][free])
    assert relfro(u.cpu().numpy(), uo) <= 1e-10
    C, Co = float(F @ u), float(cfg["F"] @ uo)
    assert abs(C - Co) <= 1e-10 * abs(Co)
    dc = tg.tg_simp_sensitivity(p, X, rho, law["E_min"], law["E_max"], law["penal"], law["nu"], u)
    want = Q.simp_sensitivity(m.cells, m.coords, cfg["rho"], law["E_min"], law["E_max"], law["penal"], law["nu"], uo)
    assert relfro(dc.cpu().numpy(), want) <= 1e-9


def test_kind_checks(tg):
    m = _distorted(3, 3)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.Q1_QUAD_VEC2)
    X = dev(m.coords, torch.float64)
    with pytest.raises(tg.TGError):
        tg.tg_assemble_bilinear(p, X, dev([1.0], torch.float64), mg.CONSTANT, 0.0)
    t = mg.tri_grid(3)
    pt = tg.tg_build_pattern(dev(t.cells, torch.int32), t.n_nodes, mg.P1_TRI)
    with pytest.raises(tg.TGError):
        tg.tg_assemble_simp(pt, dev(t.coords, torch.float64), dev(np.ones(t.n_elems), torch.float64), **LAW)
