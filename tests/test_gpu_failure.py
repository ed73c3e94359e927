"""Failure path of the bounded waits, without a GPU fault: a wait on a
barrier that nothing completes gives up, the status word reports
TG_ERR_TIMEOUT to the host, and the context keeps working."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import meshgen as mg
import oracle as O
from gpu_helpers import dev, jittered_tri, relfro

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_the_context_stays_usable():
    import paper_2602_05052_gb300 as tg
    m = jittered_tri(12)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TRI)
    tg.tg_diag_wait_timeout(p, 1000)
    torch.cuda.synchronize()
    assert tg.tg_get_device_status(p) == (7, 0)  # TG_ERR_TIMEOUT, then cleared
    assert tg.tg_get_device_status(p) == (0, -1)
    # the library keeps working on the same pattern: a backward with its global sum
    k = np.random.default_rng(3).uniform(0.5, 2, m.n_elems * 3)
    gv = np.random.default_rng(4).normal(size=p.nnz)
    X = dev(m.coords, torch.float64)
    gk, gx, gc = tg.tg_assemble_backward(p, X, dev(k, torch.float64), mg.PER_QP, 0.5, grad_vals=dev(gv, torch.float64))
    ref = O.assemble_bilinear(mg.P1_TRI, m.cells, m.coords, k, O.PER_QP, 0.5)
    rk, rx, rc = O.assemble_backward(mg.P1_TRI, m.cells, m.coords, k, O.PER_QP, 0.5,
                                     grad_csr=O.CSR(ref.row_ptr, ref.col, gv))
    assert relfro(gc.cpu().numpy(), [rc]) <= 1e-12 and relfro(gx.cpu().numpy(), rx) <= 1e-12
    assert tg.tg_get_device_status(p) == (0, -1)


def test_grid_barrier_gives_up_and_the_cg_still_runs():
    """The one-launch CG's grid barrier, bounded: with one CTA that never
    arrives the other gives up after its poll limit and the call reports
    TG_ERR_TIMEOUT; afterwards the one-launch CG runs and still equals the
    launch-per-kernel loop bit for bit."""
    import paper_2602_05052_gb300 as tg
    assert tg.tg_diag_grid_barrier_timeout(1000) == 7  # TG_ERR_TIMEOUT
    m = jittered_tri(20)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TRI)
    k = np.random.default_rng(5).uniform(0.5, 2, m.n_elems)
    vals = tg.tg_assemble_bilinear(p, dev(m.coords, torch.float64), dev(k, torch.float64), mg.PER_ELEMENT, 0.2)
    F = dev(np.random.default_rng(6).uniform(-1, 1, m.n_nodes), torch.float64)
    mask = dev(m.boundary.astype(np.uint8), torch.uint8)
    x1, it1, rel1 = tg.tg_cg_solve(p, vals, F, mask, rtol=1e-11)
    x2, it2, rel2 = tg.tg_cg_solve_noalloc(p, vals, F, mask, rtol=1e-11)
    assert rel1 <= 1e-11 and (it1, rel1) == (it2, rel2) and torch.equal(x1, x2)
