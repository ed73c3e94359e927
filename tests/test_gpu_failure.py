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
