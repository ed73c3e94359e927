"""The chunked multi-process oracle (used to time the oracle on all host
cores) gives the single-process oracle's results up to the summation order
of the chunks."""
from __future__ import annotations

import numpy as np

import meshgen as mg
import oracle as O
from oracle.chunked import ChunkedOracle


def test_chunked_oracle_equals_one_process():
    cfg = mg.diffusion2d(24)
    m = cfg["mesh"]
    K = O.assemble_bilinear(O.P1_TRI, m.cells, m.coords, cfg["kappa"], O.PER_QP, cfg["c"])
    F = O.assemble_load(O.P1_TRI, m.cells, m.coords, cfg["f"], O.PER_NODE)
    G = np.random.default_rng(3).normal(size=K.nnz)
    gk, gx, gc = O.assemble_backward(O.P1_TRI, m.cells, m.coords, cfg["kappa"], O.PER_QP, cfg["c"],
                                     grad_csr=O.CSR(K.row_ptr, K.col, G))
    for threads in (1, 3):
        ch = ChunkedOracle(m.cells, m.coords, cfg["kappa"], cfg["f"], cfg["c"], threads, seed=3)
        try:
            v, F2, gk2, gx2, gc2 = ch.step()
        finally:
            ch.close()
        assert np.allclose(v, K.val, rtol=1e-13, atol=1e-13 * np.abs(K.val).max())
        assert np.allclose(F2, F, rtol=1e-13, atol=1e-15)
        assert np.allclose(gk2, gk.ravel(), rtol=1e-13, atol=1e-15)
        assert np.allclose(gx2, gx, rtol=1e-12, atol=1e-12 * np.abs(gx).max())
        assert abs(gc2 - gc) <= 1e-12 * abs(gc)
