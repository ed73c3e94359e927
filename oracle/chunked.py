"""Chunked multi-process runs of the FP64 oracle (TEST INFRASTRUCTURE ONLY).

Used by the benchmark to time the oracle on all host cores: the elements
are split into T contiguous chunks, each chunk is assembled by its own
process into its own dictionary of keys (the oracle's plain scatter-add,
Eq. (scatter_add)), and the partial results are added in chunk order.  One
pass is what the hot path computes for the 2D diffusion workload: the
stiffness values with kappa at the points and the mass term, the load vector
of a nodal f, and the backward for an upstream gradient of the values.

The workload arrays go to the workers once, as files in a temporary
directory that they map read-only; a pass then ships only chunk bounds out
and each chunk's partial results back.  Processes start with the 'spawn'
method, so a parent that has already used a GPU is safe.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import shutil
import tempfile
from concurrent.futures import ProcessPoolExecutor

import numpy as np

_W: dict = {}


def _init(path):
    """Worker start-up: map the workload and build the oracle library."""
    import oracle as O
    O.lib()
    for k in ("cells", "coords", "kappa", "f", "rp", "col", "G", "keys"):
        _W[k] = np.load(os.path.join(path, k + ".npy"), mmap_mode="r")
    _W["c"] = float(np.load(os.path.join(path, "c.npy")))


def _pass(bounds):
    """One chunk [lo, hi) of elements: forward, load and backward by the
    oracle; the CSR entries come back as slots of the full pattern."""
    import oracle as O
    lo, hi = bounds
    cells = np.ascontiguousarray(_W["cells"][lo:hi])
    coords = _W["coords"]
    kappa = np.ascontiguousarray(_W["kappa"][lo:hi])
    c = _W["c"]
    K = O.assemble_bilinear(O.P1_TRI, cells, coords, kappa, O.PER_QP, c)
    n = coords.shape[0]
    slot = np.searchsorted(_W["keys"], K.rows_of().astype(np.int64) * n + K.col)
    nodes = np.unique(cells)
    F = O.assemble_load(O.P1_TRI, cells, coords, _W["f"], O.PER_NODE)[nodes]
    gk, gx, gc = O.assemble_backward(O.P1_TRI, cells, coords, kappa, O.PER_QP, c,
                                     grad_csr=O.CSR(_W["rp"], _W["col"], _W["G"]))
    return slot, K.val, nodes, F, gk, gx[nodes], gc


class ChunkedOracle:
    """The oracle's pass over a workload with `threads` processes (1 runs it
    in this process)."""

    def __init__(self, cells, coords, kappa, f, c, threads, seed=0, G=None):
        """G: the upstream gradient of the values (one per CSR entry of the
        mesh's pattern), else drawn from N(0, 1) with the seed."""
        import oracle as O
        self.threads = max(1, int(threads))
        self.E, self.N = len(cells), len(coords)
        K = O.assemble_bilinear(O.P1_TRI, cells, coords, kappa, O.PER_QP, c)  # the full pattern
        self.nnz = K.nnz
        G = np.random.default_rng(seed).normal(size=K.nnz) if G is None else np.asarray(G, dtype=np.float64)
        assert G.shape == (K.nnz,)
        self.dir = tempfile.mkdtemp(prefix="tg_oracle_")
        arrays = {"cells": np.ascontiguousarray(cells, dtype=np.int32), "coords": np.ascontiguousarray(coords),
                  "kappa": np.ascontiguousarray(kappa), "f": np.ascontiguousarray(f), "rp": K.row_ptr,
                  "col": K.col, "G": G, "keys": K.rows_of().astype(np.int64) * self.N + K.col,
                  "c": np.array(float(c))}
        for k, a in arrays.items():
            np.save(os.path.join(self.dir, k + ".npy"), a)
        cut = np.linspace(0, self.E, self.threads + 1).astype(np.int64)
        self.chunks = [(int(a), int(b)) for a, b in zip(cut[:-1], cut[1:])]
        if self.threads > 1:
            # a worker that fails to start breaks the pool (an exception here)
            # rather than being replaced forever
            self.pool = ProcessPoolExecutor(self.threads, mp_context=mp.get_context("spawn"), initializer=_init,
                                            initargs=(self.dir,))
            list(self.pool.map(_pass, [(0, 1)] * self.threads))  # every worker loads the library and maps the files
        else:
            self.pool = None
            _init(self.dir)

    def step(self):
        """One pass; returns (vals [nnz], F [N], grad_kappa [E * 3], grad_coords [N, 2], grad_c)."""
        parts = list(self.pool.map(_pass, self.chunks)) if self.pool else [_pass(b) for b in self.chunks]
        vals = np.zeros(self.nnz)
        F = np.zeros(self.N)
        gx = np.zeros((self.N, 2))
        gc = 0.0
        for slot, v, nodes, Fp, _, gxp, gcp in parts:  # chunk order
            vals[slot] += v
            F[nodes] += Fp
            gx[nodes] += gxp
            gc += gcp
        gk = np.concatenate([p[4] for p in parts])
        return vals, F, gk, gx, gc

    def close(self):
        if self.pool is not None:
            self.pool.shutdown()
            self.pool = None
        shutil.rmtree(self.dir, ignore_errors=True)
