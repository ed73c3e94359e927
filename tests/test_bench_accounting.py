"""The benchmark's host-side accounting, on the CPU: the algorithmic bytes
per launch (the roofline numerator) against the counts of the 1024x1024 P1
triangle grid written out from its structure, the two-roof fractions and
the replica throughput."""
from __future__ import annotations

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.fixture(scope="module")
def bench():
    import bench
    return bench


def _grid_counts(n):
    """A structured n x n grid of squares, each cut into two triangles:
    E = 2 n^2 elements, N = (n + 1)^2 nodes and 3 n^2 + 2 n edges, so the
    node-level CSR holds N diagonal entries plus two per edge."""
    E, N = 2 * n * n, (n + 1) ** 2
    edges = n * (n + 1) * 2 + n * n
    return E, N, N + 2 * edges


def test_grid_counts_match_the_mesh_generator():
    import meshgen as mg
    m = mg.tri_grid(16)
    E, N, nnz = _grid_counts(16)
    assert (m.n_elems, m.n_nodes) == (E, N)
    pairs = set()
    for c in m.cells:
        for a in c:
            for b in c:
                pairs.add((int(a), int(b)))
    assert len(pairs) == nnz


def test_algorithmic_bytes_of_the_step_kernels(bench):
    E, N, nnz = _grid_counts(1024)
    assert (E, N, nnz) == (2_097_152, 1_050_625, 7_346_177)
    s = 4  # FP32
    # backward for an upstream gradient of the values: cells (3 int32), coords,
    # kappa at 3 points and the upstream values read; dL/dkappa and dL/dx written
    assert bench.alg_bytes("bwd", E, N, nnz, s) == E * 12 + N * 8 + E * 12 + nnz * 4 + E * 12 + N * 8 == 121_692_180
    # system: cells, coords, kappa and f read once; values and F written once
    assert bench.alg_bytes("system", E, N, nnz, s) == E * 12 + N * 8 + E * 12 + N * 4 + nnz * 4 + N * 4 == 96_526_356
    assert bench.alg_bytes("fwd", E, N, nnz, s) == E * 12 + N * 8 + E * 12 + nnz * 4
    assert bench.alg_bytes("load", E, N, nnz, s) == E * 12 + N * 8 + N * 4 + N * 4
    # FP64 doubles every floating-point term, not the int32 cells
    d = bench.alg_bytes("bwd", E, N, nnz, 8) - bench.alg_bytes("bwd", E, N, nnz, 4)
    assert d == 4 * (N * 2 + E * 3 + nnz + E * 3 + N * 2)
    with pytest.raises(ValueError):
        bench.alg_bytes("no such kernel", E, N, nnz, s)


def test_two_roofs_takes_the_slower_bound(bench):
    # 1 GB at 1000 GB/s takes 1 ms; 1 GFLOP at 0.5 TFLOP/s takes 2 ms; measured 4 ms
    r = bench.two_roofs(4.0, 1e9, 1e9, 1000.0, 0.5e12)
    assert r["bound"] == "alu"
    assert r["hbm_frac"] == pytest.approx(0.25) and r["alu_frac"] == pytest.approx(0.5)
    assert r["frac_min_roof"] == pytest.approx(0.5)
    r = bench.two_roofs(4.0, 3e9, 1e9, 1000.0, 0.5e12)
    assert r["bound"] == "hbm" and r["frac_min_roof"] == pytest.approx(0.75)


def test_replica_throughput_counts_every_rank_over_the_slowest(bench):
    assert bench.replica_throughput(1000, 1, 2.0) == pytest.approx(5e5)
    assert bench.replica_throughput(1000, 4, 2.0) == pytest.approx(2e6)
    assert bench.replica_max(3.5, 1, "cpu") == 3.5
