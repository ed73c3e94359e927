"""tg_cg_solve_noalloc, the allocation-free form of the CG solve, against
tg_cg_solve on the same systems, through the C ABI.

This file is collected last so that it also runs after every other GPU test
has used the device.  It passes alone as well (the first call on the device
sets the scratch up).
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import meshgen as mg
from gpu_helpers import dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tg():
    import paper_2602_05052_gb300 as tg
    return tg


def _system(tg, n, dtype, seed):
    """Jittered P1 triangles with lognormal kappa at the points, c = 0.1,
    Dirichlet boundary, random load."""
    m = mg.jitter(mg.tri_grid(n), seed)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TRI)
    k = mg.lognormal((m.n_elems, 3), seed + 1)
    vals = tg.tg_assemble_bilinear(p, dev(m.coords, dtype), dev(k, dtype), mg.PER_QP, 0.1)
    F = dev(np.random.default_rng(seed + 2).uniform(-1, 1, m.n_nodes), dtype)
    mask = dev(m.boundary.astype(np.uint8), torch.uint8)
    return p, vals, F, mask


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_noalloc_equals_allocating_solve_on_two_calls_in_a_row(tg, dtype):
    p, vals, F, mask = _system(tg, 40, dtype, 11)
    rtol = 1e-10 if dtype == torch.float64 else 1e-5
    x_ref, it_ref, rel_ref = tg.tg_cg_solve(p, vals, F, mask, rtol=rtol)
    assert rel_ref <= rtol
    for _ in range(2):
        x, it, rel = tg.tg_cg_solve_noalloc(p, vals, F, mask, rtol=rtol)
        torch.cuda.synchronize()
        assert it == it_ref and rel == rel_ref
        assert torch.equal(x, x_ref)


def test_noalloc_interleaved_with_another_system(tg):
    """A second, larger system between two solves of the first: nothing of a
    previous call leaks through the shared scratch."""
    a = _system(tg, 24, torch.float64, 21)
    b = _system(tg, 56, torch.float64, 31)
    want_a = tg.tg_cg_solve(*a, rtol=1e-11)
    want_b = tg.tg_cg_solve(*b, rtol=1e-11)
    for sysm, want in ((a, want_a), (b, want_b), (a, want_a)):
        x, it, rel = tg.tg_cg_solve_noalloc(*sysm, rtol=1e-11)
        assert (it, rel) == want[1:]
        assert torch.equal(x, want[0])


def test_noalloc_rejects_a_system_larger_than_its_scratch(tg):
    # 1024^2 grid: 1,050,625 rows; FP64 work vectors need 4 * 8.4 MB > 16 MiB
    m = mg.tri_grid(1024)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TRI)
    vals = torch.zeros(p.nnz, dtype=torch.float64, device="cuda")
    F = torch.ones(m.n_nodes, dtype=torch.float64, device="cuda")
    x = torch.full((m.n_nodes,), 7.0, dtype=torch.float64, device="cuda")
    with pytest.raises(tg.TGError) as ei:
        tg.tg_cg_solve_noalloc(p, vals, F, None, x=x)
    assert "TG_ERR_UNSUPPORTED" in str(ei.value) and "static scratch" in str(ei.value)
    assert torch.all(x == 7.0)  # rejected before any GPU work
    assert 4 * 8 * m.n_nodes + 4096 > tg.binding.TG_CG_NOALLOC_SCRATCH_BYTES
