"""GPU parity of the pattern and the forward assembly against the FP64 oracle."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import meshgen as mg
import oracle as O
from gpu_helpers import TOL, coef, dev, host_as, jittered_tet, jittered_tri, mesh_for, relfro

pytestmark = pytest.mark.gpu

ELS = [mg.P1_TRI, mg.P2_TRI, mg.P1_TET]
DTYPES = [torch.float64, torch.float32]


@pytest.fixture(scope="module")
def tg():
    import paper_2602_05052_gb300 as tg
    return tg


# ---------------------------------------------------------------- pattern
@pytest.mark.parametrize("el", ELS + [mg.P1_TET_VEC3])
def test_pattern_bit_exact(tg, el):
    m = mesh_for(el)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, el)
    if el == mg.P1_TET_VEC3:
        ref = O.assemble_elasticity(m.cells, m.coords, np.ones(m.n_elems), np.ones(m.n_elems), O.PER_ELEMENT)
    else:
        ref = O.assemble_bilinear(el, m.cells, m.coords, np.ones(1), O.CONSTANT, 1.0)
    assert p.nnz == ref.nnz
    assert np.array_equal(p.row_ptr.cpu().numpy().astype(np.int64), ref.row_ptr)
    assert np.array_equal(p.col_idx.cpu().numpy(), ref.col)
    # element-to-slot map: slot (e, a, b) lies in row g_a at column g_b
    es = p.elem_slot.cpu().numpy().reshape(m.n_elems, m.cells.shape[1], m.cells.shape[1]).astype(np.int64)
    rows = ref.rows_of()
    if el == mg.P1_TET_VEC3:
        assert np.array_equal(rows[es] // 3, np.repeat(m.cells[:, :, None], 4, axis=2))
        assert np.array_equal(ref.col[es] // 3, np.repeat(m.cells[:, None, :], 4, axis=1))
        assert np.all(rows[es] % 3 == 0) and np.all(ref.col[es] % 3 == 0)
    else:
        nv = m.cells.shape[1]
        assert np.array_equal(rows[es], np.repeat(m.cells[:, :, None], nv, axis=2))
        assert np.array_equal(ref.col[es], np.repeat(m.cells[:, None, :], nv, axis=1))


# ---------------------------------------------------------------- bilinear forms
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("layout", [mg.PER_QP, mg.PER_ELEMENT, mg.CONSTANT])
@pytest.mark.parametrize("el", ELS)
def test_bilinear_matches_oracle(tg, el, layout, dtype):
    m = mesh_for(el)
    nq = mg.NQ[el]
    k = coef(layout, m.n_elems, nq, seed=10 + el)
    c = 0.75
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, el)
    vals = tg.tg_assemble_bilinear(p, dev(m.coords, dtype), dev(k, dtype), layout, c)
    ref = O.assemble_bilinear(el, m.cells, host_as(m.coords, dtype), host_as(k, dtype), layout, c)
    err = relfro(vals.cpu().numpy(), ref.val)
    assert err <= TOL[dtype], err
    assert tg.tg_get_device_status(p) == (0, -1)


def test_structured_poisson_bit_exact(tg):
    m = mg.tri_grid(64)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TRI)
    vals = tg.tg_assemble_bilinear(p, dev(m.coords, torch.float64), dev(np.ones(1), torch.float64), mg.CONSTANT, 0.0)
    ref = O.assemble_bilinear(mg.P1_TRI, m.cells, m.coords, np.ones(1), O.CONSTANT, 0.0)
    assert p.nnz == 29057
    assert np.array_equal(vals.cpu().numpy(), ref.val)
    F = tg.tg_assemble_load(p, dev(m.coords, torch.float64), dev(np.ones(1), torch.float64), mg.CONSTANT)
    Fr = O.assemble_load(mg.P1_TRI, m.cells, m.coords, np.ones(1), O.CONSTANT)
    assert relfro(F.cpu().numpy(), Fr) <= 1e-15


@pytest.mark.parametrize("dtype", DTYPES)
def test_forward_is_bitwise_deterministic(tg, dtype):
    m = jittered_tri(128)
    k = mg.lognormal(m.n_elems * 3, 7)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TRI)
    x, kk = dev(m.coords, dtype), dev(k, dtype)
    first = tg.tg_assemble_bilinear(p, x, kk, mg.PER_QP, 1.0).clone()
    for _ in range(9):
        again = tg.tg_assemble_bilinear(p, x, kk, mg.PER_QP, 1.0)
        assert torch.equal(first, again)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("el", ELS)
def test_atomic_variant_within_tolerance(tg, el, dtype):
    m = mesh_for(el)
    k = coef(mg.PER_QP, m.n_elems, mg.NQ[el], seed=3)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, el)
    a = tg.tg_assemble_bilinear_atomic(p, dev(m.coords, dtype), dev(k, dtype), mg.PER_QP, 0.5)
    ref = O.assemble_bilinear(el, m.cells, host_as(m.coords, dtype), host_as(k, dtype), O.PER_QP, 0.5)
    assert relfro(a.cpu().numpy(), ref.val) <= TOL[dtype]


# ---------------------------------------------------------------- load vector
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("layout", [mg.PER_NODE, mg.PER_QP, mg.CONSTANT])
@pytest.mark.parametrize("el", ELS + [mg.P1_TET_VEC3])
def test_load_matches_oracle(tg, el, layout, dtype):
    m = mesh_for(el)
    ncomp = 3 if el == mg.P1_TET_VEC3 else 1
    nq = mg.NQ[el]
    g = np.random.default_rng(20 + el)
    n = {mg.PER_NODE: m.n_nodes, mg.PER_QP: m.n_elems * nq, mg.CONSTANT: 1}[layout] * ncomp
    f = g.uniform(-1, 1, size=n)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, el)
    F = tg.tg_assemble_load(p, dev(m.coords, dtype), dev(f, dtype), layout, ncomp)
    ref = O.assemble_load(el, m.cells, host_as(m.coords, dtype), host_as(f, dtype), layout, ncomp)
    assert relfro(F.cpu().numpy(), ref) <= TOL[dtype]


# ---------------------------------------------------------------- elasticity
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("layout", [mg.PER_ELEMENT, mg.PER_QP])
def test_elasticity_matches_oracle(tg, layout, dtype):
    m = mesh_for(mg.P1_TET_VEC3)
    lam = coef(layout, m.n_elems, 4, seed=31, lo=0.5, hi=2.0)
    mu = coef(layout, m.n_elems, 4, seed=32, lo=0.3, hi=1.0)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TET_VEC3)
    vals = tg.tg_assemble_elasticity(p, dev(m.coords, dtype), dev(lam, dtype), dev(mu, dtype), layout)
    ref = O.assemble_elasticity(m.cells, host_as(m.coords, dtype), host_as(lam, dtype), host_as(mu, dtype), layout)
    assert p.nnz == ref.nnz
    assert relfro(vals.cpu().numpy(), ref.val) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("fl", [mg.PER_NODE, mg.PER_QP, mg.CONSTANT])
@pytest.mark.parametrize("el", [mg.P1_TRI, mg.P2_TRI, mg.P1_TET])
def test_system_equals_bilinear_and_load_bitwise(tg, el, fl, dtype):
    """The one-pass system assembly returns exactly the separate calls' values."""
    m = mesh_for(el)
    nq = mg.NQ[el]
    k = coef(mg.PER_QP, m.n_elems, nq, seed=81)
    g = np.random.default_rng(82)
    nf = {mg.PER_NODE: m.n_nodes, mg.PER_QP: m.n_elems * nq, mg.CONSTANT: 1}[fl]
    f = g.uniform(-1, 1, size=nf)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, el)
    x, kd, fd = dev(m.coords, dtype), dev(k, dtype), dev(f, dtype)
    vals, F = tg.tg_assemble_system(p, x, kd, mg.PER_QP, 0.7, fd, fl)
    assert torch.equal(vals, tg.tg_assemble_bilinear(p, x, kd, mg.PER_QP, 0.7))
    assert torch.equal(F, tg.tg_assemble_load(p, x, fd, fl))
    ref = O.assemble_load(el, m.cells, host_as(m.coords, dtype), host_as(f, dtype), fl)
    assert relfro(F.cpu().numpy(), ref) <= TOL[dtype]


# ---------------------------------------------------------------- full-size workloads, sampled rows
def _sampled_rows_check(tg, p, vals, ref_fn, n_rows, rows_per_node, seed, tol):
    g = np.random.default_rng(seed)
    nodes = np.unique(g.integers(0, n_rows // rows_per_node, size=400))
    mask = np.zeros(n_rows // rows_per_node, np.uint8)
    mask[nodes] = 1
    ref = ref_fn(mask)
    rp = p.row_ptr.cpu().numpy().astype(np.int64)
    v = vals.cpu().numpy()
    got, want = [], []
    for nd in nodes:
        for r in range(rows_per_node * nd, rows_per_node * nd + rows_per_node):
            assert rp[r + 1] - rp[r] == ref.row_ptr[r + 1] - ref.row_ptr[r]
            got.append(v[rp[r]:rp[r + 1]])
            want.append(ref.val[ref.row_ptr[r]:ref.row_ptr[r + 1]])
            assert np.array_equal(p.col_idx[int(rp[r]):int(rp[r + 1])].cpu().numpy(),
                                  ref.col[ref.row_ptr[r]:ref.row_ptr[r + 1]])
    assert relfro(np.concatenate(got), np.concatenate(want)) <= tol


@pytest.mark.parametrize("dtype", DTYPES)
def test_diffusion2d_full_size_sampled(tg, dtype):
    cfg = mg.diffusion2d(1024)
    m = cfg["mesh"]
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TRI)
    assert p.nnz == 7346177
    vals = tg.tg_assemble_bilinear(p, dev(m.coords, dtype), dev(cfg["kappa"], dtype), mg.PER_QP, cfg["c"])
    xs, ks = host_as(m.coords, dtype), host_as(cfg["kappa"], dtype)
    _sampled_rows_check(tg, p, vals,
                        lambda mask: O.assemble_bilinear(O.P1_TRI, m.cells, xs, ks, O.PER_QP, cfg["c"], row_mask=mask),
                        m.n_nodes, 1, 5, TOL[dtype])
    F = tg.tg_assemble_load(p, dev(m.coords, dtype), dev(cfg["f"], dtype), mg.PER_NODE)
    Fr = O.assemble_load(O.P1_TRI, m.cells, xs, host_as(cfg["f"], dtype), O.PER_NODE)
    assert relfro(F.cpu().numpy(), Fr) <= TOL[dtype]
    assert tg.tg_get_device_status(p) == (0, -1)


def test_elasticity3d_full_size_sampled(tg):
    cfg = mg.elasticity3d(64)
    m = cfg["mesh"]
    dtype = torch.float32
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TET_VEC3)
    assert p.nnz == 36168777
    vals = tg.tg_assemble_elasticity(p, dev(m.coords, dtype), dev(cfg["lam"], dtype), dev(cfg["mu"], dtype),
                                     mg.PER_ELEMENT)
    xs, ls, ms = host_as(m.coords, dtype), host_as(cfg["lam"], dtype), host_as(cfg["mu"], dtype)
    _sampled_rows_check(tg, p, vals,
                        lambda mask: O.assemble_elasticity(m.cells, xs, ls, ms, O.PER_ELEMENT, row_mask=mask),
                        3 * m.n_nodes, 3, 6, TOL[dtype])


# ---------------------------------------------------------------- edge cases
def test_empty_mesh(tg):
    cells = torch.empty((0, 3), dtype=torch.int32, device="cuda")
    p = tg.tg_build_pattern(cells, 5, mg.P1_TRI)
    assert p.nnz == 0 and p.max_row_len == 0
    assert torch.all(p.row_ptr == 0)
    x = torch.zeros((5, 2), dtype=torch.float64, device="cuda")
    vals = tg.tg_assemble_bilinear(p, x, torch.ones(1, dtype=torch.float64, device="cuda"), mg.CONSTANT, 1.0)
    assert vals.numel() == 0
    F = tg.tg_assemble_load(p, x, torch.ones(1, dtype=torch.float64, device="cuda"), mg.CONSTANT)
    assert torch.all(F == 0)


def test_single_element_each_kind(tg):
    cases = [(mg.P1_TRI, [[0, 1, 2]], [[0, 0], [1, 0], [0.25, 0.8]]),
             (mg.P2_TRI, [[0, 1, 2, 3, 4, 5]], [[0, 0], [1, 0], [0.25, 0.8], [0.5, 0], [0.625, 0.4], [0.125, 0.4]]),
             (mg.P1_TET, [[0, 1, 2, 3]], [[0, 0, 0], [1, 0, 0], [0.2, 0.9, 0], [0.1, 0.2, 0.7]])]
    for el, cells, X in cases:
        cells, X = np.array(cells), np.array(X, float)
        p = tg.tg_build_pattern(dev(cells, torch.int32), X.shape[0], el)
        v = tg.tg_assemble_bilinear(p, dev(X, torch.float64), dev([1.3], torch.float64), mg.CONSTANT, 0.4)
        ref = O.assemble_bilinear(el, cells, X, np.array([1.3]), O.CONSTANT, 0.4)
        assert relfro(v.cpu().numpy(), ref.val) <= 1e-14


@pytest.mark.parametrize("el", [mg.P1_TRI, mg.P1_TET])
def test_isolated_nodes_and_shuffled_numbering(tg, el):
    """Nodes that no element uses (zero rows, zero load, zero gradient) and a
    random node numbering (the row blocks' internal order then differs from
    the node order everywhere) match the oracle."""
    m = mesh_for(el)
    g = np.random.default_rng(90)
    n_iso = 37
    N = m.n_nodes + n_iso
    relabel = g.permutation(N)[:m.n_nodes]  # used nodes get random ids; the rest are isolated
    cells = relabel[m.cells]
    X = np.zeros((N, m.coords.shape[1]))
    X[relabel] = m.coords
    X[np.setdiff1d(np.arange(N), relabel)] = g.uniform(0, 1, size=(n_iso, m.coords.shape[1]))
    nq = mg.NQ[el]
    k = coef(mg.PER_QP, len(cells), nq, seed=91)
    f = g.uniform(-1, 1, N)
    p = tg.tg_build_pattern(dev(cells, torch.int32), N, el)
    x = dev(X, torch.float64)
    vals, F = tg.tg_assemble_system(p, x, dev(k, torch.float64), mg.PER_QP, 0.3, dev(f, torch.float64), mg.PER_NODE)
    ref = O.assemble_bilinear(el, cells, X, k, O.PER_QP, 0.3)
    assert np.array_equal(p.row_ptr.cpu().numpy(), ref.row_ptr) and np.array_equal(p.col_idx.cpu().numpy(), ref.col)
    assert relfro(vals.cpu().numpy(), ref.val) <= 1e-12
    assert relfro(F.cpu().numpy(), O.assemble_load(el, cells, X, f, O.PER_NODE)) <= 1e-12
    gv = g.normal(size=p.nnz)
    gk, gx, gc = tg.tg_assemble_backward(p, x, dev(k, torch.float64), mg.PER_QP, 0.3, grad_vals=dev(gv, torch.float64))
    rk, rx, rc = O.assemble_backward(el, cells, X, k, O.PER_QP, 0.3, grad_csr=O.CSR(ref.row_ptr, ref.col, gv))
    assert relfro(gk.cpu().numpy(), rk) <= 1e-12 and relfro(gx.cpu().numpy(), rx) <= 1e-12
    assert relfro(gc.cpu().numpy(), [rc]) <= 1e-12
    iso = np.setdiff1d(np.arange(N), relabel)
    assert np.all(F.cpu().numpy()[iso] == 0) and np.all(gx.cpu().numpy()[iso] == 0)


def test_degenerate_element_is_flagged(tg):
    m = mg.tri_grid(8)  # dyadic coordinates: the collinear triangle has det exactly 0
    X = m.coords.copy()
    e_bad = 17
    a, b, c = m.cells[e_bad]
    X[c] = 0.5 * (X[a] + X[b])
    P = X[m.cells]
    det = (P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1]) - (P[:, 1, 1] - P[:, 0, 1]) * (P[:, 2, 0] - P[:, 0, 0])
    assert np.flatnonzero(det == 0).min() == e_bad
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TRI)
    tg.tg_assemble_bilinear(p, dev(X, torch.float64), dev([1.0], torch.float64), mg.CONSTANT, 0.0)
    st, bad = tg.tg_get_device_status(p)
    assert st == 3 and bad == e_bad
    assert tg.tg_get_device_status(p) == (0, -1)  # read clears


def test_bad_cells_rejected_at_build(tg):
    m = mg.tri_grid(4)
    cells = m.cells.copy()
    cells[5, 1] = m.n_nodes + 3
    with pytest.raises(tg.TGError) as ei:
        tg.tg_build_pattern(dev(cells, torch.int32), m.n_nodes, mg.P1_TRI)
    assert ei.value.status == 2 and "element 5" in str(ei.value)
    cells = m.cells.copy()
    cells[7, 2] = cells[7, 0]
    with pytest.raises(tg.TGError) as ei:
        tg.tg_build_pattern(dev(cells, torch.int32), m.n_nodes, mg.P1_TRI)
    assert ei.value.status == 3 and "element 7" in str(ei.value)


def test_wrong_kind_and_dtype_rejected(tg):
    m = mesh_for(mg.P1_TET_VEC3)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TET_VEC3)
    with pytest.raises(tg.TGError):
        tg.tg_assemble_bilinear(p, dev(m.coords, torch.float64), dev([1.0], torch.float64), mg.CONSTANT, 0.0)
    with pytest.raises(TypeError):
        tg.tg_assemble_elasticity(p, dev(m.coords, torch.float64), dev([1.0], torch.float32), dev([1.0], torch.float64),
                                  mg.CONSTANT)


def test_generic_path_when_blocks_do_not_fit(tg):
    """A random numbering of a 90,601-node mesh makes every block's vertex ids
    span more than 2^16, so the pattern has no row blocks and the generic
    row-owner kernels serve forward, system, backward and the batch."""
    m = jittered_tri(300)
    g = np.random.default_rng(95)
    relabel = g.permutation(m.n_nodes)
    cells = relabel[m.cells]
    X = np.empty_like(m.coords)
    X[relabel] = m.coords
    k = coef(mg.PER_QP, len(cells), 3, seed=96)
    f = g.uniform(-1, 1, m.n_nodes)
    p = tg.tg_build_pattern(dev(cells, torch.int32), m.n_nodes, mg.P1_TRI)
    assert (p.rows_per_block, p.n_blocks) == (0, 0)
    assert p.layouts & (tg.LAYOUT_ROW_BLOCKS | tg.LAYOUT_FANS) == 0
    q = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TRI)
    assert q.rows_per_block > 0 and q.n_blocks == -(-m.n_nodes // q.rows_per_block)
    x, kd, fd = dev(X, torch.float64), dev(k, torch.float64), dev(f, torch.float64)
    vals, F = tg.tg_assemble_system(p, x, kd, mg.PER_QP, 0.2, fd, mg.PER_NODE)
    ref = O.assemble_bilinear(mg.P1_TRI, cells, X, k, O.PER_QP, 0.2)
    assert relfro(vals.cpu().numpy(), ref.val) <= 1e-12
    assert relfro(F.cpu().numpy(), O.assemble_load(mg.P1_TRI, cells, X, f, O.PER_NODE)) <= 1e-12
    assert torch.equal(vals, tg.tg_assemble_bilinear(p, x, kd, mg.PER_QP, 0.2))
    gv = g.normal(size=p.nnz)
    gk, gx, gc = tg.tg_assemble_backward(p, x, kd, mg.PER_QP, 0.2, grad_vals=dev(gv, torch.float64))
    rk, rx, rc = O.assemble_backward(mg.P1_TRI, cells, X, k, O.PER_QP, 0.2, grad_csr=O.CSR(ref.row_ptr, ref.col, gv))
    assert relfro(gk.cpu().numpy(), rk) <= 1e-12 and relfro(gx.cpu().numpy(), rx) <= 1e-12
    assert relfro(gc.cpu().numpy(), [rc]) <= 1e-12
    b = tg.tg_batch_create([p, p])
    out = [torch.empty(p.nnz, dtype=torch.float64, device="cuda") for _ in range(2)]
    tg.tg_batch_assemble(b, [x, x], [kd, kd], mg.PER_QP, [0.2, 0.2], out)
    assert torch.equal(out[0], vals) and torch.equal(out[1], vals)


def test_vertex_joining_two_fans(tg):
    """A vertex where two separate fans of triangles meet (a triangle hung on
    the corner of a grid by that vertex alone): the pattern then keeps the
    element-order Reduce, and every output matches the oracle."""
    m = jittered_tri(12, seed=41)
    X = np.vstack([m.coords, [[-0.30, -0.05], [-0.05, -0.30]]])
    corner = int(np.flatnonzero((m.coords[:, 0] == 0) & (m.coords[:, 1] == 0))[0])
    N = m.n_nodes + 2
    cells = np.vstack([m.cells, [[corner, N - 2, N - 1]]])
    g = np.random.default_rng(42)
    k = g.uniform(0.5, 2.0, size=(len(cells), 3))
    f = g.uniform(-1, 1, N)
    p = tg.tg_build_pattern(dev(cells, torch.int32), N, mg.P1_TRI)
    assert p.n_blocks > 0
    assert p.layouts & tg.LAYOUT_ROW_BLOCKS and not p.layouts & tg.LAYOUT_FANS
    assert tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, mg.P1_TRI).layouts & tg.LAYOUT_FANS
    x = dev(X, torch.float64)
    vals, F = tg.tg_assemble_system(p, x, dev(k, torch.float64), mg.PER_QP, 0.6, dev(f, torch.float64), mg.PER_NODE)
    ref = O.assemble_bilinear(mg.P1_TRI, cells, X, k, O.PER_QP, 0.6)
    assert np.array_equal(p.col_idx.cpu().numpy(), ref.col)
    assert relfro(vals.cpu().numpy(), ref.val) <= 1e-12
    assert relfro(F.cpu().numpy(), O.assemble_load(mg.P1_TRI, cells, X, f, O.PER_NODE)) <= 1e-12
    gv = g.normal(size=p.nnz)
    gk, gx, gc = tg.tg_assemble_backward(p, x, dev(k, torch.float64), mg.PER_QP, 0.6, grad_vals=dev(gv, torch.float64))
    rk, rx, rc = O.assemble_backward(mg.P1_TRI, cells, X, k, O.PER_QP, 0.6, grad_csr=O.CSR(ref.row_ptr, ref.col, gv))
    assert relfro(gk.cpu().numpy().ravel(), rk) <= 1e-12 and relfro(gx.cpu().numpy(), rx) <= 1e-12
    xf, kf = dev(X, torch.float32), dev(k, torch.float32)
    v32 = tg.tg_assemble_bilinear(p, xf, kf, mg.PER_QP, 0.6)
    r32 = O.assemble_bilinear(mg.P1_TRI, cells, host_as(X, torch.float32), host_as(k, torch.float32), O.PER_QP, 0.6)
    assert relfro(v32.cpu().numpy(), r32.val) <= 2e-6


def test_fp64_reciprocal_within_one_ulp(tg):
    """The FP64 reciprocal that the P1 forward kernels take of |det J|
    (Newton's iteration from an FP32 seed) is within one unit in the last
    place of the correctly rounded 1/x over the seed's range, at its edges and
    at powers of two, for both signs; outside that range it is the quotient
    itself."""
    g = np.random.default_rng(77)
    inside = 2.0 ** g.uniform(-120, 119, 400000) * g.uniform(1, 2, 400000)
    edges = np.array([2.0 ** -120, np.nextafter(2.0 ** -120, 1), 2.0 ** 119.9999, np.nextafter(2.0 ** 120, 0), 1.0,
                      3.0, 1 / 3, np.nextafter(1.0, 2), np.nextafter(1.0, 0), 0.1, 1e-30, 1e30])
    pow2 = 2.0 ** np.arange(-120, 120)
    near = np.concatenate([np.nextafter(pow2[1:], 0), np.nextafter(pow2[:-1], np.inf)])
    x = np.concatenate([inside, edges, pow2, near])
    x = np.concatenate([x, -x])
    outside = np.array([1e-300, 2.0 ** -121, np.nextafter(2.0 ** -120, 0), 2.0 ** 120, 1e300, -1e-300, -2.0 ** 121])
    y = tg.tg_diag_recip(torch.as_tensor(np.concatenate([x, outside]), device="cuda")).cpu().numpy()
    want = 1.0 / x
    err = np.abs(y[:len(x)] - want) / np.spacing(np.abs(want))
    assert err.max() <= 1.0, err.max()
    assert np.array_equal(y[len(x):], 1.0 / outside)
    assert tg.tg_diag_recip(torch.empty(0, dtype=torch.float64, device="cuda")).numel() == 0


@pytest.mark.parametrize("el,dtype", [(mg.P1_TRI, torch.float64), (mg.P1_TET, torch.float64),
                                      (mg.P1_TET, torch.float32)])
def test_two_pass_forward_and_system(tg, el, dtype):
    """P1 meshes of at least 65,536 elements in FP64, and tetrahedral ones in
    FP32, are assembled in two passes (every element's K_e and F_e once into
    the pattern's scratch, then the rows' and nodes' sums): the system equals
    the separate forward and load calls bitwise, both meet the oracle, and a
    degenerate element is flagged with zero entries as in one pass."""
    m = jittered_tri(192) if el == mg.P1_TRI else jittered_tet(24)
    assert m.n_elems >= 1 << 16
    k = coef(mg.PER_QP, m.n_elems, mg.NQ[el], seed=91)
    f = np.random.default_rng(92).uniform(-1, 1, m.n_nodes)
    p = tg.tg_build_pattern(dev(m.cells, torch.int32), m.n_nodes, el)
    x, kd, fd = dev(m.coords, dtype), dev(k, dtype), dev(f, dtype)
    vals, F = tg.tg_assemble_system(p, x, kd, mg.PER_QP, 0.4, fd, mg.PER_NODE)
    assert torch.equal(vals, tg.tg_assemble_bilinear(p, x, kd, mg.PER_QP, 0.4))
    assert torch.equal(F, tg.tg_assemble_load(p, x, fd, mg.PER_NODE))
    xs, ks, fs = host_as(m.coords, dtype), host_as(k, dtype), host_as(f, dtype)
    ref = O.assemble_bilinear(el, m.cells, xs, ks, O.PER_QP, 0.4)
    assert relfro(vals.cpu().numpy(), ref.val) <= TOL[dtype]
    assert relfro(F.cpu().numpy(), O.assemble_load(el, m.cells, xs, fs, O.PER_NODE)) <= TOL[dtype]
    # a collapsed element: flagged, and it adds nothing
    X = m.coords.copy()
    a, b = m.cells[17][0], m.cells[17][1]
    X[b] = X[a]
    vals2 = tg.tg_assemble_bilinear(p, dev(X, dtype), kd, mg.PER_QP, 0.4)
    st, bad = tg.tg_get_device_status(p)
    assert st != 0 and bad <= 17
    assert torch.isfinite(vals2).all()
