"""Properties of the seeded input generators (sizes, orientation, conformity)."""
import numpy as np

import meshgen as mg


def _signed_area(m):
    X = m.coords[m.cells[:, :3]]
    return 0.5 * ((X[:, 1, 0] - X[:, 0, 0]) * (X[:, 2, 1] - X[:, 0, 1]) - (X[:, 1, 1] - X[:, 0, 1]) * (X[:, 2, 0] - X[:, 0, 0]))


def _edge_count_nnz(cells, n_nodes):
    nv = cells.shape[1]
    pairs = np.stack([np.repeat(cells, nv, axis=1).ravel(), np.tile(cells, (1, nv)).ravel()], 1).astype(np.int64)
    key = np.unique(pairs[:, 0] * n_nodes + pairs[:, 1])
    return key.size


def test_tri_grid_sizes_and_orientation():
    m = mg.tri_grid(64)
    assert (m.n_elems, m.n_nodes) == (8192, 4225)
    assert _edge_count_nnz(m.cells, m.n_nodes) == 29057
    assert np.all(_signed_area(m) > 0)
    assert abs(_signed_area(m).sum() - 1.0) < 1e-14


def test_diffusion2d_full_size_shape():
    c = mg.diffusion2d(1024)
    m = c["mesh"]
    assert (m.n_elems, m.n_nodes) == (2097152, 1050625)
    # nnz = N + 2 * #edges, #edges = 3 n^2 + 2 n for this triangulation
    assert m.n_nodes + 2 * (3 * 1024 ** 2 + 2 * 1024) == 7346177
    assert np.all(_signed_area(m) > 0)
    assert c["kappa"].shape == (2097152, 3)
    assert np.all(c["kappa"] > 0)


def test_hilbert_order_is_a_permutation_with_locality():
    base = mg.jitter(mg.tri_grid(32), 2)
    h = mg.hilbert_order(base)
    a = np.sort(base.cells, axis=1)
    b = np.sort(h.cells, axis=1)
    ka = np.sort(a[:, 0] * 10 ** 8 + a[:, 1] * 10 ** 4 + a[:, 2])
    kb = np.sort(b[:, 0] * 10 ** 8 + b[:, 1] * 10 ** 4 + b[:, 2])
    assert np.array_equal(ka, kb)
    cen = h.coords[h.cells].mean(1)
    step = np.linalg.norm(np.diff(cen, axis=0), axis=1)
    assert np.median(step) < 1.5 / 32


def test_p2_grid_conforming():
    m = mg.p2_tri_grid(5, jitter_seed=1)
    assert m.n_nodes == 11 * 11 and m.n_elems == 50
    # each edge node is shared by at most two elements, vertices are edge endpoints' midpoints
    for k, (a, b) in zip((3, 4, 5), ((0, 1), (1, 2), (2, 0))):
        mid = 0.5 * (m.coords[m.cells[:, a]] + m.coords[m.cells[:, b]])
        assert np.allclose(m.coords[m.cells[:, k]], mid)
    counts = np.bincount(m.cells[:, 3:].ravel(), minlength=m.n_nodes)
    assert counts.max() == 2
    assert np.all(_signed_area(m) > 0)


def test_kuhn_tets_fill_the_cube():
    m = mg.kuhn_tet_grid(3)
    X = m.coords[m.cells]
    det = np.linalg.det(np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], -1))
    assert abs(np.abs(det).sum() / 6 - 1.0) < 1e-14
    assert np.all(np.abs(det) > 0)
    # conforming: every interior face is shared by exactly two tets
    faces = np.sort(np.concatenate([m.cells[:, [1, 2, 3]], m.cells[:, [0, 2, 3]], m.cells[:, [0, 1, 3]], m.cells[:, [0, 1, 2]]]), 1)
    _, cnt = np.unique(faces, axis=0, return_counts=True)
    assert cnt.max() == 2
    n = 3
    assert (cnt == 1).sum() == 6 * 2 * n * n  # boundary triangles


def test_elasticity3d_sizes():
    c = mg.elasticity3d(64)
    m = c["mesh"]
    assert (m.n_elems, m.n_nodes) == (1572864, 274625)
    assert c["lam"].min() >= 0.5 and c["lam"].max() <= 2.0
    assert c["mu"].min() >= 0.3 and c["mu"].max() <= 1.0


def test_batch_sizes_range_and_determinism():
    s1 = mg.batch_sizes()
    s2 = mg.batch_sizes()
    assert s1 == s2 and len(s1) == 256
    nodes = [(2 * n + 1) ** 2 for n in s1]
    assert min(nodes) >= 1600 and max(nodes) <= 51000


def test_smooth_kappa_star_bounds():
    m = mg.kuhn_tet_grid(4)
    k = mg.smooth_kappa_star(m.coords[m.cells].mean(1))
    assert np.all(k > 0.59) and np.all(k < 1.41)
