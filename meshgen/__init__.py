"""Seeded synthetic inputs: simplex meshes and coefficient fields.

This module is shared by the oracle tests, the GPU parity tests and the
benchmark.  It holds mesh construction (node coordinates, element
connectivity, orderings) and random draws only; it contains none of the
assembly arithmetic, so neither side of a parity comparison can inherit a
mistake from it.

Conventions (the input recipe of the benchmark workloads):

* 2D grids: unit square, ``(n+1)^2`` nodes numbered lexicographically
  (``id = j*(n+1) + i`` for ``x = i/n, y = j/n``); every cell is cut by the
  diagonal from ``(i, j)`` to ``(i+1, j+1)`` into two counter-clockwise
  right triangles.
* P2 triangles: six nodes per element, the three vertices followed by the
  edge nodes of the edges (0,1), (1,2), (2,0).  Edge nodes sit at the edge
  midpoints (straight-sided elements).
* 3D grids: unit cube, ``(n+1)^3`` nodes numbered lexicographically; each
  hexahedral cell is cut into the six Kuhn tetrahedra, one per permutation
  of the axes (the monotone lattice paths from the cell's low corner to its
  high corner).
* Jitter moves interior nodes only, each coordinate independently by
  ``U(-0.2h, 0.2h)``; this keeps every triangle positively oriented.
* Hilbert order: elements are stably sorted by the 2D Hilbert index of their
  centroid quantised to a ``2^16 x 2^16`` grid.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------
# element kinds (names shared with the C ABI enum by value, not by code)
P1_TRI, P2_TRI, P1_TET, P1_TET_VEC3, Q1_QUAD_VEC2 = 0, 1, 2, 3, 4
NV = {P1_TRI: 3, P2_TRI: 6, P1_TET: 4, P1_TET_VEC3: 4, Q1_QUAD_VEC2: 4}
DIM = {P1_TRI: 2, P2_TRI: 2, P1_TET: 3, P1_TET_VEC3: 3, Q1_QUAD_VEC2: 2}
NQ = {P1_TRI: 3, P2_TRI: 6, P1_TET: 4, P1_TET_VEC3: 4, Q1_QUAD_VEC2: 4}

# coefficient layouts
PER_ELEMENT, PER_QP, PER_NODE, CONSTANT = 0, 1, 2, 3


@dataclass
class Mesh:
    el: int
    coords: np.ndarray          # [N, d] float64
    cells: np.ndarray           # [E, nv] int32
    boundary: np.ndarray        # [N] bool, node on the domain boundary
    h: float = 0.0
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.coords.shape[0])

    @property
    def n_elems(self) -> int:
        return int(self.cells.shape[0])


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# --------------------------------------------------------------------------
# 2D structured triangle grids
def tri_grid(n: int) -> Mesh:
    """Unit square, n x n cells, two right triangles per cell."""
    m = n + 1
    ii, jj = np.meshgrid(np.arange(m), np.arange(m), indexing="xy")
    coords = np.stack([ii.ravel() / n, jj.ravel() / n], axis=1).astype(np.float64)
    ci, cj = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    ci = ci.ravel()
    cj = cj.ravel()
    v00 = cj * m + ci
    v10 = v00 + 1
    v01 = v00 + m
    v11 = v01 + 1
    lower = np.stack([v00, v10, v11], axis=1)
    upper = np.stack([v00, v11, v01], axis=1)
    cells = np.empty((2 * n * n, 3), dtype=np.int32)
    cells[0::2] = lower
    cells[1::2] = upper
    x = coords[:, 0]
    y = coords[:, 1]
    on_bnd = (ii.ravel() == 0) | (ii.ravel() == n) | (jj.ravel() == 0) | (jj.ravel() == n)
    return Mesh(P1_TRI, coords, cells, on_bnd, h=1.0 / n, meta={"n": n})


def quad_grid(nx: int, ny: int, lx: float = 1.0, ly: float = 1.0) -> Mesh:
    """[0, lx] x [0, ly] cut into nx x ny bilinear quadrilaterals; nodes
    numbered lexicographically (id = j (nx + 1) + i), each cell's corners
    counter-clockwise from its low corner."""
    mx = nx + 1
    ii, jj = np.meshgrid(np.arange(mx), np.arange(ny + 1), indexing="xy")
    coords = np.stack([ii.ravel() * (lx / nx), jj.ravel() * (ly / ny)], axis=1).astype(np.float64)
    ci, cj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    v00 = (cj * mx + ci).ravel()
    cells = np.stack([v00, v00 + 1, v00 + mx + 1, v00 + mx], axis=1).astype(np.int32)
    on_bnd = (ii.ravel() == 0) | (ii.ravel() == nx) | (jj.ravel() == 0) | (jj.ravel() == ny)
    return Mesh(Q1_QUAD_VEC2, coords, cells, on_bnd, h=min(lx / nx, ly / ny), meta={"nx": nx, "ny": ny})


def cantilever(nx: int = 60, ny: int = 30, lx: float = 60.0, ly: float = 30.0, load: float = -100.0) -> dict:
    """Plane-stress cantilever of the SIMP compliance benchmark: quads,
    clamped on x = 0, a downward traction on the part of x = lx with
    y <= 0.1 ly, lumped to its nodes (each edge of length l gives l t / 2 to
    its two ends), uniform density 0.5."""
    mesh = quad_grid(nx, ny, lx, ly)
    x, y = mesh.coords[:, 0], mesh.coords[:, 1]
    F = np.zeros(2 * mesh.n_nodes)
    edge_nodes = np.flatnonzero(np.isclose(x, lx) & (y <= 0.1 * ly + 1e-12))
    edge_nodes = edge_nodes[np.argsort(y[edge_nodes])]
    for a, b in zip(edge_nodes[:-1], edge_nodes[1:]):
        le = y[b] - y[a]
        F[2 * a + 1] += load * le / 2
        F[2 * b + 1] += load * le / 2
    clamped = np.repeat(np.isclose(x, 0.0), 2)
    return {"mesh": mesh, "F": F, "dirichlet": clamped, "rho": np.full(mesh.n_elems, 0.5), "E_min": 70.0,
            "E_max": 70000.0, "penal": 3.0, "nu": 0.3}


def jitter(mesh: Mesh, seed: int, frac: float = 0.2) -> Mesh:
    """Move interior nodes by U(-frac*h, frac*h) per coordinate."""
    g = rng(seed)
    d = mesh.coords.shape[1]
    disp = g.uniform(-frac * mesh.h, frac * mesh.h, size=(mesh.n_nodes, d))
    disp[mesh.boundary] = 0.0
    out = Mesh(mesh.el, mesh.coords + disp, mesh.cells.copy(), mesh.boundary.copy(), mesh.h, dict(mesh.meta))
    return out


def _hilbert_d2(x: np.ndarray, y: np.ndarray, bits: int) -> np.ndarray:
    """Hilbert curve index of integer points (x, y) in [0, 2^bits)^2."""
    x = x.astype(np.int64).copy()
    y = y.astype(np.int64).copy()
    side = 1 << bits
    d = np.zeros_like(x)
    s = side >> 1
    while s > 0:
        rx = ((x & s) > 0).astype(np.int64)
        ry = ((y & s) > 0).astype(np.int64)
        d += s * s * ((3 * rx) ^ ry)
        flip = (ry == 0) & (rx == 1)
        x = np.where(flip, side - 1 - x, x)
        y = np.where(flip, side - 1 - y, y)
        swap = ry == 0
        x, y = np.where(swap, y, x), np.where(swap, x, y)
        s >>= 1
    return d


def hilbert_order(mesh: Mesh, bits: int = 16) -> Mesh:
    """Reorder elements along the 2D Hilbert curve of their centroids."""
    nv_geo = 3
    cen = mesh.coords[mesh.cells[:, :nv_geo]].mean(axis=1)
    lo = mesh.coords.min(axis=0)
    hi = mesh.coords.max(axis=0)
    scale = (1 << bits) - 1
    q = np.clip(np.floor((cen - lo) / (hi - lo) * scale + 0.5), 0, scale).astype(np.int64)
    key = _hilbert_d2(q[:, 0], q[:, 1], bits)
    perm = np.argsort(key, kind="stable")
    out = Mesh(mesh.el, mesh.coords, np.ascontiguousarray(mesh.cells[perm]), mesh.boundary, mesh.h, dict(mesh.meta))
    out.meta["hilbert"] = True
    return out


def p2_tri_grid(n: int, jitter_seed: int | None = None, frac: float = 0.2) -> Mesh:
    """P2 triangles on the n x n grid; nodes on the (2n+1)^2 half-step lattice.

    Vertex (i, j) of the coarse grid is lattice node (2i, 2j); the edge node
    of the edge between coarse vertices p and q is lattice node p + q.
    """
    base = tri_grid(n)
    if jitter_seed is not None:
        base = jitter(base, jitter_seed, frac)
    m = n + 1
    M = 2 * n + 1
    vi = np.arange(m * m) % m
    vj = np.arange(m * m) // m
    lat_of_vertex = (2 * vj) * M + 2 * vi
    c = base.cells.astype(np.int64)
    pi = np.stack([c % m, c // m], axis=-1)  # [E,3,2] coarse lattice coords

    def edge_node(a, b):
        s = pi[:, a] + pi[:, b]
        return s[:, 1] * M + s[:, 0]

    cells = np.empty((c.shape[0], 6), dtype=np.int64)
    cells[:, 0:3] = lat_of_vertex[c]
    cells[:, 3] = edge_node(0, 1)
    cells[:, 4] = edge_node(1, 2)
    cells[:, 5] = edge_node(2, 0)
    coords = np.full((M * M, 2), np.nan)
    coords[lat_of_vertex] = base.coords
    for a, b, k in ((0, 1, 3), (1, 2, 4), (2, 0, 5)):
        coords[cells[:, k]] = 0.5 * (base.coords[c[:, a]] + base.coords[c[:, b]])
    assert not np.isnan(coords).any()
    li = np.arange(M * M) % M
    lj = np.arange(M * M) // M
    bnd = (li == 0) | (li == M - 1) | (lj == 0) | (lj == M - 1)
    return Mesh(P2_TRI, coords, cells.astype(np.int32), bnd, h=1.0 / n, meta={"n": n})


# --------------------------------------------------------------------------
# 3D structured tetrahedral grids
_KUHN_PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


def kuhn_tet_grid(n: int) -> Mesh:
    """Unit cube, n^3 hexahedra, six Kuhn tetrahedra per hexahedron."""
    m = n + 1
    idx = np.arange(m ** 3)
    i = idx % m
    j = (idx // m) % m
    k = idx // (m * m)
    coords = np.stack([i / n, j / n, k / n], axis=1).astype(np.float64)
    ci, cj, ck = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ci, cj, ck = ci.ravel(order="F"), cj.ravel(order="F"), ck.ravel(order="F")
    stride = np.array([1, m, m * m], dtype=np.int64)
    base = ck * m * m + cj * m + ci
    tets = []
    for p in _KUHN_PERMS:
        v0 = base
        v1 = v0 + stride[p[0]]
        v2 = v1 + stride[p[1]]
        v3 = v2 + stride[p[2]]
        tets.append(np.stack([v0, v1, v2, v3], axis=1))
    cells = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    bnd = (i == 0) | (i == n) | (j == 0) | (j == n) | (k == 0) | (k == n)
    return Mesh(P1_TET, coords, cells, bnd, h=1.0 / n, meta={"n": n})


# --------------------------------------------------------------------------
# coefficient and load draws
def boundary_facets(mesh: Mesh) -> np.ndarray:
    """Facets that belong to exactly one element (the domain boundary):
    edges of P1 triangles ([F, 2]) or faces of P1 tetrahedra ([F, 3]), each
    with its vertices in ascending order, facets in lexicographic order."""
    cells = np.asarray(mesh.cells)
    nv = cells.shape[1]
    d = nv - 1
    local = [c for c in __import__("itertools").combinations(range(nv), d)]
    f = np.sort(np.concatenate([cells[:, list(c)] for c in local]), axis=1)
    uniq, count = np.unique(f, axis=0, return_counts=True)
    return uniq[count == 1].astype(np.int32)


def lognormal(shape, seed: int, sigma: float = 1.0) -> np.ndarray:
    return np.exp(rng(seed).normal(0.0, sigma, size=shape))


def uniform(shape, seed: int, lo: float, hi: float) -> np.ndarray:
    return rng(seed).uniform(lo, hi, size=shape)


def round_to(a: np.ndarray, dtype) -> np.ndarray:
    """Round to ``dtype`` and promote back to float64 (what an FP32 run sees)."""
    return np.asarray(a, dtype=dtype).astype(np.float64)


# --------------------------------------------------------------------------
# the benchmark workloads (sizes are parameters so tests can shrink them)
def poisson2d(n: int = 64) -> dict:
    """Structured P1 Poisson on the unit square: kappa = 1, c = 0, f = 1."""
    mesh = tri_grid(n)
    return {"mesh": mesh, "kappa": np.ones(mesh.n_elems * 3), "c": 0.0, "f": 1.0}


def diffusion2d(n: int = 1024, seed_jitter: int = 2, seed_kappa: int = 22, seed_f: int = 222) -> dict:
    """Jittered, Hilbert-ordered P1 triangles; lognormal kappa at 3 points."""
    mesh = hilbert_order(jitter(tri_grid(n), seed_jitter))
    kappa = lognormal((mesh.n_elems, 3), seed_kappa)
    f = uniform(mesh.n_nodes, seed_f, -1.0, 1.0)
    return {"mesh": mesh, "kappa": kappa, "c": 1.0, "f": f}


def elasticity3d(n: int = 64, seed: int = 3) -> dict:
    """Kuhn tetrahedra of the unit cube; Lame lambda, mu per element."""
    mesh = kuhn_tet_grid(n)
    mesh.el = P1_TET_VEC3
    g = rng(seed)
    lam = g.uniform(0.5, 2.0, size=mesh.n_elems)
    mu = g.uniform(0.3, 1.0, size=mesh.n_elems)
    return {"mesh": mesh, "lam": lam, "mu": mu, "body_force": np.array([0.0, 0.0, -1.0])}


def batch_sizes(n_inst: int = 256, seed: int = 4, lo: int = 2000, hi: int = 50000) -> list[int]:
    """Grid sizes n_i of the batched P2 instances (target node counts U{lo..hi})."""
    g = rng(seed)
    nodes = g.integers(lo, hi + 1, size=n_inst)
    return [max(1, int(round((math.sqrt(int(N)) - 1.0) / 2.0))) for N in nodes]


def batched_p2(n_inst: int = 256, seed: int = 4, sizes: list[int] | None = None) -> list[dict]:
    """Independent jittered, Hilbert-ordered P2 instances with lognormal kappa at 6 points."""
    if sizes is None:
        sizes = batch_sizes(n_inst, seed)
    g = rng(seed + 1000)
    seeds = g.integers(0, 2 ** 31 - 1, size=(len(sizes), 2))
    out = []
    for (n, (sj, sk)) in zip(sizes, seeds):
        mesh = p2_tri_grid(n, jitter_seed=int(sj))
        mesh = hilbert_order(mesh)
        kappa = lognormal((mesh.n_elems, 6), int(sk))
        out.append({"mesh": mesh, "kappa": kappa, "c": 0.0})
    return out


def smooth_kappa_star(centroids: np.ndarray, seed: int = 5) -> np.ndarray:
    """kappa*(x) = 1 + 0.4 * sum_m a_m sin(pi k_m . x) / 4, a_m ~ U(-1,1), k_m in {1,2}^3."""
    g = rng(seed)
    a = g.uniform(-1.0, 1.0, size=4)
    k = g.integers(1, 3, size=(4, 3))
    s = np.zeros(centroids.shape[0])
    for m in range(4):
        s += a[m] * np.sin(np.pi * centroids @ k[m].astype(np.float64)) / 4.0
    return 1.0 + 0.4 * s


def differentiable3d(n: int = 48, seed: int = 5) -> dict:
    """Kuhn tetrahedra; learnable per-element kappa ~ U(0.5, 1.5); f = 1."""
    mesh = kuhn_tet_grid(n)
    kappa = rng(seed + 1).uniform(0.5, 1.5, size=mesh.n_elems)
    cen = mesh.coords[mesh.cells].mean(axis=1)
    kstar = smooth_kappa_star(cen, seed)
    return {"mesh": mesh, "kappa": kappa, "kappa_star": kstar, "f": 1.0}


def fd_directions(n_dir: int, size: int, seed: int = 55) -> np.ndarray:
    """Unit random directions for finite-difference gradient checks."""
    v = rng(seed).normal(size=(n_dir, size))
    return v / np.linalg.norm(v, axis=1, keepdims=True)
