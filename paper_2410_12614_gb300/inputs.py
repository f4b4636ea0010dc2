"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module only *generates* inputs: structured simplex meshes with jittered
interior vertices, lognormal coefficients at quadrature points and Gaussian
vectors.  It holds none of the method's arithmetic (no basis functions, no
geometry, no quadrature, no contraction), so that the CPU oracle and the GPU
library can both be fed from it without sharing any computation.

Mesh recipe (the paper's Gmsh meshes are replaced by structured meshes):

* square, N x N boxes of side h = 1/N, vertex (i, j) at (i h, j h) with id
  ``j (N+1) + i``; box (i, j) is cut along its (i,j)-(i+1,j+1) diagonal into
  the triangles (v00, v10, v11) and (v00, v11, v01); the cell id of box (i, j)
  is ``2 (j N + i) + {0, 1}``.
* cube, N^3 boxes, vertex (i, j, k) with id ``(k (N+1) + j) (N+1) + i``; each
  box is cut into the six Kuhn tetrahedra
  ``[o, o + e_a, o + e_a + e_b, o + (1,1,1)]`` for the permutations (a, b, c)
  of the axes in lexicographic order; cell id ``6 box + perm``, box id
  ``(k N + j) N + i``.  The Kuhn split is conforming across boxes.
* boxed cells (quadrilaterals, hexahedra): the same vertex grids, one cell
  per box with its 2^d corners in tensor order (corner v at box offset
  (bit_0(v), bit_1(v), bit_2(v))); cell id = box id.
* jitter: every strictly interior vertex moves each coordinate by an
  independent U(-alpha h, alpha h) draw.  alpha <= 0.2 keeps every cell valid.
* kappa[c, q] = exp(N(0, 1)), i.i.d. per cell and quadrature point.

Random numbers come from numpy's PCG64 generator seeded with the given seed.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

__all__ = [
    "square_mesh",
    "cube_mesh",
    "quad_mesh",
    "hex_mesh",
    "structured_mesh",
    "lognormal_kappa",
    "gaussian_vector",
    "batched_workload",
]


def square_mesh(n: int, alpha: float = 0.0, seed: int = 0):
    """Unit square, n x n boxes, 2 triangles each.  Returns (vertices, cells).

    vertices: float64 [(n+1)^2, 2]; cells: int32 [2 n^2, 3].
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    h = 1.0 / n
    j, i = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    vertices = np.stack([i.ravel() * h, j.ravel() * h], axis=1).astype(np.float64)
    cells = np.empty((2 * n * n, 3), dtype=np.int32)
    c = 0
    for jj in range(n):
        for ii in range(n):
            v00 = jj * (n + 1) + ii
            v10 = v00 + 1
            v01 = v00 + (n + 1)
            v11 = v01 + 1
            cells[c] = (v00, v10, v11)
            cells[c + 1] = (v00, v11, v01)
            c += 2
    _jitter(vertices, n, 2, alpha, h, seed)
    return vertices, cells


_KUHN_PERMS = list(itertools.permutations(range(3)))  # lexicographic order


def cube_mesh(n: int, alpha: float = 0.0, seed: int = 0):
    """Unit cube, n^3 boxes, 6 Kuhn tetrahedra each.  Returns (vertices, cells).

    vertices: float64 [(n+1)^3, 3]; cells: int32 [6 n^3, 4].
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    h = 1.0 / n
    k, j, i = np.meshgrid(np.arange(n + 1), np.arange(n + 1), np.arange(n + 1), indexing="ij")
    vertices = np.stack([i.ravel() * h, j.ravel() * h, k.ravel() * h], axis=1).astype(np.float64)

    def vid(ii, jj, kk):
        return (kk * (n + 1) + jj) * (n + 1) + ii

    # vectorised over boxes
    kb, jb, ib = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ib, jb, kb = ib.ravel(), jb.ravel(), kb.ravel()
    cells = np.empty((n ** 3, 6, 4), dtype=np.int64)
    for p_idx, perm in enumerate(_KUHN_PERMS):
        corner = [ib.copy(), jb.copy(), kb.copy()]
        cells[:, p_idx, 0] = vid(*corner)
        for step in range(3):
            corner[perm[step]] = corner[perm[step]] + 1
            cells[:, p_idx, step + 1] = vid(*corner)
    cells = cells.reshape(-1, 4).astype(np.int32)
    _jitter(vertices, n, 3, alpha, h, seed)
    return vertices, cells


def _box_cells(n: int, d: int):
    nv = 1 << d
    grids = np.meshgrid(*[np.arange(n)] * d, indexing="ij")      # [k][j][i] order for d = 3
    idx = [g.ravel() for g in grids[::-1]]                        # i, j(, k): x fastest
    cells = np.empty((n ** d, nv), dtype=np.int64)
    for v in range(nv):
        vid = np.zeros(n ** d, dtype=np.int64)
        for axis in reversed(range(d)):
            vid = vid * (n + 1) + idx[axis] + ((v >> axis) & 1)
        cells[:, v] = vid
    return cells.astype(np.int32)


def quad_mesh(n: int, alpha: float = 0.0, seed: int = 0):
    """Unit square, n x n quadrilaterals (vertex ids as square_mesh).
    Returns (vertices float64 [(n+1)^2, 2], cells int32 [n^2, 4])."""
    if n < 1:
        raise ValueError("n must be >= 1")
    h = 1.0 / n
    j, i = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    vertices = np.stack([i.ravel() * h, j.ravel() * h], axis=1).astype(np.float64)
    cells = _box_cells(n, 2)
    _jitter(vertices, n, 2, alpha, h, seed)
    return vertices, cells


def hex_mesh(n: int, alpha: float = 0.0, seed: int = 0):
    """Unit cube, n^3 hexahedra (vertex ids as cube_mesh).
    Returns (vertices float64 [(n+1)^3, 3], cells int32 [n^3, 8])."""
    if n < 1:
        raise ValueError("n must be >= 1")
    h = 1.0 / n
    k, j, i = np.meshgrid(np.arange(n + 1), np.arange(n + 1), np.arange(n + 1), indexing="ij")
    vertices = np.stack([i.ravel() * h, j.ravel() * h, k.ravel() * h], axis=1).astype(np.float64)
    cells = _box_cells(n, 3)
    _jitter(vertices, n, 3, alpha, h, seed)
    return vertices, cells


def structured_mesh(cell_type: str, n: int, alpha: float, seed: int):
    """``cell_type`` in {"triangle", "tetrahedron", "quadrilateral", "hexahedron"}."""
    if cell_type in ("triangle", "tri"):
        return square_mesh(n, alpha, seed)
    if cell_type in ("tetrahedron", "tet"):
        return cube_mesh(n, alpha, seed)
    if cell_type in ("quadrilateral", "quad"):
        return quad_mesh(n, alpha, seed)
    if cell_type in ("hexahedron", "hex"):
        return hex_mesh(n, alpha, seed)
    raise ValueError(f"unknown cell type {cell_type!r}")


def _jitter(vertices, n, d, alpha, h, seed):
    if alpha == 0.0:
        return
    if not (0.0 <= alpha < 0.25):
        raise ValueError("alpha must lie in [0, 0.25)")
    rng = np.random.default_rng(seed)
    idx = np.rint(vertices / h).astype(np.int64)
    interior = np.all((idx > 0) & (idx < n), axis=1)
    shift = rng.uniform(-alpha * h, alpha * h, size=vertices.shape)
    vertices[interior] += shift[interior]


def lognormal_kappa(n_cells: int, n_q: int, seed: int) -> np.ndarray:
    """kappa[c, q] = exp(N(0,1)), float64 [n_cells, n_q]."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.standard_normal((n_cells, n_q)))


def gaussian_vector(n: int, seed: int, dtype=np.float32) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n).astype(dtype)


def batched_workload(n_meshes: int = 256, seed: int = 6, lo: float = 1e3, hi: float = 2e5):
    """Descriptors of the uneven batched workload.

    Each entry: dict(cell_type, degree, n, alpha, seed).  Cell counts are
    log-uniform in [lo, hi]; type triangle/tetrahedron with probability 1/2;
    degree uniform in 1..6 (triangles) or 1..5 (tetrahedra); grid size from
    the target count (tri: n = round(sqrt(t/2)), tet: n = round((t/6)^(1/3))).
    """
    rng = np.random.default_rng(seed)
    out = []
    for m in range(n_meshes):
        target = math.exp(rng.uniform(math.log(lo), math.log(hi)))
        is_tet = bool(rng.integers(0, 2))
        if is_tet:
            deg = int(rng.integers(1, 6))
            n = max(1, int(round((target / 6.0) ** (1.0 / 3.0))))
            out.append(dict(cell_type="tetrahedron", degree=deg, n=n, alpha=0.15, seed=1000 + m))
        else:
            deg = int(rng.integers(1, 7))
            n = max(1, int(round(math.sqrt(target / 2.0))))
            out.append(dict(cell_type="triangle", degree=deg, n=n, alpha=0.2, seed=1000 + m))
    return out
