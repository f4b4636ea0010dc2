"""FP64 CPU oracle for batched finite-element cell kernels and global assembly.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library (``paper_2410_12614_gb300``) and never calls it.

Contents and the passages they follow (Croci & Wells, "Mixed-precision finite
element kernels and assembly"):

* ``gauss_jacobi`` / ``collapsed_rule`` -- quadrature exact to degree 2m-1 on
  the reference simplex by the collapsed (Duffy) conical product of
  Gauss-Jacobi rules; the paper only requires exact rules (Sec. 3.1 footnote)
  and states 2p-exact rules for the workloads.  Nodes and weights come from
  the Golub-Welsch eigenproblem of the Jacobi matrix (numpy ``eigh``).
* ``strang_fix_3`` -- the 3-point degree-2 triangle rule with interior points.
* ``lattice_nodes`` / ``tabulate`` -- degree-p Lagrange basis on equispaced
  lattice nodes, evaluated in the product form of Appendix A (Nicolaides'
  representation phi_a = prod_i prod_{j<a_i} (p lambda_i - j)/(j+1)) and
  differentiated by the product rule (Appendix A, derivative formula).
* C routines in ``fe_oracle.c``: geometry by LU (Sec. 4.2), element matrices
  by the literal quadrature sum (Sec. 3.1), canonical dof map, CSR pattern,
  assembly A^g = L D L^T (Sec. 3.3), kappa_q^A (Corollary 4.10), adjoint.
* ``Problem.action`` / ``assemble_vector`` -- Algorithm 2 (the action of a
  form on a known FE function, b = sum_s B_s r_s) and v^g = L b (Sec. 3.3).
* ``Problem.gather_values`` / ``adjoint_stiffness_values`` -- the transpose of
  the assembly and dL/dkappa for L = sum_e g_e A^g_e (calculus on Sec. 3.1).
* ``error_bound`` / ``subnormal_term`` -- the per-cell bound of Theorem 4.8 /
  Corollary 4.10 in the form used by the tests, written out to all orders
  with the gradual-underflow terms of narrow formats (see their docstrings).

Everything is FP64; nothing is tuned.
"""
from __future__ import annotations

import ctypes
import itertools
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "libfe_oracle.so")
_SRC = os.path.join(_HERE, "fe_oracle.c")
_lock = threading.Lock()
_lib = None

# Unit roundoffs (Table 1 of the paper; e4m3 and tf32 added).
UNIT_ROUNDOFF = {
    "fp64": 2.0 ** -53,
    "fp32": 2.0 ** -24,
    "tf32": 2.0 ** -11,
    "fp16": 2.0 ** -11,
    "bf16": 2.0 ** -8,
    "e4m3": 2.0 ** -4,
}


def build(force: bool = False) -> str:
    """Compile fe_oracle.c with gcc (no fast-math)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
            i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
            f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
            c_int, c_i64 = ctypes.c_int, ctypes.c_int64
            lib.fo_geometry.argtypes = [c_int, f64p, f64p, f64p, f64p]
            lib.fo_mesh_geometry.argtypes = [c_int, c_i64, i32p, f64p, f64p, ctypes.c_void_p]
            lib.fo_element_matrices.argtypes = [c_int, c_i64, c_i64, i32p, f64p, c_int, c_int, f64p, f64p,
                                                f64p, f64p, c_int, f64p]
            lib.fo_kappa_q.argtypes = [c_int, c_i64, c_i64, i32p, f64p, c_int, c_int, f64p, f64p, f64p,
                                       f64p, c_int, f64p, f64p]
            lib.fo_dofmap.argtypes = [c_int, c_int, i32p, c_i64, c_i64, i32p, i32p, ctypes.POINTER(c_i64)]
            lib.fo_csr_pattern.argtypes = [c_i64, c_i64, c_int, i32p, i64p, ctypes.c_void_p]
            lib.fo_assemble.argtypes = [c_i64, c_int, i32p, f64p, i64p, i32p, c_i64, c_int, f64p]
            lib.fo_adjoint_stiffness.argtypes = [c_int, c_i64, i32p, f64p, c_i64, c_int, c_int, f64p, f64p,
                                                 f64p, i32p, f64p, f64p, ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.POINTER(ctypes.c_double)]
            lib.fo_element_matrices_box.argtypes = [c_int, c_i64, c_i64, i32p, f64p, c_int, c_int, f64p, f64p,
                                                    f64p, f64p, f64p, c_int, f64p]
            lib.fo_kappa_q_box.argtypes = [c_int, c_i64, c_i64, i32p, f64p, c_int, c_int, f64p, f64p, f64p,
                                           f64p, f64p, c_int, f64p, f64p]
            lib.fo_dofmap_weights.argtypes = [c_int, c_int, i32p, c_i64, c_i64, i32p, i32p, ctypes.POINTER(c_i64)]
            for f in ("fo_geometry", "fo_mesh_geometry", "fo_element_matrices", "fo_kappa_q", "fo_dofmap",
                      "fo_csr_pattern", "fo_assemble", "fo_adjoint_stiffness", "fo_element_matrices_box",
                      "fo_kappa_q_box", "fo_dofmap_weights"):
                getattr(lib, f).restype = c_int
            _lib = lib
    return _lib


def _check(status, what):
    if status != 0:
        raise RuntimeError(f"oracle {what} failed with status {status}")


def _dim(cell_type):
    if cell_type in ("triangle", "tri", 2, "quadrilateral", "quad"):
        return 2
    if cell_type in ("tetrahedron", "tet", 3, "hexahedron", "hex"):
        return 3
    raise ValueError(cell_type)


def is_boxed(cell_type) -> bool:
    return cell_type in ("quadrilateral", "quad", "hexahedron", "hex")


# --------------------------------------------------------------------------
# Quadrature
# --------------------------------------------------------------------------
def gauss_jacobi(m: int, alpha: int):
    """m-point Gauss rule on [0, 1] for the weight (1 - t)^alpha.

    Golub-Welsch: the nodes are the eigenvalues of the symmetric Jacobi matrix
    of the monic Jacobi polynomials P^(alpha, 0) on [-1, 1]; the weights are
    mu_0 times the squared first components of the normalised eigenvectors,
    mu_0 = int_{-1}^{1} (1 - x)^alpha dx = 2^(alpha+1)/(alpha+1).  The map
    t = (1 + x)/2 turns (1-x)^alpha dx into 2^(alpha+1) (1-t)^alpha dt.
    Returns (nodes ascending, weights).
    """
    a, b = float(alpha), 0.0
    diag = np.empty(m)
    off = np.empty(max(m - 1, 0))
    for n in range(m):
        s = 2 * n + a + b
        diag[n] = (b - a) / (a + b + 2) if s == 0 else (b * b - a * a) / (s * (s + 2))
    for n in range(1, m):
        s = 2 * n + a + b
        off[n - 1] = math.sqrt(4 * n * (n + a) * (n + b) * (n + a + b) / (s * s * (s + 1) * (s - 1)))
    T = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
    x, V = np.linalg.eigh(T)
    mu0 = 2.0 ** (a + 1) / (a + 1)
    wx = mu0 * V[0, :] ** 2
    t = (1.0 + x) / 2.0
    wt = wx / 2.0 ** (a + 1)
    return t, wt


def collapsed_rule(cell_type, m: int):
    """Collapsed conical product rule, exact to degree 2m-1, n_q = m^d.

    Triangle: x = a (1 - b), y = b; Jacobian (1 - b).
    Tetrahedron: x = a (1-b)(1-c), y = b (1-c), z = c; Jacobian (1-b)(1-c)^2.
    Point order: q = ia + m (ib + m ic) (the first collapsed coordinate runs
    fastest), 1-D nodes ascending.  Returns (points [n_q, d], weights [n_q]).
    """
    d = _dim(cell_type)
    ta, wa = gauss_jacobi(m, 0)
    tb, wb = gauss_jacobi(m, 1)
    pts, wts = [], []
    if d == 2:
        for ib in range(m):
            for ia in range(m):
                a, b = ta[ia], tb[ib]
                pts.append((a * (1 - b), b))
                wts.append(wa[ia] * wb[ib])
    else:
        tc, wc = gauss_jacobi(m, 2)
        for ic in range(m):
            for ib in range(m):
                for ia in range(m):
                    a, b, c = ta[ia], tb[ib], tc[ic]
                    pts.append((a * (1 - b) * (1 - c), b * (1 - c), c))
                    wts.append(wa[ia] * wb[ib] * wc[ic])
    return np.array(pts, dtype=np.float64), np.array(wts, dtype=np.float64)


def strang_fix_3():
    """3-point, degree-2 triangle rule with interior points (1/6,1/6),
    (2/3,1/6), (1/6,2/3), each of weight 1/6 (reference area 1/2)."""
    pts = np.array([[1 / 6, 1 / 6], [2 / 3, 1 / 6], [1 / 6, 2 / 3]], dtype=np.float64)
    wts = np.full(3, 1 / 6, dtype=np.float64)
    return pts, wts


def tensor_rule(cell_type, m: int):
    """Tensor-product Gauss-Legendre rule on the unit square / cube [0, 1]^d
    (the boxed reference cells of Sec. 5.1): m points per direction, exact to
    degree 2m-1 in each variable, n_q = m^d, point q = ia + m (ib + m ic) (x
    fastest), 1-D nodes ascending; the 1-D rule is gauss_jacobi(m, 0)."""
    d = _dim(cell_type)
    t, w = gauss_jacobi(m, 0)
    pts, wts = [], []
    for idx in itertools.product(range(m), repeat=d):
        i = idx[::-1]                        # x fastest
        pts.append([t[a] for a in i])
        wts.append(float(np.prod([w[a] for a in i])))
    return np.array(pts, dtype=np.float64), np.array(wts, dtype=np.float64)


def rule_for_degree(cell_type, p: int):
    """2p-exact rule with m = p + 1 points per direction: the collapsed rule on
    simplices, the tensor Gauss-Legendre rule on boxed cells."""
    if is_boxed(cell_type):
        return tensor_rule(cell_type, p + 1)
    return collapsed_rule(cell_type, p + 1)


# --------------------------------------------------------------------------
# Lagrange basis on equispaced lattice nodes (Appendix A, product form)
# --------------------------------------------------------------------------
def lattice_nodes(d: int, p: int) -> np.ndarray:
    """Barycentric multi-indices a in N^(d+1), |a| = p, in local order.

    Order: support size, then the support's vertex tuple (lexicographic),
    then a in descending lexicographic order.  Vertices come first in cell
    vertex order, then edges 01,02,(03),12,(13),(23), faces, interior.
    """
    idx = [a for a in itertools.product(range(p + 1), repeat=d + 1) if sum(a) == p]

    def key(a):
        sup = tuple(i for i in range(d + 1) if a[i] > 0)
        return (len(sup), sup, tuple(-x for x in a))

    idx.sort(key=key)
    return np.array(idx, dtype=np.int32)


def node_points(d: int, p: int) -> np.ndarray:
    """Reference coordinates X_a = (a_1, ..., a_d) / p of the lattice nodes."""
    a = lattice_nodes(d, p)
    return a[:, 1:].astype(np.float64) / p


def _barycentric(points):
    X = np.asarray(points, dtype=np.float64)
    lam = np.empty((X.shape[0], X.shape[1] + 1))
    lam[:, 0] = 1.0 - X.sum(axis=1)
    lam[:, 1:] = X
    return lam


def tabulate(d: int, p: int, points):
    """phi [n_phi, n_q] and dphi [d, n_phi, n_q] at the given reference points.

    phi_a(lambda) = prod_i prod_{j=0}^{a_i - 1} (p lambda_i - j) / (j + 1).
    d phi_a / d lambda_i by the product rule over the factors of index i;
    d lambda_0 / d X_s = -1 and d lambda_i / d X_s = delta_is.
    """
    nodes = lattice_nodes(d, p)
    lam = _barycentric(points)
    n_q = lam.shape[0]
    n_phi = nodes.shape[0]
    phi = np.zeros((n_phi, n_q))
    dphi = np.zeros((d, n_phi, n_q))
    for k, a in enumerate(nodes):
        for q in range(n_q):
            # factors f[i][j] = (p lam_i - j)/(j+1), j < a_i
            fac = []
            for i in range(d + 1):
                for j in range(a[i]):
                    fac.append((i, (p * lam[q, i] - j) / (j + 1), p / (j + 1)))
            val = 1.0
            for _, f, _ in fac:
                val *= f
            phi[k, q] = val
            dlam = np.zeros(d + 1)
            for r, (i, _, df) in enumerate(fac):
                prod = df
                for r2, (_, f2, _) in enumerate(fac):
                    if r2 != r:
                        prod *= f2
                dlam[i] += prod
            for s in range(d):
                dphi[s, k, q] = dlam[s + 1] - dlam[0]
    return phi, dphi


def n_phi(d: int, p: int) -> int:
    return math.comb(p + d, d)


# --------------------------------------------------------------------------
# Q_p Lagrange basis on boxed cells (Sec. 3.1, boxed cells; Appendix A, the
# product representation of tensor-product Lagrange polynomials)
# --------------------------------------------------------------------------
def box_nodes(d: int, p: int) -> np.ndarray:
    """Lattice indices a in {0..p}^d of the equispaced nodes X_a = a / p, in
    lexicographic order with the x index fastest: node k = a_0 + (p+1)(a_1 +
    (p+1) a_2).  Cell vertex v of a boxed cell is the corner with coordinates
    (bit_0(v), bit_1(v), bit_2(v))."""
    out = []
    for idx in itertools.product(range(p + 1), repeat=d):
        out.append(idx[::-1])
    return np.array(out, dtype=np.int32)


def box_node_weights(d: int, p: int) -> np.ndarray:
    """[n_phi, 2^d]: the Q1 (multilinear) coordinates of each node times p^d,
    w_v = prod_i (a_i if bit_i(v) else p - a_i): the node's weights over the
    cell's vertices, from which the canonical dof key is formed."""
    a = box_nodes(d, p)
    nv = 1 << d
    W = np.ones((a.shape[0], nv), dtype=np.int64)
    for v in range(nv):
        for i in range(d):
            W[:, v] *= np.where((v >> i) & 1, a[:, i], p - a[:, i])
    return W.astype(np.int32)


def tabulate_box(d: int, p: int, points):
    """phi [n_phi, n_q] and dphi [d, n_phi, n_q] of the Q_p basis at reference
    points: phi_a(X) = prod_i l_{a_i}(X_i) with the 1-D equispaced Lagrange
    factors l_j(t) = prod_{m != j} (p t - m) / (j - m) (a product of first-degree
    monomials, Appendix A), derivatives by the product rule."""
    X = np.asarray(points, dtype=np.float64)
    n_q = X.shape[0]
    nodes = box_nodes(d, p)

    def lag(j, t):
        v = np.ones_like(t)
        for m in range(p + 1):
            if m != j:
                v = v * (p * t - m) / (j - m)
        return v

    def dlag(j, t):
        tot = np.zeros_like(t)
        for r in range(p + 1):
            if r == j:
                continue
            term = np.full_like(t, p / (j - r))
            for m in range(p + 1):
                if m != j and m != r:
                    term = term * (p * t - m) / (j - m)
            tot = tot + term
        return tot

    phi = np.zeros((nodes.shape[0], n_q))
    dphi = np.zeros((d, nodes.shape[0], n_q))
    for k, a in enumerate(nodes):
        f = [lag(a[i], X[:, i]) for i in range(d)]
        df = [dlag(a[i], X[:, i]) for i in range(d)]
        phi[k] = np.prod(f, axis=0)
        for s in range(d):
            dphi[s, k] = np.prod([df[i] if i == s else f[i] for i in range(d)], axis=0)
    return phi, dphi


# --------------------------------------------------------------------------
# Mesh-level routines (C)
# --------------------------------------------------------------------------
def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def geometry(xv):
    """J, det J, J^{-1} of one simplex from its (d+1) x d vertex array."""
    xv = _c(xv, np.float64)
    d = xv.shape[1]
    J = np.zeros(d * d)
    det = np.zeros(1)
    Jinv = np.zeros(d * d)
    _check(_load().fo_geometry(d, xv.ravel(), J, det, Jinv), "geometry")
    return J.reshape(d, d), float(det[0]), Jinv.reshape(d, d)


def mesh_geometry(vertices, cells, with_G: bool = True):
    vertices, cells = _c(vertices, np.float64), _c(cells, np.int32)
    d = vertices.shape[1]
    nc = cells.shape[0]
    det = np.zeros(nc)
    G = np.zeros((nc, d, d)) if with_G else None
    _check(_load().fo_mesh_geometry(d, nc, cells, vertices, det,
                                    G.ctypes.data if with_G else None), "mesh_geometry")
    return det, G


class Problem:
    """A mesh + degree + quadrature rule with the reference tabulation."""

    def __init__(self, vertices, cells, p: int, points, weights):
        self.vertices = _c(vertices, np.float64)
        self.cells = _c(cells, np.int32)
        self.d = self.vertices.shape[1]
        self.p = int(p)
        self.points = _c(points, np.float64)
        self.weights = _c(weights, np.float64)
        self.n_q = self.weights.shape[0]
        self.n_cells = self.cells.shape[0]
        # boxed cells (quadrilaterals, hexahedra) have 2^d vertices in tensor order
        self.boxed = self.cells.shape[1] == (1 << self.d)
        if self.boxed:
            self.n_phi = (self.p + 1) ** self.d
            self.phi, self.dphi = tabulate_box(self.d, self.p, self.points)
            _, dpsi = tabulate_box(self.d, 1, self.points)        # Q1 map derivatives [d][2^d][n_q]
            self.dpsi = _c(dpsi, np.float64)
        else:
            self.n_phi = n_phi(self.d, self.p)
            self.phi, self.dphi = tabulate(self.d, self.p, self.points)
        self.phi = _c(self.phi, np.float64)
        self.dphi = _c(self.dphi, np.float64)
        self._dofs = None
        self._pattern = None

    # element matrices --------------------------------------------------
    def element_matrices(self, kappa, form: str, c0: int = 0, c1: int | None = None):
        """A [n_cells, n_phi, n_phi] (rows outside [c0, c1) are left zero)."""
        c1 = self.n_cells if c1 is None else c1
        kappa = _c(kappa, np.float64).reshape(self.n_cells, self.n_q)
        A = np.zeros((self.n_cells, self.n_phi, self.n_phi))
        f = {"mass": 1, "stiffness": 2}[form]
        if self.boxed:
            _check(_load().fo_element_matrices_box(self.d, c0, c1, self.cells, self.vertices, self.n_phi, self.n_q,
                                                   self.weights, self.phi, self.dphi, self.dpsi, kappa.ravel(), f,
                                                   A.reshape(-1)), "element_matrices_box")
            return A
        _check(_load().fo_element_matrices(self.d, c0, c1, self.cells, self.vertices, self.n_phi, self.n_q,
                                           self.weights, self.phi, self.dphi, kappa.ravel(), f, A.reshape(-1)),
               "element_matrices")
        return A

    def element_matrices_subset(self, kappa, form: str, cell_ids):
        """Element matrices of the listed cells only, [len(cell_ids), n_phi, n_phi]."""
        cell_ids = np.asarray(cell_ids, dtype=np.int64)
        sub = Problem.__new__(Problem)
        sub.__dict__.update(self.__dict__)
        sub.cells = _c(self.cells[cell_ids], np.int32)
        sub.n_cells = len(cell_ids)
        kap = _c(np.asarray(kappa).reshape(self.n_cells, self.n_q)[cell_ids], np.float64)
        return Problem.element_matrices(sub, kap, form)

    def kappa_q(self, kappa, form: str, A, cell_ids=None):
        """Per-cell kappa_q^A (Corollary 4.10) for the given exact matrices."""
        kappa = _c(kappa, np.float64).reshape(-1, self.n_q)
        cells = self.cells if cell_ids is None else _c(self.cells[np.asarray(cell_ids)], np.int32)
        if cell_ids is not None:
            kappa = _c(kappa[np.asarray(cell_ids)], np.float64)
        nc = cells.shape[0]
        kq = np.zeros(nc)
        f = {"mass": 1, "stiffness": 2}[form]
        if self.boxed:
            _check(_load().fo_kappa_q_box(self.d, 0, nc, cells, self.vertices, self.n_phi, self.n_q, self.weights,
                                          self.phi, self.dphi, self.dpsi, kappa.ravel(), f,
                                          _c(A, np.float64).reshape(-1), kq), "kappa_q_box")
            return kq
        _check(_load().fo_kappa_q(self.d, 0, nc, cells, self.vertices, self.n_phi, self.n_q, self.weights,
                                  self.phi, self.dphi, kappa.ravel(), f, _c(A, np.float64).reshape(-1), kq),
               "kappa_q")
        return kq

    def point_geometry(self, cell_ids=None):
        """Boxed cells: |det J_q| [nc, n_q] and G_q = |det J_q| J_q^-1 J_q^-T
        [nc, n_q, d, d] at every quadrature point (numpy det / inv of
        J_q = sum_v x_v grad psi_v(X_q)^T; bound arithmetic only)."""
        cells = self.cells if cell_ids is None else self.cells[np.asarray(cell_ids)]
        x = self.vertices[cells]                                        # [nc, nv, d]
        J = np.einsum("cvi,jvq->cqij", x, self.dpsi)
        det = np.linalg.det(J)
        Ji = np.linalg.inv(J)
        G = np.abs(det)[:, :, None, None] * np.einsum("cqik,cqjk->cqij", Ji, Ji)
        return np.abs(det), G

    # dof map / pattern ----------------------------------------------------
    def cell_dofs(self):
        if self._dofs is None and self.boxed:
            W = _c(box_node_weights(self.d, self.p), np.int32)
            dofs = np.zeros((self.n_cells, self.n_phi), dtype=np.int32)
            nd = ctypes.c_int64(0)
            _check(_load().fo_dofmap_weights(1 << self.d, self.n_phi, W.ravel(), self.vertices.shape[0],
                                             self.n_cells, self.cells, dofs.reshape(-1), ctypes.byref(nd)),
                   "dofmap_weights")
            self._dofs = (dofs, int(nd.value))
        if self._dofs is None:
            nodes = _c(lattice_nodes(self.d, self.p), np.int32)
            dofs = np.zeros((self.n_cells, self.n_phi), dtype=np.int32)
            nd = ctypes.c_int64(0)
            _check(_load().fo_dofmap(self.d, self.n_phi, nodes.ravel(), self.vertices.shape[0], self.n_cells,
                                     self.cells, dofs.reshape(-1), ctypes.byref(nd)), "dofmap")
            self._dofs = (dofs, int(nd.value))
        return self._dofs

    @property
    def n_dofs(self):
        return self.cell_dofs()[1]

    def csr_pattern(self):
        if self._pattern is None:
            dofs, nd = self.cell_dofs()
            row_ptr = np.zeros(nd + 1, dtype=np.int64)
            lib = _load()
            _check(lib.fo_csr_pattern(nd, self.n_cells, self.n_phi, dofs.reshape(-1), row_ptr, None), "pattern")
            col = np.zeros(int(row_ptr[-1]), dtype=np.int32)
            _check(lib.fo_csr_pattern(nd, self.n_cells, self.n_phi, dofs.reshape(-1), row_ptr, col.ctypes.data),
                   "pattern")
            self._pattern = (row_ptr, col)
        return self._pattern

    def assemble(self, A, absval: bool = False):
        dofs, nd = self.cell_dofs()
        row_ptr, col = self.csr_pattern()
        vals = np.zeros(col.shape[0])
        _check(_load().fo_assemble(self.n_cells, self.n_phi, dofs.reshape(-1), _c(A, np.float64).reshape(-1),
                                   row_ptr, col, col.shape[0], int(absval), vals), "assemble")
        return vals

    def assemble_subset(self, A_subset, cell_ids, absval: bool = False):
        """Assemble only the listed cells' element matrices into the full pattern."""
        dofs, nd = self.cell_dofs()
        row_ptr, col = self.csr_pattern()
        sub = _c(dofs[np.asarray(cell_ids)], np.int32)
        vals = np.zeros(col.shape[0])
        _check(_load().fo_assemble(sub.shape[0], self.n_phi, sub.reshape(-1), _c(A_subset, np.float64).reshape(-1),
                                   row_ptr, col, col.shape[0], int(absval), vals), "assemble_subset")
        return vals

    def dof_points(self):
        """Physical coordinates of every global dof (from the cell that first lists it)."""
        dofs, nd = self.cell_dofs()
        if self.boxed:
            lam = box_node_weights(self.d, self.p).astype(np.float64) / float(self.p) ** self.d
        else:
            lam = _barycentric(node_points(self.d, self.p))
        pts = np.full((nd, self.d), np.nan)
        xv = self.vertices[self.cells]  # [nc, nv, d]
        phys = np.einsum("kv,cvi->cki", lam, xv)
        pts[dofs.reshape(-1)] = phys.reshape(-1, self.d)
        return pts

    # adjoint --------------------------------------------------------------
    def adjoint_stiffness(self, kappa, u, v, vertices=None, want_kappa=True, want_x=True):
        dofs, nd = self.cell_dofs()
        verts = self.vertices if vertices is None else _c(vertices, np.float64)
        kappa = _c(kappa, np.float64).reshape(self.n_cells, self.n_q)
        gk = np.zeros((self.n_cells, self.n_q)) if want_kappa else None
        gx = np.zeros_like(verts) if want_x else None
        L = ctypes.c_double(0.0)
        _check(_load().fo_adjoint_stiffness(self.d, self.n_cells, self.cells, verts, verts.shape[0], self.n_phi,
                                            self.n_q, self.weights, self.dphi, kappa.ravel(), dofs.reshape(-1),
                                            _c(u, np.float64), _c(v, np.float64),
                                            gk.ctypes.data if want_kappa else None,
                                            gx.ctypes.data if want_x else None, ctypes.byref(L)), "adjoint")
        return float(L.value), gk, gx

    # adjoint for a general gradient on the CSR values ---------------------------
    def gather_values(self, g):
        """G^c [n_cells, n_phi, n_phi] with G^c_kl = g at the CSR slot of
        (dof(c, k), dof(c, l)): the transpose of the assembly A^g = L D L^T
        (Sec. 3.3), so that sum_e g_e A^g_e = sum_c sum_kl G^c_kl A^c_kl."""
        dofs, nd = self.cell_dofs()
        row_ptr, col = self.csr_pattern()
        rows = np.repeat(np.arange(nd, dtype=np.int64), np.diff(row_ptr))
        keys = rows * nd + col.astype(np.int64)                  # increasing along the CSR order
        q = dofs[:, :, None].astype(np.int64) * nd + dofs[:, None, :].astype(np.int64)
        slot = np.searchsorted(keys, q.ravel()).reshape(q.shape)
        assert np.array_equal(keys[slot], q), "entry outside the pattern"
        return np.asarray(g, np.float64)[slot]

    def adjoint_stiffness_values(self, kappa, g):
        """L = sum_e g_e A^g_e for the stiffness form and a given gradient g on
        the CSR values, and dL/dkappa_cq = sum_kl G^c_kl dA^c_kl/dkappa_cq with
        dA^c_kl/dkappa_cq = w_q grad phi_l(X_q)^T G grad phi_k(X_q) (the element
        matrix definition, Sec. 3.1; G = |det J| J^-1 J^-T).  A^c is linear in
        kappa, so L = sum_cq kappa_cq dL/dkappa_cq."""
        kappa = np.asarray(kappa, np.float64).reshape(self.n_cells, self.n_q)
        Gc = self.gather_values(g)
        det, G = mesh_geometry(self.vertices, self.cells)
        # grad phi_l^T G grad phi_k at every point, contracted with G^c_kl
        gk = self.weights[None, :] * np.einsum("ckl,slq,cst,tkq->cq", Gc, self.dphi, G, self.dphi, optimize=True)
        return float(np.sum(kappa * gk)), gk

    # linear forms: the action of a form on a known FE function (Algorithm 2) --
    def action(self, kappa, w, form: str, with_magnitude: bool = False):
        """Per-cell vectors b [n_cells, n_phi] of v_j = a_K(w, phi_j) (Sec. 3.1) for
        the FE function with global coefficients w, by Algorithm 2 in FP64:
        r_s = vstack_q(w_q z(X_q) (G grad w)_s(X_q)) (Poisson; mass: w_q z |det J| w(X_q)),
        b = sum_s B_s r_s, with grad w(X_q) = sum_k w_k B_skq the reference gradient.
        with_magnitude: also sum_{s,q} |B_skq| sum_t |w_q z G_st| sum_j |B_tjq| |w_j|,
        the magnitude a componentwise rounding bound scales with."""
        dofs, nd = self.cell_dofs()
        kappa = np.asarray(kappa, np.float64).reshape(self.n_cells, self.n_q)
        wc = np.asarray(w, np.float64)[dofs]                                 # [nc, n_phi]
        det, G = mesh_geometry(self.vertices, self.cells)                    # G = |det J| J^-1 J^-T
        wk = self.weights[None, :] * kappa                                   # w_q z(X_q)
        if form == "mass":
            val = np.einsum("ck,kq->cq", wc, self.phi)                      # w(X_q)
            r = wk * np.abs(det)[:, None] * val
            b = np.einsum("kq,cq->ck", self.phi, r)
            if not with_magnitude:
                return b
            mr = wk * np.abs(det)[:, None] * np.einsum("ck,kq->cq", np.abs(wc), np.abs(self.phi))
            return b, np.einsum("kq,cq->ck", np.abs(self.phi), mr)
        gw = np.einsum("ck,skq->csq", wc, self.dphi)                        # reference gradient of w
        r = wk[:, None, :] * np.einsum("cst,ctq->csq", G, gw)
        b = np.einsum("skq,csq->ck", self.dphi, r)
        if not with_magnitude:
            return b
        agw = np.einsum("ck,skq->csq", np.abs(wc), np.abs(self.dphi))
        mr = wk[:, None, :] * np.einsum("cst,ctq->csq", np.abs(G), agw)
        return b, np.einsum("skq,csq->ck", np.abs(self.dphi), mr)

    def assemble_vector(self, b):
        """v^g = L b (Sec. 3.3): each cell vector added into its dofs."""
        dofs, nd = self.cell_dofs()
        v = np.zeros(nd)
        np.add.at(v, dofs.reshape(-1), np.asarray(b, np.float64).reshape(-1))
        return v

    def with_vertices(self, vertices):
        other = Problem.__new__(Problem)
        other.__dict__.update(self.__dict__)
        other.vertices = _c(vertices, np.float64)
        return other


# --------------------------------------------------------------------------
# Error bounds (Theorem 4.8 / Corollary 4.10, Corollary 4.11)
# --------------------------------------------------------------------------
def error_bound(kq, u_s: float, K: int, u_acc: float = 2.0 ** -23, u_out: float = 2.0 ** -24,
                storage_roundings: int = 2, u_pre: float = 0.0, abs_rel=0.0):
    """Per-cell relative max-norm bound for a reduced-precision contraction.

        err_c <= rho kappa_q^A(c) + gamma_K(2 u_acc) (1 + rho) kappa_q^A(c) + u_out + abs_rel(c),
        rho    = (1 + u_s)^r (1 + u_pre) - 1.

    Derivation (Theorem 4.8 / Corollary 4.10 with u_g = u_p ~ 0, FP64
    geometry and tabulation, written out to all orders): every product of the
    contraction is fl(C_i) fl(P_i) with fl(x) = x (1 + delta) + eta, |delta| <=
    u_s for a normal result and |eta| <= half the subnormal spacing otherwise
    (only one of the two is nonzero).  For normal operands a product then
    carries the relative error (1 + u_s)^2 - 1 = 2 u_s + u_s^2 (r = 2: C and
    the tabulated operand; the u_s^2 term matters for e4m3, u_s = 2^-4).
    u_pre is the relative error C already carries before its storage rounding
    (a coefficient window and a geometry factor formed in FP32).  The products'
    sum over K terms in FP32 adds gamma_K(2 u_acc) times the sum of the rounded
    products' magnitudes (<= (1 + rho) sum |C||P|), the accumulation roundoff
    doubled to allow truncating accumulation; u_out is the FP32 store.
    sum_i |C_i||P_i| over the folded pairs is at most sum_st |B_s||C_st||B_t|^T,
    the numerator of kappa_q^A, so each term is relative to ||A^c||_max through
    kappa_q^A(c).  abs_rel(c) (see subnormal_term) carries the eta terms of
    operands that fall into gradual underflow, relative to ||A^c||_max.
    """
    x = K * 2.0 * u_acc
    gamma = x / (1.0 - x)
    rho = (1.0 + u_s) ** storage_roundings * (1.0 + u_pre) - 1.0
    kq = np.asarray(kq)
    return rho * kq + gamma * (1.0 + rho) * kq + u_out + np.asarray(abs_rel)


def operand_magnitudes(problem, form: str):
    """Plan-level magnitudes of the tabulated operand (Sec. 3.1, B_s = the
    reference derivatives, mass: the basis values):
    Pi_max = max_kl sum_q (sum_s |B_skq|)(sum_t |B_tlq|), which bounds
    sum over the folded pairs (s <= t) and points of |B_skq B_tlq + [s != t] B_tkq B_slq|,
    and Bmax = max |B_skq|, so that every folded entry is at most
    n_f Bmax^2 (n_f = 2 for the stiffness form, 1 for the mass form)."""
    B = problem.dphi if form == "stiffness" else problem.phi[None]
    b = np.abs(B).sum(axis=0)                        # [n_phi, n_q]: sum_s |B_skq|
    return float((b @ b.T).max()), float(np.abs(B).max())


def subnormal_term(problem, kappa, form: str, A, mbits: int, emin: int, target: int, cell_ids=None):
    """abs_rel(c) of error_bound for a storage format with `mbits` explicit
    mantissa bits and smallest normal exponent `emin`, whose operands are
    brought by powers of two to the binade [2^(target-1), 2^target) (per cell
    for C: max_q|w_q kappa_cq| max_st|G_st|, mass |det J|; once for the
    tabulated operand: its largest entry; target = 1: no scaling).

    A value rounded in gradual underflow has absolute error at most
    h = 2^(emin - mbits - 1) in scaled units.  The scale 2^e puts the scale's
    magnitude M (computed by the kernels in FP32) in [2^(target-1), 2^target),
    so 2^-e <= M 2^(1 - target) up to that FP32 rounding; with a factor two to
    spare, unscaled a_C = h 2^(2 - target) M_c for C (M_c the exact magnitude;
    without scaling a_C = h) and a_P = h 2^(2 - target) n_f Bmax^2 for the
    operand.
    Per entry (k, l) the eta terms add at most
    (1 + u_s) (a_C Pi_kl + a_P sum_i |C_i|) + K a_C a_P; their maximum over
    (k, l), divided by ||A^c||_max, is returned per cell (A: the exact element
    matrices of the cells, in the order of cell_ids)."""
    kappa = np.asarray(kappa, np.float64).reshape(-1, problem.n_q)
    cells = problem.cells if cell_ids is None else problem.cells[np.asarray(cell_ids)]
    if cell_ids is not None:
        kappa = kappa[np.asarray(cell_ids)]
    wk = np.abs(problem.weights[None, :] * kappa)                        # |w_q kappa_cq|
    d = problem.d
    if getattr(problem, "boxed", False):
        # geometry at every point: C_(st),q = w_q kappa_cq G_st(X_q)
        adet, Gq = problem.point_geometry(cell_ids)
        if form == "stiffness":
            Cs = np.stack([np.abs(Gq[:, :, s, t]) for s in range(d) for t in range(s, d)], axis=2) * wk[:, :, None]
            K = problem.n_q * d * (d + 1) // 2
            n_f = 2.0
        else:
            Cs = (adet * wk)[:, :, None]
            K = problem.n_q
            n_f = 1.0
        M = Cs.reshape(len(Cs), -1).max(axis=1)
        SC = Cs.reshape(len(Cs), -1).sum(axis=1)
        pi_max, bmax = operand_magnitudes(problem, form)
        h = 2.0 ** (emin - mbits - 1)
        a_C = h * 2.0 ** (2 - target) * M if target > 1 else np.full_like(M, h)
        a_P = h * 2.0 ** (2 - target) * n_f * bmax ** 2 if target > 1 else h
        u_s = 2.0 ** -(mbits + 1)
        S = (1.0 + u_s) * (a_C * pi_max + a_P * SC) + K * a_C * a_P
        amax = np.abs(np.asarray(A)).reshape(len(M), -1).max(axis=1)
        return S / amax
    det, G = mesh_geometry(problem.vertices, cells)
    if form == "stiffness":
        Gs = np.stack([np.abs(G[:, s, t]) for s in range(d) for t in range(s, d)], axis=1)
        M = wk.max(axis=1) * Gs.max(axis=1)
        SC = wk.sum(axis=1) * Gs.sum(axis=1)
        K = problem.n_q * d * (d + 1) // 2
        n_f = 2.0
    else:
        M = wk.max(axis=1) * np.abs(det)
        SC = wk.sum(axis=1) * np.abs(det)
        K = problem.n_q
        n_f = 1.0
    pi_max, bmax = operand_magnitudes(problem, form)
    h = 2.0 ** (emin - mbits - 1)
    a_C = h * 2.0 ** (2 - target) * M if target > 1 else np.full_like(M, h)
    a_P = h * 2.0 ** (2 - target) * n_f * bmax ** 2 if target > 1 else h
    u_s = 2.0 ** -(mbits + 1)
    S = (1.0 + u_s) * (a_C * pi_max + a_P * SC) + K * a_C * a_P
    amax = np.abs(np.asarray(A)).reshape(len(M), -1).max(axis=1)
    return S / amax
