"""Pins of the oracle's boxed cells (quadrilaterals, hexahedra; Sec. 3.1):
the tensor Gauss-Legendre rule, the Q_p basis in product form (Appendix A),
the per-point multilinear geometry, the element matrices, kappa_q^A and the
canonical dof map.

* rule: sum of weights 1; exact for x^a y^b z^c up to degree 2m-1 in each
  variable (1 / prod (a_i + 1)), inexact at 2m;
* basis: Kronecker property at the nodes, partition of unity, reproduction
  of every Q_p monomial and of its gradient;
* Q1 on the unit square and cube: the textbook matrices
  (tests/golden/q1_reference_matrices.json);
* an affine parallelepiped: mass sum = |det J| for kappa = 1, zero stiffness
  row sums, the energy identity u^T K v = sum_q w_q |det J| grad f . grad g for
  Q_p polynomials f, g with analytic gradients, agreement with a higher rule;
* a non-affine (jittered) hexahedral mesh: symmetry, zero row sums, the mass
  sum against the volume integral of det J by a separate high-order rule;
* kappa_q^A: an exact-arithmetic (fractions) brute force of Corollary 4.10 on
  a non-affine Q2 quadrilateral with a rational Newton-Cotes tensor rule;
* dof map: n_dofs = (pN+1)^d on structured meshes, one physical point per dof
  from every cell that lists it, distinct points for distinct dofs.
"""
import itertools
import json
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
from paper_2410_12614_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("cell", ["quadrilateral", "hexahedron"])
@pytest.mark.parametrize("m", [1, 2, 3, 5])
def test_tensor_rule_exactness(cell, m):
    pts, w = oracle.tensor_rule(cell, m)
    d = pts.shape[1]
    assert abs(w.sum() - 1.0) < 1e-14
    for a in itertools.product(range(2 * m), repeat=d):
        approx = np.sum(w * np.prod(pts ** np.array(a), axis=1))
        assert abs(approx - 1.0 / np.prod(np.array(a) + 1.0)) < 1e-14
    a = (2 * m,) + (0,) * (d - 1)
    assert abs(np.sum(w * pts[:, 0] ** (2 * m)) - 1.0 / (2 * m + 1)) > 1e-6


@pytest.mark.parametrize("d,p", [(2, 1), (2, 3), (3, 2), (3, 4)])
def test_box_basis_properties(d, p):
    nodes = oracle.box_nodes(d, p).astype(np.float64) / p
    phi, dphi = oracle.tabulate_box(d, p, nodes)
    assert np.allclose(phi, np.eye(len(nodes)), atol=1e-12)
    rng = np.random.default_rng(1)
    X = rng.uniform(0, 1, (50, d))
    phi, dphi = oracle.tabulate_box(d, p, X)
    assert np.allclose(phi.sum(axis=0), 1.0, atol=1e-12)
    assert np.allclose(dphi.sum(axis=1), 0.0, atol=1e-10)
    for a in itertools.product(range(p + 1), repeat=d):
        f_nodes = np.prod(nodes ** np.array(a), axis=1)
        f_pts = np.prod(X ** np.array(a), axis=1)
        assert np.allclose(f_nodes @ phi, f_pts, atol=1e-11)
        for s in range(d):
            da = np.array(a)
            if da[s] == 0:
                g = np.zeros(len(X))
            else:
                e = da.copy()
                e[s] -= 1
                g = da[s] * np.prod(X ** e, axis=1)
            assert np.allclose(f_nodes @ dphi[s], g, atol=1e-9)


def test_q1_unit_square_and_cube_closed_forms():
    with open(os.path.join(GOLDEN, "q1_reference_matrices.json")) as f:
        g = json.load(f)
    v = np.array([[0, 0], [1, 0], [0, 1], [1, 1]], dtype=np.float64)
    pr = oracle.Problem(v, np.array([[0, 1, 2, 3]], dtype=np.int32), 1, *oracle.tensor_rule("quadrilateral", 2))
    one = np.ones((1, pr.n_q))
    assert np.allclose(pr.element_matrices(one, "mass")[0] * 36, g["square_mass_times_36"], atol=1e-13)
    assert np.allclose(pr.element_matrices(one, "stiffness")[0] * 6, g["square_stiffness_times_6"], atol=1e-13)
    v3 = np.array([[(c >> 0) & 1, (c >> 1) & 1, (c >> 2) & 1] for c in range(8)], dtype=np.float64)
    pr3 = oracle.Problem(v3, np.arange(8, dtype=np.int32)[None], 1, *oracle.tensor_rule("hexahedron", 2))
    m1, k1 = np.array(g["cube_1d_mass"]), np.array(g["cube_1d_stiffness"])
    M = np.zeros((8, 8))
    K = np.zeros((8, 8))
    for a in range(8):
        for b in range(8):
            bits = [((a >> i) & 1, (b >> i) & 1) for i in range(3)]
            M[a, b] = np.prod([m1[x, y] for x, y in bits])
            K[a, b] = sum(k1[bits[s]] * np.prod([m1[bits[i]] for i in range(3) if i != s]) for s in range(3))
    one = np.ones((1, pr3.n_q))
    assert np.allclose(pr3.element_matrices(one, "mass")[0], M, atol=1e-14)
    assert np.allclose(pr3.element_matrices(one, "stiffness")[0], K, atol=1e-13)


@pytest.mark.parametrize("d,p", [(2, 2), (2, 4), (3, 1), (3, 3)])
def test_affine_parallelepiped_identities(d, p):
    rng = np.random.default_rng(10 + p)
    J = np.eye(d) + 0.3 * rng.standard_normal((d, d))
    x0 = rng.standard_normal(d)
    corners = np.array([[(c >> i) & 1 for i in range(d)] for c in range(1 << d)], dtype=np.float64)
    v = x0 + corners @ J.T
    cells = np.arange(1 << d, dtype=np.int32)[None]
    pr = oracle.Problem(v, cells, p, *oracle.tensor_rule("hexahedron" if d == 3 else "quadrilateral", p + 1))
    one = np.ones((1, pr.n_q))
    M = pr.element_matrices(one, "mass")[0]
    K = pr.element_matrices(one, "stiffness")[0]
    assert abs(M.sum() - abs(np.linalg.det(J))) < 1e-13
    assert np.abs(K.sum(axis=1)).max() < 1e-11 * np.abs(K).max()
    # energy identity for f = prod X_i^a_i, g = prod X_i^b_i (X the reference coordinates)
    nodes = oracle.box_nodes(d, p).astype(np.float64) / p
    pts, w = pr.points, pr.weights
    Jinv = np.linalg.inv(J)
    kap = np.exp(rng.standard_normal((1, pr.n_q)))
    Kk = pr.element_matrices(kap, "stiffness")[0]
    for a, b in [((1,) * d, (p,) + (0,) * (d - 1)), ((p,) * d, (0,) * (d - 1) + (1,))]:
        def val_grad(e, X):
            e = np.array(e)
            f = np.prod(X ** e, axis=1)
            g = np.zeros((len(X), d))
            for s in range(d):
                if e[s]:
                    ee = e.copy()
                    ee[s] -= 1
                    g[:, s] = e[s] * np.prod(X ** ee, axis=1)
            return f, g
        u, _ = val_grad(a, nodes)
        vv, _ = val_grad(b, nodes)
        _, ga = val_grad(a, pts)
        _, gb = val_grad(b, pts)
        phys_a, phys_b = ga @ Jinv, gb @ Jinv          # grad_x f = J^-T grad_X f
        exact = np.sum(w * kap[0] * abs(np.linalg.det(J)) * np.sum(phys_a * phys_b, axis=1))
        assert abs(u @ Kk @ vv - exact) < 1e-11 * max(1.0, abs(exact))
    # a higher rule gives the same matrices (the integrands are polynomial here)
    pr2 = oracle.Problem(v, cells, p, *oracle.tensor_rule("hexahedron" if d == 3 else "quadrilateral", p + 3))
    assert np.allclose(pr2.element_matrices(np.ones((1, pr2.n_q)), "stiffness")[0], K, atol=1e-12 * np.abs(K).max())


def test_jittered_hex_mesh_invariants():
    v, c = inputs.hex_mesh(3, 0.15, 4)
    p = 2
    pr = oracle.Problem(v, c, p, *oracle.rule_for_degree("hexahedron", p))
    one = np.ones((pr.n_cells, pr.n_q))
    M = pr.element_matrices(one, "mass")
    K = pr.element_matrices(one, "stiffness")
    assert np.allclose(K, np.transpose(K, (0, 2, 1)), atol=0)
    assert np.abs(K.sum(axis=2)).max() < 1e-12 * np.abs(K).max()
    # det J of a trilinear map is of degree <= 2 in each variable: the m = 3 rule
    # integrates it exactly, so the mass sum equals the cell volume from a
    # separate rule (m = 6) applied to det J directly
    X, W = oracle.tensor_rule("hexahedron", 6)
    _, dpsi = oracle.tabulate_box(3, 1, X)
    x = v[c]
    J = np.einsum("cvi,jvq->cqij", x, dpsi)
    vol = np.abs(np.linalg.det(J)) @ W
    assert np.allclose(M.sum(axis=(1, 2)), vol, rtol=1e-13)


def _rational_q2_quad_kappa_q():
    """kappa_q^A of the Q2 stiffness form on one non-affine quadrilateral by
    exact rational arithmetic: vertices (0,0), (2,0), (0,1), (3,2) (corners in
    tensor order), the 2-point rule (1/4, 3/4; weights 1/2) in each direction
    (any rule defines kappa_q^A; this one keeps every value rational),
    kappa = 1.  The result is 1307/917."""
    t = [Fr(1, 4), Fr(3, 4)]
    wt = [Fr(1, 2), Fr(1, 2)]
    corners = [(Fr(0), Fr(0)), (Fr(2), Fr(0)), (Fr(0), Fr(1)), (Fr(3), Fr(2))]
    p = 2

    def lag(j, s):
        v = Fr(1)
        for m in range(p + 1):
            if m != j:
                v *= (p * s - m) / Fr(j - m)
        return v

    def dlag(j, s):
        tot = Fr(0)
        for r in range(p + 1):
            if r == j:
                continue
            term = Fr(p, j - r)
            for m in range(p + 1):
                if m != j and m != r:
                    term *= (p * s - m) / Fr(j - m)
            tot += term
        return tot

    nodes = [(i, j) for j in range(3) for i in range(3)]
    N = [[Fr(0)] * 9 for _ in range(9)]
    A = [[Fr(0)] * 9 for _ in range(9)]
    for qy in range(len(t)):
        for qx in range(len(t)):
            X, Y = t[qx], t[qy]
            w = wt[qx] * wt[qy]
            # J = sum_v x_v grad psi_v, psi = ((1-X)(1-Y), X(1-Y), (1-X)Y, XY)
            dpsi = [(-(1 - Y), -(1 - X)), ((1 - Y), -X), (-Y, (1 - X)), (Y, X)]
            J = [[sum(corners[v][i] * dpsi[v][j] for v in range(4)) for j in range(2)] for i in range(2)]
            det = J[0][0] * J[1][1] - J[0][1] * J[1][0]
            Ji = [[J[1][1] / det, -J[0][1] / det], [-J[1][0] / det, J[0][0] / det]]
            G = [[abs(det) * sum(Ji[i][k] * Ji[j][k] for k in range(2)) for j in range(2)] for i in range(2)]
            grads = [(dlag(a, X) * lag(b, Y), lag(a, X) * dlag(b, Y)) for a, b in nodes]
            for k in range(9):
                for l in range(9):
                    for s in range(2):
                        for u in range(2):
                            A[k][l] += w * grads[k][s] * G[s][u] * grads[l][u]
                            N[k][l] += w * abs(grads[k][s]) * abs(G[s][u]) * abs(grads[l][u])
    nmax = max(max(r) for r in N)
    amax = max(max(abs(x) for x in r) for r in A)
    return nmax / amax, (t, wt, corners)


def test_kappa_q_box_exact_brute_force():
    kq_exact, (t, wt, corners) = _rational_q2_quad_kappa_q()
    m = len(t)
    pts = np.array([[float(t[qx]), float(t[qy])] for qy in range(m) for qx in range(m)])
    w = np.array([float(wt[qx] * wt[qy]) for qy in range(m) for qx in range(m)])
    v = np.array([[float(a), float(b)] for a, b in corners])
    pr = oracle.Problem(v, np.array([[0, 1, 2, 3]], dtype=np.int32), 2, pts, w)
    kap = np.ones((1, m * m))
    A = pr.element_matrices(kap, "stiffness")
    kq = pr.kappa_q(kap, "stiffness", A)
    assert kq_exact == Fr(1307, 917)
    assert abs(kq[0] - float(kq_exact)) < 1e-13 * float(kq_exact)


@pytest.mark.parametrize("cell,n,p", [("quadrilateral", 3, 1), ("quadrilateral", 3, 3), ("hexahedron", 2, 1),
                                      ("hexahedron", 2, 2), ("hexahedron", 2, 3)])
def test_box_dofmap(cell, n, p):
    v, c = inputs.structured_mesh(cell, n, 0.15, 7)
    pr = oracle.Problem(v, c, p, *oracle.rule_for_degree(cell, p))
    d = pr.d
    assert pr.n_dofs == (p * n + 1) ** d
    dofs, nd = pr.cell_dofs()
    lam = oracle.box_node_weights(d, p).astype(np.float64) / float(p) ** d
    phys = np.einsum("kv,cvi->cki", lam, v[c])
    first = np.full((nd, d), np.nan)
    for cc in range(pr.n_cells):
        for k in range(pr.n_phi):
            g = dofs[cc, k]
            if np.isnan(first[g, 0]):
                first[g] = phys[cc, k]
            else:
                assert np.allclose(first[g], phys[cc, k], atol=1e-14)
    assert len(np.unique(np.round(first, 12), axis=0)) == nd
