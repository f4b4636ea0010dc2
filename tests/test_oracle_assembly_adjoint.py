"""Pins for the oracle's dof map, CSR pattern, assembly and adjoint.

Dof map: n_dofs = (pN+1)^d on the structured meshes (equispaced nodes of a
degree-p simplex mesh coincide with the fine lattice), every dof has one
physical point on all cells that list it and distinct dofs have distinct
points (continuity of the Lagrange space), vertex dofs take the vertex id and
the remaining keys are strictly increasing (the canonical numbering).
Pattern: brute force from a dense boolean matrix; P1 closed form
nnz = n_v + 2 n_edges.  Assembly (Sec. 3.3, A^g = L D L^T): dense
brute-force scatter with numpy, K^g 1 = 0, 1^T M^g 1 = sum of weighted
volumes, and the global energy identity.  Adjoint: central differences
(exact in kappa, which enters linearly), translation invariance and the
homogeneity identity sum_v x_v . dL/dx_v = (d-2) L.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2410_12614_gb300 import inputs


def _problem(cell, n, p, alpha=0.15, seed=3):
    v, c = inputs.structured_mesh(cell, n, alpha, seed)
    return oracle.Problem(v, c, p, *oracle.rule_for_degree(cell, p))


@pytest.mark.parametrize("cell,n,p", [("triangle", 3, 1), ("triangle", 4, 3), ("triangle", 2, 6),
                                      ("tetrahedron", 2, 1), ("tetrahedron", 2, 3), ("tetrahedron", 3, 2),
                                      ("tetrahedron", 1, 5)])
def test_dofmap_counts_and_continuity(cell, n, p):
    d = 2 if cell == "triangle" else 3
    pr = _problem(cell, n, p)
    dofs, nd = pr.cell_dofs()
    assert nd == (p * n + 1) ** d
    assert set(np.unique(dofs)) == set(range(nd))
    # vertex dofs are the vertex ids
    assert np.array_equal(dofs[:, : d + 1], pr.cells)
    # one physical point per dof, agreed on by every cell
    lam = np.hstack([1 - oracle.node_points(d, p).sum(1, keepdims=True), oracle.node_points(d, p)])
    phys = np.einsum("kv,cvi->cki", lam, pr.vertices[pr.cells]).reshape(-1, d)
    ref = pr.dof_points()
    np.testing.assert_allclose(phys, ref[dofs.reshape(-1)], rtol=0, atol=1e-14)
    # distinct dofs -> distinct points
    r = np.round(ref, 10)
    assert len(np.unique(r, axis=0)) == nd
    # no dof appears twice in one cell
    assert all(len(set(row)) == pr.n_phi for row in dofs)


def test_canonical_key_order():
    pr = _problem("tetrahedron", 2, 4)
    d = 3
    dofs, nd = pr.cell_dofs()
    nodes = oracle.lattice_nodes(d, 4)
    keys = {}
    for ci, cell in enumerate(pr.cells):
        for k, a in enumerate(nodes):
            sup = sorted((int(cell[i]), int(a[i])) for i in range(d + 1) if a[i] > 0)
            if len(sup) == 1:
                continue
            key = (len(sup), tuple(g for g, _ in sup), tuple(m for _, m in sup))
            keys.setdefault(int(dofs[ci, k]), set()).add(key)
    assert all(len(s) == 1 for s in keys.values())
    ordered = [next(iter(keys[i])) for i in range(pr.vertices.shape[0], nd)]
    assert all(ordered[i] < ordered[i + 1] for i in range(len(ordered) - 1))


def _dense_pattern(dofs, nd):
    P = np.zeros((nd, nd), dtype=bool)
    for row in dofs:
        P[np.ix_(row, row)] = True
    return P


@pytest.mark.parametrize("cell,n,p", [("triangle", 3, 2), ("tetrahedron", 2, 2), ("tetrahedron", 1, 4)])
def test_pattern_brute_force(cell, n, p):
    pr = _problem(cell, n, p)
    dofs, nd = pr.cell_dofs()
    rp, ci = pr.csr_pattern()
    P = _dense_pattern(dofs, nd)
    for i in range(nd):
        assert np.array_equal(ci[rp[i]:rp[i + 1]], np.nonzero(P[i])[0])
    assert rp[-1] == P.sum()


def test_p1_triangle_pattern_closed_form():
    n = 32
    pr = _problem("triangle", n, 1, alpha=0.2)
    edges = 2 * n * (n + 1) + n * n  # horizontal + vertical + one diagonal per box
    assert pr.csr_pattern()[0][-1] == (n + 1) ** 2 + 2 * edges == 7361


def test_p1_tet_pattern_closed_form():
    n = 6
    pr = _problem("tetrahedron", n, 1)
    edges = 3 * n * (n + 1) ** 2 + 3 * n * n * (n + 1) + n ** 3  # axis, face-diagonal, body-diagonal
    assert pr.csr_pattern()[0][-1] == (n + 1) ** 3 + 2 * edges


@pytest.mark.parametrize("cell,n,p", [("triangle", 3, 3), ("tetrahedron", 2, 2), ("tetrahedron", 2, 3)])
def test_assembly_brute_force_and_invariants(cell, n, p):
    d = 2 if cell == "triangle" else 3
    pr = _problem(cell, n, p)
    kap = inputs.lognormal_kappa(pr.n_cells, pr.n_q, 12)
    dofs, nd = pr.cell_dofs()
    rp, ci = pr.csr_pattern()
    for form in ("stiffness", "mass"):
        A = pr.element_matrices(kap, form)
        vals = pr.assemble(A)
        D = np.zeros((nd, nd))
        for c in range(pr.n_cells):
            np.add.at(D, (dofs[c][:, None], dofs[c][None, :]), A[c])
        S = np.zeros((nd, nd))
        for i in range(nd):
            S[i, ci[rp[i]:rp[i + 1]]] = vals[rp[i]:rp[i + 1]]
        np.testing.assert_allclose(S, D, rtol=0, atol=1e-14 * np.abs(D).max())
        np.testing.assert_allclose(S, S.T, rtol=0, atol=1e-14 * np.abs(D).max())
        if form == "stiffness":
            np.testing.assert_allclose(S.sum(axis=1), 0.0, atol=1e-12 * np.abs(S).max())
        else:
            det, _ = oracle.mesh_geometry(pr.vertices, pr.cells, with_G=False)
            total = float(np.sum((kap @ pr.weights) * np.abs(det)))
            assert abs(S.sum() - total) <= 1e-13 * total


def test_global_energy_identity():
    cell, p = "tetrahedron", 3
    pr = _problem(cell, 2, p)
    d = 3
    kap = inputs.lognormal_kappa(pr.n_cells, pr.n_q, 13)
    vals = pr.assemble(pr.element_matrices(kap, "stiffness"))
    rp, ci = pr.csr_pattern()
    pts = pr.dof_points()
    rng = np.random.default_rng(14)
    expo = [e for e in itertools.product(range(p + 1), repeat=d) if sum(e) <= p]
    cf, cg = rng.standard_normal(len(expo)), rng.standard_normal(len(expo))
    f = lambda x: sum(a * np.prod(x ** np.array(e), axis=-1) for a, e in zip(cf, expo))
    g = lambda x: sum(a * np.prod(x ** np.array(e), axis=-1) for a, e in zip(cg, expo))

    def grad(cfs, x):
        out = np.zeros(x.shape)
        for a, e in zip(cfs, expo):
            for s in range(d):
                if e[s]:
                    e2 = list(e)
                    e2[s] -= 1
                    out[..., s] += a * e[s] * np.prod(x ** np.array(e2), axis=-1)
        return out

    uf, ug = f(pts), g(pts)
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    lhs = np.sum(uf[rows] * vals * ug[ci])
    lam_q = np.hstack([1 - pr.points.sum(1, keepdims=True), pr.points])
    rhs = 0.0
    for c in range(pr.n_cells):
        xv = pr.vertices[pr.cells[c]]
        vol = abs(np.linalg.det((xv[1:] - xv[0]).T))
        xq = lam_q @ xv
        rhs += np.sum(pr.weights * kap[c] * vol * np.sum(grad(cf, xq) * grad(cg, xq), axis=1))
    assert abs(lhs - rhs) <= 1e-11 * abs(rhs)


# ---------------------------------------------------------------------------
# adjoint of L = v^T A^g u (Poisson)
# ---------------------------------------------------------------------------
def _L(pr, kap, u, v):
    vals = pr.assemble(pr.element_matrices(kap, "stiffness"))
    rp, ci = pr.csr_pattern()
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    return float(np.sum(v[rows] * vals * u[ci]))


@pytest.mark.parametrize("cell,p", [("triangle", 2), ("tetrahedron", 2)])
def test_adjoint_matches_finite_differences(cell, p):
    d = 2 if cell == "triangle" else 3
    pr = _problem(cell, 2, p)
    kap = inputs.lognormal_kappa(pr.n_cells, pr.n_q, 21)
    u = inputs.gaussian_vector(pr.n_dofs, 22).astype(np.float64)
    v = inputs.gaussian_vector(pr.n_dofs, 23).astype(np.float64)
    L, gk, gx = pr.adjoint_stiffness(kap, u, v)
    assert abs(L - _L(pr, kap, u, v)) <= 1e-12 * abs(L)
    rng = np.random.default_rng(5)
    # kappa enters linearly: central differences are exact up to rounding
    for _ in range(6):
        c, q = rng.integers(pr.n_cells), rng.integers(pr.n_q)
        h = 1e-3
        kp, km = kap.copy(), kap.copy()
        kp[c, q] += h
        km[c, q] -= h
        fd = (_L(pr, kp, u, v) - _L(pr, km, u, v)) / (2 * h)
        assert abs(fd - gk[c, q]) <= 1e-9 * (abs(gk).max())
    # vertex coordinates: central differences with step 1e-6 (kappa held fixed)
    for _ in range(6):
        vi, i = rng.integers(pr.vertices.shape[0]), rng.integers(d)
        h = 1e-6
        xp, xm = pr.vertices.copy(), pr.vertices.copy()
        xp[vi, i] += h
        xm[vi, i] -= h
        fd = (_L(pr.with_vertices(xp), kap, u, v) - _L(pr.with_vertices(xm), kap, u, v)) / (2 * h)
        assert abs(fd - gx[vi, i]) <= 1e-6 * np.abs(gx).max()
    # translation invariance and homogeneity of degree d-2
    np.testing.assert_allclose(gx.sum(axis=0), 0.0, atol=1e-12 * np.abs(gx).max())
    assert abs(np.sum(pr.vertices * gx) - (d - 2) * L) <= 1e-11 * max(abs(L), np.abs(gx).max())


# ---------------------------------------------------------------------------
# adjoint of L = sum_e g_e A^g_e (Poisson) for a general gradient g on the CSR values
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("cell,n,p", [("triangle", 3, 2), ("tetrahedron", 2, 2), ("tetrahedron", 1, 3)])
def test_gather_is_the_transpose_of_the_assembly(cell, n, p):
    pr = _problem(cell, n, p)
    rp, ci = pr.csr_pattern()
    rng = np.random.default_rng(31)
    A = rng.standard_normal((pr.n_cells, pr.n_phi, pr.n_phi))     # any element matrices
    g = rng.standard_normal(len(ci))
    assert abs(g @ pr.assemble(A) - np.sum(pr.gather_values(g) * A)) <= 1e-12 * np.sum(np.abs(A))


@pytest.mark.parametrize("cell,p", [("triangle", 2), ("tetrahedron", 2)])
def test_values_adjoint_rank_one_is_the_quadratic_form_adjoint(cell, p):
    # g_e = v_i u_j on the slot (i, j) makes sum_e g_e A^g_e = v^T A^g u
    pr = _problem(cell, 2, p)
    kap = inputs.lognormal_kappa(pr.n_cells, pr.n_q, 32)
    u = inputs.gaussian_vector(pr.n_dofs, 33).astype(np.float64)
    v = inputs.gaussian_vector(pr.n_dofs, 34).astype(np.float64)
    rp, ci = pr.csr_pattern()
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    L, gk = pr.adjoint_stiffness_values(kap, v[rows] * u[ci])
    L2, gk2, _ = pr.adjoint_stiffness(kap, u, v, want_x=False)
    assert abs(L - L2) <= 1e-12 * abs(L2)
    assert np.abs(gk - gk2).max() <= 1e-12 * np.abs(gk2).max()


def test_values_adjoint_matches_finite_differences_in_kappa():
    pr = _problem("tetrahedron", 2, 2)
    kap = inputs.lognormal_kappa(pr.n_cells, pr.n_q, 35)
    rp, ci = pr.csr_pattern()
    g = inputs.gaussian_vector(len(ci), 36).astype(np.float64)

    def L_of(k):
        return float(g @ pr.assemble(pr.element_matrices(k, "stiffness")))

    L, gk = pr.adjoint_stiffness_values(kap, g)
    assert abs(L - L_of(kap)) <= 1e-12 * np.sum(np.abs(g))
    rng = np.random.default_rng(37)
    for _ in range(6):
        c, q = rng.integers(pr.n_cells), rng.integers(pr.n_q)
        kp, km = kap.copy(), kap.copy()
        kp[c, q] += 1e-3
        km[c, q] -= 1e-3
        fd = (L_of(kp) - L_of(km)) / 2e-3
        assert abs(fd - gk[c, q]) <= 1e-9 * np.abs(gk).max()


def _L_complex(pr, kap, u, v, X):
    """L = sum_c u_c^T A^c v_c (stiffness) for complex vertex coordinates X: the
    element matrix definition (Sec. 3.1) with |det J| replaced by sign(det J) det J
    (analytic in X, equal to |det J| for real X), J^-1 by complex inversion."""
    dofs, _ = pr.cell_dofs()
    x = X[pr.cells]                                                  # [nc, d+1, d]
    J = np.transpose(x[:, 1:, :] - x[:, :1, :], (0, 2, 1))           # J[:, i, j] = x^{j+1}_i - x^0_i
    det = np.linalg.det(J)
    sgn = np.sign(det.real)
    Ji = np.linalg.inv(J)
    # physical gradients J^-T grad phi at every point: [nc, k, q, i]
    grad = np.einsum("cri,rkq->ckqi", Ji, pr.dphi)
    Ac = np.einsum("q,cq,c,ckqi,clqi->ckl", pr.weights, kap, sgn * det, grad, grad)
    return np.einsum("ck,ckl,cl->", u[dofs], Ac, v[dofs])


@pytest.mark.parametrize("cell,p", [("triangle", 3), ("tetrahedron", 2)])
def test_adjoint_vertex_gradient_by_complex_step(cell, p):
    """dL/dx of the oracle's closed form against the complex-step derivative
    Im L(x + i h e) / h with h = 1e-30: no subtractive cancellation, so the two
    must agree to rounding (1e-13 of the largest gradient entry)."""
    pr = _problem(cell, 2, p)
    kap = inputs.lognormal_kappa(pr.n_cells, pr.n_q, 41)
    u = inputs.gaussian_vector(pr.n_dofs, 42).astype(np.float64)
    v = inputs.gaussian_vector(pr.n_dofs, 43).astype(np.float64)
    L, _, gx = pr.adjoint_stiffness(kap, u, v)
    X0 = pr.vertices.astype(np.complex128)
    assert abs(_L_complex(pr, kap, u, v, X0).real - L) <= 1e-12 * abs(L)
    h = 1e-30
    for vi in range(pr.vertices.shape[0]):
        for i in range(pr.d):
            X = X0.copy()
            X[vi, i] += 1j * h
            cs = _L_complex(pr, kap, u, v, X).imag / h
            assert abs(cs - gx[vi, i]) <= 1e-13 * np.abs(gx).max(), (vi, i, cs, gx[vi, i])
