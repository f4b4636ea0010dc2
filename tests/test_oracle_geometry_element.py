"""Pins for the oracle's geometry and element matrices.

Geometry (Sec. 4.2): the knife tetrahedron of Sec. 5.2 with its printed
det J = eps and kappa_inf = (2+eps)(3+eps)/eps, its closed-form inverse,
J^{-1} J = I, and agreement with LAPACK's det/inv on random cells.
Element matrices (Sec. 3.1): P1 closed forms on the reference cells and on
arbitrary cells (K = (sum_q w_q kappa_q)|det J| grad(lambda_k).grad(lambda_l)
with the barycentric gradients from a numpy solve), zero row sums, mass sum
equal to the weighted volume, symmetry, definiteness, the energy identity
u^T A v = sum_q w_q kappa_q |det J| grad f(x_q).grad g(x_q) for interpolants
of polynomials (which never touches the tabulation B), and agreement with a
higher-order rule when kappa = 1 (exactness).
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2410_12614_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _knife(eps, transformed):
    v = np.array([[0, 0, 0], [1, 1, 0], [1, 0, 1], [eps, 1, -1]], dtype=np.float64)
    if transformed:
        v = v / math.sqrt(3.0) + np.array([1 / 3, 2 / 3, 4 / 3])
    return v


@pytest.mark.parametrize("eps", [1e-1, 1e-3, 1e-6, 1e-9])
def test_knife_tet_closed_forms(eps):
    with open(os.path.join(GOLDEN, "e2_knife_tet.json")) as f:
        g = json.load(f)
    M = np.array([[eps if x == "eps" else x for x in row] for row in g["printed_M"]], dtype=np.float64)
    J, det, Jinv = oracle.geometry(_knife(eps, False))
    np.testing.assert_array_equal(J, M.T)
    assert abs(det - eps) <= 1e-15
    kinf = (2 + eps) * (3 + eps) / eps
    k1 = np.abs(J).sum(axis=0).max() * np.abs(Jinv).sum(axis=0).max()
    assert abs(k1 - kinf) <= 1e-14 * kinf * kinf
    adj = np.array([[-1, 1, 1], [1 + eps, -1, -1], [1, eps - 1, -1]], dtype=np.float64)
    Jinv_exact = adj.T / eps
    np.testing.assert_allclose(Jinv, Jinv_exact, rtol=0, atol=4e-16 * kinf * np.abs(Jinv_exact).max())
    # scaled and translated cell: det = eps 3^{-3/2}; errors grow like u kappa
    J2, det2, Jinv2 = oracle.geometry(_knife(eps, True))
    u = 2.0 ** -53
    assert abs(det2 - eps * 3 ** -1.5) <= 50 * u * kinf * eps
    err = np.abs(Jinv2 @ J2 - np.eye(3)).max()
    assert err <= 50 * u * kinf
    # G = |det J| J^{-1} J^{-T} in closed form for the scaled cell
    _, G = oracle.mesh_geometry(_knife(eps, True), np.array([[0, 1, 2, 3]], dtype=np.int32))
    G_exact = (eps / math.sqrt(3.0)) * Jinv_exact @ Jinv_exact.T
    assert np.abs(G[0] - G_exact).max() <= 200 * u * kinf * np.abs(G_exact).max()


def test_geometry_matches_lapack_on_random_cells():
    rng = np.random.default_rng(11)
    for d in (2, 3):
        for _ in range(50):
            xv = rng.standard_normal((d + 1, d))
            J, det, Jinv = oracle.geometry(xv)
            Jr = (xv[1:] - xv[0]).T
            np.testing.assert_array_equal(J, Jr)
            assert abs(det - np.linalg.det(Jr)) <= 1e-13 * max(1.0, abs(det))
            np.testing.assert_allclose(Jinv, np.linalg.inv(Jr), rtol=1e-11, atol=1e-11)


def test_degenerate_cell_reported():
    xv = np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0], [0, 1, 0]], dtype=np.float64)
    with pytest.raises(RuntimeError):
        oracle.geometry(xv)


@pytest.mark.parametrize("d", [2, 3])
def test_p1_reference_cell_closed_forms(d):
    with open(os.path.join(GOLDEN, "p1_reference_matrices.json")) as f:
        g = json.load(f)
    verts = np.vstack([np.zeros(d), np.eye(d)])
    cells = np.arange(d + 1, dtype=np.int32)[None, :]
    cell = "triangle" if d == 2 else "tetrahedron"
    pts, w = oracle.collapsed_rule(cell, 2)
    pr = oracle.Problem(verts, cells, 1, pts, w)
    one = np.ones((1, pr.n_q))
    K = pr.element_matrices(one, "stiffness")[0]
    M = pr.element_matrices(one, "mass")[0]
    if d == 2:
        Kx = np.array(g["triangle"]["stiffness"])
        Mx = np.array(g["triangle"]["mass_times_24"]) / 24.0
    else:
        Kx = np.array(g["tetrahedron"]["stiffness_times_6"]) / 6.0
        Mx = np.array(g["tetrahedron"]["mass_times_120"]) / 120.0
    np.testing.assert_allclose(K, Kx, rtol=0, atol=1e-15)
    np.testing.assert_allclose(M, Mx, rtol=0, atol=1e-16)


def _bary_gradients(xv):
    """Physical gradients of the barycentric coordinates, [d+1, d], by solving
    [1 x_k] c = e: lambda_k(x) = c_k0 + c_k . x."""
    d = xv.shape[1]
    T = np.hstack([np.ones((d + 1, 1)), xv])
    C = np.linalg.inv(T)  # columns: coefficients of lambda_k
    return C[1:, :].T


@pytest.mark.parametrize("cell", ["triangle", "tetrahedron"])
def test_p1_any_cell_with_pointwise_kappa(cell):
    d = 2 if cell == "triangle" else 3
    v, c = inputs.structured_mesh(cell, 3, 0.2, 5)
    pts, w = oracle.collapsed_rule(cell, 2)
    pr = oracle.Problem(v, c, 1, pts, w)
    kap = inputs.lognormal_kappa(pr.n_cells, pr.n_q, 6)
    K = pr.element_matrices(kap, "stiffness")
    for ci in range(pr.n_cells):
        xv = v[c[ci]]
        vol = abs(np.linalg.det((xv[1:] - xv[0]).T))
        Gl = _bary_gradients(xv)
        Kx = (w @ kap[ci]) * vol * Gl @ Gl.T
        np.testing.assert_allclose(K[ci], Kx, rtol=1e-12, atol=1e-14 * np.abs(Kx).max())


def _poly(coef, expo, x):
    return sum(cf * np.prod(x ** np.array(e), axis=-1) for cf, e in zip(coef, expo))


def _poly_grad(coef, expo, x):
    d = x.shape[-1]
    out = np.zeros(x.shape)
    for cf, e in zip(coef, expo):
        for s in range(d):
            if e[s] == 0:
                continue
            e2 = list(e)
            e2[s] -= 1
            out[..., s] += cf * e[s] * np.prod(x ** np.array(e2), axis=-1)
    return out


@pytest.mark.parametrize("cell,p", [("triangle", 2), ("triangle", 4), ("tetrahedron", 2), ("tetrahedron", 3)])
def test_energy_identity_and_invariants(cell, p):
    d = 2 if cell == "triangle" else 3
    v, c = inputs.structured_mesh(cell, 2, 0.2 if d == 2 else 0.15, 3)
    pts, w = oracle.rule_for_degree(cell, p)
    pr = oracle.Problem(v, c, p, pts, w)
    kap = inputs.lognormal_kappa(pr.n_cells, pr.n_q, 4)
    K = pr.element_matrices(kap, "stiffness")
    M = pr.element_matrices(kap, "mass")
    det, _ = oracle.mesh_geometry(v, c, with_G=False)
    # symmetry, row sums, mass sum
    np.testing.assert_allclose(K, K.transpose(0, 2, 1), rtol=0, atol=1e-15 * np.abs(K).max())
    np.testing.assert_allclose(K.sum(axis=2), 0.0, atol=1e-13 * np.abs(K).max())
    vols = np.array([abs(np.linalg.det((v[cc][1:] - v[cc][0]).T)) for cc in c])
    np.testing.assert_allclose(M.sum(axis=(1, 2)), (kap @ w) * vols, rtol=1e-13)
    # definiteness on every cell
    for ci in range(pr.n_cells):
        ek = np.linalg.eigvalsh(K[ci])
        em = np.linalg.eigvalsh(M[ci])
        assert ek[0] > -1e-12 * ek[-1] and abs(ek[0]) < 1e-12 * ek[-1] and ek[1] > 1e-8 * ek[-1]
        assert em[0] > 0
    # energy identity for two random polynomials of degree p
    rng = np.random.default_rng(9)
    expo = [e for e in itertools.product(range(p + 1), repeat=d) if sum(e) <= p]
    cf, cg = rng.standard_normal(len(expo)), rng.standard_normal(len(expo))
    lam_nodes = np.hstack([1 - oracle.node_points(d, p).sum(1, keepdims=True), oracle.node_points(d, p)])
    lam_q = np.hstack([1 - pts.sum(1, keepdims=True), pts])
    for ci in range(pr.n_cells):
        xv = v[c[ci]]
        xn = lam_nodes @ xv
        xq = lam_q @ xv
        uf, ug = _poly(cf, expo, xn), _poly(cg, expo, xn)
        fac = w * kap[ci] * vols[ci]
        eK = np.sum(fac * np.sum(_poly_grad(cf, expo, xq) * _poly_grad(cg, expo, xq), axis=1))
        eM = np.sum(fac * _poly(cf, expo, xq) * _poly(cg, expo, xq))
        assert abs(uf @ K[ci] @ ug - eK) <= 1e-11 * (abs(eK) + np.abs(K[ci]).max())
        assert abs(uf @ M[ci] @ ug - eM) <= 1e-11 * (abs(eM) + np.abs(M[ci]).max())


@pytest.mark.parametrize("cell,p", [("triangle", 3), ("tetrahedron", 2), ("tetrahedron", 4)])
def test_higher_order_rule_agrees_for_constant_kappa(cell, p):
    v, c = inputs.structured_mesh(cell, 2, 0.15, 8)
    a = oracle.Problem(v, c, p, *oracle.collapsed_rule(cell, p + 1))
    b = oracle.Problem(v, c, p, *oracle.collapsed_rule(cell, p + 3))
    for form in ("stiffness", "mass"):
        Aa = a.element_matrices(np.ones((a.n_cells, a.n_q)), form)
        Ab = b.element_matrices(np.ones((b.n_cells, b.n_q)), form)
        np.testing.assert_allclose(Aa, Ab, rtol=0, atol=1e-13 * np.abs(Ab).max())


def test_kappa_q_p1_mass_is_one_and_at_least_one():
    v, c = inputs.cube_mesh(2, 0.15, 1)
    pts, w = oracle.collapsed_rule("tetrahedron", 2)
    pr = oracle.Problem(v, c, 1, pts, w)
    kap = inputs.lognormal_kappa(pr.n_cells, pr.n_q, 2)
    M = pr.element_matrices(kap, "mass")
    # P1 mass: every term of sum |B||C||B| is nonnegative, so there is no cancellation
    np.testing.assert_allclose(pr.kappa_q(kap, "mass", M), 1.0, rtol=1e-14)
    pr3 = oracle.Problem(v, c, 3, *oracle.rule_for_degree("tetrahedron", 3))
    kap3 = inputs.lognormal_kappa(pr3.n_cells, pr3.n_q, 2)
    for form in ("stiffness", "mass"):
        A = pr3.element_matrices(kap3, form)
        assert np.all(pr3.kappa_q(kap3, form, A) >= 1.0 - 1e-14)


def _golden_kq():
    with open(os.path.join(os.path.dirname(__file__), "golden", "kappa_q_closed_forms.json")) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _golden_kq(), ids=lambda c: c["name"])
def test_kappa_q_closed_forms(case):
    """kappa_q^A of Corollary 4.10 for the stiffness form equals hand-derived
    values on cells whose G has nonzero off-diagonal entries (a dropped |.| on
    G, dropped off-diagonal pairs or a wrong index in the oracle change it);
    translating and scaling the cell leaves it unchanged."""
    d = 3 if case["cell_type"] == "tetrahedron" else 2
    xv = np.array(case["vertices"], dtype=np.float64)
    cells = np.arange(d + 1, dtype=np.int32)[None, :]
    p = case["degree"]
    if "rule" in case:
        pts, wts = oracle.strang_fix_3()
    else:
        pts, wts = oracle.rule_for_degree(case["cell_type"], 2)
    rng = np.random.default_rng(7)
    for shift, scale in ((0.0, 1.0), (3.25, 0.125), (-1.5, 7.0)):
        v = shift + scale * xv
        pr = oracle.Problem(v, cells, p, pts, wts)
        if case["kappa"] == 1.0:
            kap = np.ones((1, pr.n_q))
        else:
            kap = np.exp(rng.standard_normal((1, pr.n_q)))
        A = pr.element_matrices(kap, "stiffness")
        kq = pr.kappa_q(kap, "stiffness", A)
        np.testing.assert_allclose(kq, case["kappa_q"], rtol=1e-13)
        for wrong in case["wrong_if"].values():
            assert abs(kq[0] - wrong) > 0.1
