"""Pins for the oracle's quadrature rules and Lagrange tabulation.

Quadrature: exact integration of monomials against the Dirichlet closed form
int_T x^a y^b z^c = a! b! c! / (a+b+c+d)! (Sec. 3.1 requires exact rules),
sharpness one degree above, and the textbook rules of tests/golden.
Basis (Appendix A product form): Kronecker property at the lattice nodes,
partition of unity, exact reproduction of every polynomial of degree <= p and
of its gradient (which pins the product-rule derivatives independently of
their formula), and the P1 gradients.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dirichlet(expo):
    d = len(expo)
    return math.prod(math.factorial(e) for e in expo) / math.factorial(sum(expo) + d)


def _monomials(d, deg):
    return [e for e in itertools.product(range(deg + 1), repeat=d) if sum(e) <= deg]


@pytest.mark.parametrize("cell", ["triangle", "tetrahedron"])
@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 6, 9])
def test_collapsed_rule_exact_to_2m_minus_1(cell, m):
    d = 2 if cell == "triangle" else 3
    pts, w = oracle.collapsed_rule(cell, m)
    assert pts.shape == (m ** d, d)
    assert np.all(w > 0)
    # every point inside the reference simplex
    assert np.all(pts >= 0) and np.all(pts.sum(axis=1) <= 1)
    for e in _monomials(d, 2 * m - 1):
        approx = float(np.sum(w * np.prod(pts ** np.array(e), axis=1)))
        exact = _dirichlet(e)
        assert abs(approx - exact) <= 2e-14 * exact + 1e-17, (e, approx, exact)


@pytest.mark.parametrize("cell", ["triangle", "tetrahedron"])
@pytest.mark.parametrize("m", [1, 2, 3, 4])
def test_collapsed_rule_not_exact_at_2m(cell, m):
    d = 2 if cell == "triangle" else 3
    pts, w = oracle.collapsed_rule(cell, m)
    worst = 0.0
    for e in _monomials(d, 2 * m):
        if sum(e) != 2 * m:
            continue
        approx = float(np.sum(w * np.prod(pts ** np.array(e), axis=1)))
        worst = max(worst, abs(approx - _dirichlet(e)) / _dirichlet(e))
    assert worst > 1e-6


def test_weights_sum_to_reference_volume():
    for m in range(1, 10):
        assert abs(oracle.collapsed_rule("triangle", m)[1].sum() - 0.5) < 1e-15
        assert abs(oracle.collapsed_rule("tetrahedron", m)[1].sum() - 1.0 / 6.0) < 1e-15


def test_gauss_jacobi_textbook_rules():
    with open(os.path.join(GOLDEN, "gauss_jacobi_small.json")) as f:
        g = json.load(f)
    s3 = 1 / math.sqrt(3)
    expect = {
        (1, 0): ([0.5], [1.0]),
        (2, 0): ([(1 - s3) / 2, (1 + s3) / 2], [0.5, 0.5]),
        (1, 1): ([1 / 3], [0.5]),
        (1, 2): ([0.25], [1 / 3]),
    }
    t1, t2 = 0.4 - math.sqrt(0.06), 0.4 + math.sqrt(0.06)
    w2 = (1 / 6 - 0.5 * t1) / (t2 - t1)
    expect[(2, 1)] = ([t1, t2], [0.5 - w2, w2])
    assert len(g["rules"]) == len(expect)
    for (m, a), (nodes, wts) in expect.items():
        t, w = oracle.gauss_jacobi(m, a)
        np.testing.assert_allclose(t, nodes, rtol=0, atol=2e-16)
        np.testing.assert_allclose(w, wts, rtol=0, atol=2e-16)


def test_strang_fix_rule_degree_2():
    pts, w = oracle.strang_fix_3()
    for e in _monomials(2, 2):
        approx = float(np.sum(w * np.prod(pts ** np.array(e), axis=1)))
        assert abs(approx - _dirichlet(e)) < 1e-16


def test_unit_roundoffs_match_table_1():
    with open(os.path.join(GOLDEN, "table1_unit_roundoff.json")) as f:
        g = json.load(f)
    for k, e in g["u_log2"].items():
        assert oracle.UNIT_ROUNDOFF[k] == 2.0 ** e


# ---------------------------------------------------------------------------
# basis
# ---------------------------------------------------------------------------
CASES = [(2, p) for p in range(1, 7)] + [(3, p) for p in range(1, 9)]


@pytest.mark.parametrize("d,p", CASES)
def test_basis_kronecker_at_nodes(d, p):
    X = oracle.node_points(d, p)
    phi, _ = oracle.tabulate(d, p, X)
    assert phi.shape == (math.comb(p + d, d),) * 2
    np.testing.assert_allclose(phi, np.eye(phi.shape[0]), rtol=0, atol=1e-13)


def _random_points(d, n, seed):
    rng = np.random.default_rng(seed)
    pts = rng.dirichlet(np.ones(d + 1), size=n)[:, 1:]
    return pts


@pytest.mark.parametrize("d,p", [(2, 1), (2, 3), (2, 6), (3, 1), (3, 2), (3, 4), (3, 6)])
def test_basis_reproduces_polynomials_and_gradients(d, p):
    X = oracle.node_points(d, p)
    Y = _random_points(d, 25, 7 + p)
    phi, dphi = oracle.tabulate(d, p, Y)
    np.testing.assert_allclose(phi.sum(axis=0), 1.0, atol=1e-13)
    np.testing.assert_allclose(dphi.sum(axis=1), 0.0, atol=1e-11)
    for e in _monomials(d, p):
        e = np.array(e)
        f_nodes = np.prod(X ** e, axis=1)
        f_exact = np.prod(Y ** e, axis=1)
        np.testing.assert_allclose(f_nodes @ phi, f_exact, atol=1e-12)
        for s in range(d):
            if e[s] == 0:
                g_exact = np.zeros(len(Y))
            else:
                e2 = e.copy()
                e2[s] -= 1
                g_exact = e[s] * np.prod(Y ** e2, axis=1)
            np.testing.assert_allclose(f_nodes @ dphi[s], g_exact, atol=1e-10 * p ** 2)


@pytest.mark.parametrize("d", [2, 3])
def test_p1_gradients_and_node_order(d):
    phi, dphi = oracle.tabulate(d, 1, np.full((1, d), 0.2))
    g = dphi[:, :, 0].T  # [n_phi, d]
    expect = np.vstack([-np.ones(d), np.eye(d)])
    assert np.array_equal(g, expect)
    # vertices first in cell-vertex order, then edges 01, 02, ...
    nodes = oracle.lattice_nodes(d, 3)
    assert [tuple(nodes[i]) for i in range(d + 1)] == [tuple(3 * np.eye(d + 1, dtype=int)[i]) for i in range(d + 1)]
    e0 = nodes[d + 1]
    assert e0[0] == 2 and e0[1] == 1  # first edge node: on edge 01, closer to vertex 0
