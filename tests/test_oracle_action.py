"""Pins of the oracle's linear forms (Algorithm 2) and vector assembly (Sec. 3.3).

* b^c equals A^c w^c with A^c from the literal element-matrix loops (a
  different computation of the same quantity);
* mass: sum_k b_k = sum_q w_q z |det J| w(X_q), and for w = 1 exactly the
  weighted cell volume (partition of unity, independent of B);
* stiffness: zero for constant w (sum_k grad phi_k = 0);
* stiffness with z = 1 and w interpolating a linear function a.x: the global
  vector vanishes at every interior dof (int grad phi_i . a = 0 when phi_i
  vanishes on the boundary);
* v^g = L b against a brute-force dense scatter.
"""
import numpy as np
import pytest

import oracle
from paper_2410_12614_gb300 import inputs

CASES = [("triangle", 3, 1), ("triangle", 2, 3), ("tetrahedron", 2, 1), ("tetrahedron", 2, 2), ("tetrahedron", 1, 3)]


def _problem(cell, n, p, seed):
    v, c = inputs.structured_mesh(cell, n, 0.15, seed)
    ref = oracle.Problem(v, c, p, *oracle.rule_for_degree(cell, p))
    kap = inputs.lognormal_kappa(ref.n_cells, ref.n_q, seed + 1)
    w = inputs.gaussian_vector(ref.cell_dofs()[1], seed + 2).astype(np.float64)
    return ref, kap, w


@pytest.mark.parametrize("cell,n,p", CASES)
def test_action_is_element_matrix_times_w(cell, n, p):
    ref, kap, w = _problem(cell, n, p, 70 + p)
    dofs, _ = ref.cell_dofs()
    for form in ("stiffness", "mass"):
        A = ref.element_matrices(kap, form)
        b = ref.action(kap, w, form)
        Aw = np.einsum("ckl,cl->ck", A, w[dofs])
        assert np.abs(b - Aw).max() <= 1e-12 * np.abs(Aw).max()


@pytest.mark.parametrize("cell,n,p", CASES)
def test_mass_action_sums_and_constants(cell, n, p):
    ref, kap, w = _problem(cell, n, p, 80 + p)
    det, _ = oracle.mesh_geometry(ref.vertices, ref.cells)
    dofs, nd = ref.cell_dofs()
    b = ref.action(kap, w, "mass")
    wq = np.einsum("ck,kq->cq", w[dofs], ref.phi)
    expect = np.einsum("q,cq,cq->c", ref.weights, kap, wq) * np.abs(det)
    assert np.allclose(b.sum(axis=1), expect, rtol=1e-13, atol=0)
    ones = ref.action(np.ones_like(kap), np.ones(nd), "mass")
    vol = np.abs(det) / (2.0 if ref.d == 2 else 6.0)
    assert np.allclose(ones.sum(axis=1), vol, rtol=1e-13, atol=0)
    s = ref.action(kap, np.full(nd, 3.0), "stiffness")
    assert np.abs(s).max() <= 1e-12 * np.abs(ref.action(kap, w, "stiffness")).max()


@pytest.mark.parametrize("cell,n,p", [("triangle", 4, 1), ("triangle", 3, 2), ("tetrahedron", 3, 1), ("tetrahedron", 2, 2)])
def test_stiffness_action_of_linear_function_vanishes_inside(cell, n, p):
    ref, _, _ = _problem(cell, n, p, 90 + p)
    a = np.array([0.7, -1.3, 0.4])[: ref.d]
    pts = ref.dof_points()
    w = pts @ a
    v = ref.assemble_vector(ref.action(np.ones((ref.n_cells, ref.n_q)), w, "stiffness"))
    interior = np.all((pts > 1e-9) & (pts < 1 - 1e-9), axis=1)
    assert interior.any()
    scale = np.abs(ref.action(np.ones((ref.n_cells, ref.n_q)), w, "stiffness")).max()
    assert np.abs(v[interior]).max() <= 1e-12 * scale


def test_vector_assembly_brute_force():
    ref, kap, w = _problem("tetrahedron", 2, 2, 95)
    dofs, nd = ref.cell_dofs()
    b = ref.action(kap, w, "stiffness")
    dense = np.zeros(nd)
    for c in range(ref.n_cells):
        for k in range(ref.n_phi):
            dense[dofs[c, k]] += b[c, k]
    assert np.allclose(ref.assemble_vector(b), dense, rtol=0, atol=1e-13 * np.abs(dense).max())
