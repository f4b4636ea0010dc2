"""GPU adjoint of the assembly for a general gradient g on the CSR values
(fe_adjoint_values, L = sum_e g_e A^g_e, stiffness) against the FP64 oracle.

dL/dkappa and L against the oracle's adjoint_stiffness_values (pinned on the
CPU by the transpose identity of the gather, the rank-one case and central
differences in kappa), dL/dvertices against central differences of the
oracle's L(x) (step 1e-6, kappa held fixed), the rank-one gradient
g_ij = v_i u_j against fe_adjoint, the torch.autograd.Function
AssembleStiffness, and bitwise repeatability.  Sizes: small meshes with a
ragged last CTA, and P2 tetrahedra on 16^3 x 6 boxes.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2410_12614_gb300 import api, inputs

from gpu_util import cuda, to_np

pytestmark = pytest.mark.gpu


def _case(cell, n, p, seeds):
    v, c = inputs.structured_mesh(cell, n, 0.15, seeds[0])
    pts, w = api.quadrature_rule(cell, p + 1)
    plan = api.Plan(cell, v, c, p, pts, w, forms=("stiffness",), precisions=("bf16",))
    kap = inputs.lognormal_kappa(plan.n_cells, plan.n_q, seeds[1])
    g = inputs.gaussian_vector(plan.nnz, seeds[2]).astype(np.float64)
    ref = oracle.Problem(v, c, p, *oracle.rule_for_degree(cell, p))
    return plan, ref, v, c, kap, g


def _oracle_L(ref, v, c, kap, g, p, cell):
    r = oracle.Problem(v, c, p, *oracle.rule_for_degree(cell, p))
    return float(g @ r.assemble(r.element_matrices(kap, "stiffness")))


@pytest.mark.parametrize("cell,n,p", [("triangle", 3, 2), ("triangle", 2, 5), ("tetrahedron", 2, 1),
                                      ("tetrahedron", 2, 2), ("tetrahedron", 2, 3)])
def test_values_adjoint_vs_oracle_and_fd(cell, n, p):
    plan, ref, v, c, kap, g = _case(cell, n, p, (41, 42, 43))
    L, gk, gx = plan.adjoint_values(cuda(kap), cuda(g))
    plan.sync()
    Lo, gko = ref.adjoint_stiffness_values(kap, g)
    assert abs(float(L.item()) - Lo) <= 1e-12 * np.sum(np.abs(g)) * np.abs(kap).max()
    assert np.abs(to_np(gk) - gko).max() <= 1e-12 * np.abs(gko).max()
    gx = to_np(gx)
    rng = np.random.default_rng(44)
    d = v.shape[1]
    for _ in range(5):
        vi, i = rng.integers(v.shape[0]), rng.integers(d)
        xp, xm = v.copy(), v.copy()
        xp[vi, i] += 1e-6
        xm[vi, i] -= 1e-6
        fd = (_oracle_L(ref, xp, c, kap, g, p, cell) - _oracle_L(ref, xm, c, kap, g, p, cell)) / 2e-6
        assert abs(fd - gx[vi, i]) <= 1e-6 * (np.abs(gx).max() + 1.0), (vi, i, fd, gx[vi, i])


def test_rank_one_gradient_matches_quadratic_form_adjoint():
    plan, ref, v, c, kap, _ = _case("tetrahedron", 3, 2, (45, 46, 47))
    u = inputs.gaussian_vector(plan.n_dofs, 48)
    w = inputs.gaussian_vector(plan.n_dofs, 49)
    rp, ci = plan.csr_pattern()
    rp, ci = rp.cpu().numpy().astype(np.int64), ci.cpu().numpy().astype(np.int64)
    rows = np.repeat(np.arange(plan.n_dofs), np.diff(rp))
    g = w.astype(np.float64)[rows] * u.astype(np.float64)[ci]
    L1, gk1, gx1 = plan.adjoint_values(cuda(kap), cuda(g))
    L2, gk2, gx2 = plan.adjoint(cuda(kap), cuda(u), cuda(w))
    plan.sync()
    assert abs(float(L1.item()) - float(L2.item())) <= 1e-12 * abs(float(L2.item()))
    assert torch.allclose(gk1, gk2, rtol=0, atol=1e-12 * float(gk2.abs().max()))
    assert torch.allclose(gx1, gx2, rtol=0, atol=1e-12 * float(gx2.abs().max()))


def test_autograd_assemble_stiffness_and_repeatability():
    plan, ref, v, c, kap, g = _case("tetrahedron", 16, 2, (50, 51, 52))
    kt = cuda(kap).requires_grad_(True)
    xt = cuda(v).requires_grad_(True)
    vals = api.AssembleStiffness.apply(kt, xt, plan, "bf16")
    (vals * cuda(g).to(vals.dtype)).sum().backward()
    # the backward is the FP64 adjoint of the exact form for the gradient it received
    gv = cuda(g).to(vals.dtype).double()
    L, gk, gx = plan.adjoint_values(cuda(kap), gv)
    L2, gk2, gx2 = plan.adjoint_values(cuda(kap), gv)
    plan.sync()
    assert torch.equal(kt.grad, gk) and torch.equal(xt.grad, gx)
    assert torch.equal(gk, gk2) and torch.equal(gx, gx2) and torch.equal(L, L2)
    # against the oracle on sampled cells (16^3 x 6 = 24,576 cells)
    Lo, gko = ref.adjoint_stiffness_values(kap, to_np(gv))
    assert np.abs(to_np(gk) - gko).max() <= 1e-12 * np.abs(gko).max()
