"""Boxed cells on the GPU (quadrilaterals and hexahedra; Sec. 3.1, the paper's
60x case of Sec. 5.5) against the oracle.

Jittered structured meshes (non-affine cells: J, det J and G vary with the
quadrature point), kappa lognormal(0,1), the (p+1)^d tensor Gauss-Legendre
rule.  Every format of the tensor-core contraction and the FP64 path:
element matrices of every cell within the per-cell bound of Corollary 4.10
(kappa_q^A from the oracle with the geometry of every point) or 1e-12 (FP64),
the CSR pattern bit-exact, the assembled CSR within the bound of Corollary
4.11 and equal to the assembly of the GPU's own element matrices.  The
meshes span two tiles of 128 cells with a ragged second one.
"""
import numpy as np
import pytest

import oracle
from paper_2410_12614_gb300 import api, inputs

from gpu_util import FP64_TOL, cell_bounds, cell_errors, csr_bound, cuda, to_np

pytestmark = pytest.mark.gpu

ALL = ("bf16", "fp16", "tf32", "tf32x3", "e4m3")
CASES = [("hexahedron", 6, 1), ("hexahedron", 6, 2), ("hexahedron", 6, 3), ("hexahedron", 5, 4),
         ("hexahedron", 5, 5), ("quadrilateral", 12, 1), ("quadrilateral", 12, 3), ("quadrilateral", 12, 6),
         ("quadrilateral", 12, 8)]


@pytest.mark.parametrize("cell,n,p", CASES)
def test_boxed_cells_every_format(cell, n, p):
    v, c = inputs.structured_mesh(cell, n, 0.15, 200 + p)
    pts, w = api.quadrature_rule(cell, p + 1)
    plan = api.Plan(cell, v, c, p, pts, w, precisions=ALL)
    ref = oracle.Problem(v, c, p, *oracle.rule_for_degree(cell, p))
    assert plan.n_phi == (p + 1) ** ref.d and plan.n_dofs == ref.n_dofs
    rp, ci = plan.csr_pattern()
    orp, oci = ref.csr_pattern()
    assert np.array_equal(rp.cpu().numpy(), orp) and np.array_equal(ci.cpu().numpy(), oci)
    kap = inputs.lognormal_kappa(plan.n_cells, plan.n_q, 300 + p)
    kd = cuda(kap)
    worst = {}
    for form in ("stiffness", "mass"):
        A = ref.element_matrices(kap, form)
        g_exact = ref.assemble(A)
        for prec in ("fp64",) + ALL:
            els = plan.element_matrices(kd, forms=(form,), prec=prec)
            vals = plan.assemble(kd, forms=(form,), prec=prec)
            plan.sync()
            got, gv = to_np(els[form]), to_np(vals[form])
            err = cell_errors(got, A)
            if prec == "fp64":
                assert err.max() <= FP64_TOL, (form, float(err.max()))
                assert np.abs(gv - g_exact).max() <= FP64_TOL * np.abs(g_exact).max()
            else:
                bnd = cell_bounds(ref, kap, form, prec, A)
                worst[(form, prec)] = float((err / bnd).max())
                assert np.all(err <= bnd), (form, prec, float((err / bnd).max()))
                assert np.all(np.abs(gv - g_exact) <= csr_bound(ref, A, bnd)), (form, prec)
            own = ref.assemble(got)
            assert np.abs(gv - own).max() <= (1e-13 if prec == "fp64" else 1e-5) * np.abs(g_exact).max()
    print(cell, p, {k: round(x, 3) for k, x in worst.items()})


def test_boxed_assembly_deterministic_and_host_path():
    v, c = inputs.hex_mesh(6, 0.15, 7)
    plan = api.Plan("hexahedron", v, c, 2, precisions=("bf16",))
    kap = inputs.lognormal_kappa(plan.n_cells, plan.n_q, 8)
    kd = cuda(kap)
    a = plan.assemble(kd, prec="bf16")
    b = plan.assemble(kd, prec="bf16")
    plan.sync()
    import torch
    kh = torch.from_numpy(kap).pin_memory()
    h = plan.assemble_host(kh, prec="bf16")
    for f in a:
        assert torch.equal(a[f], b[f])
        assert torch.equal(a[f].cpu(), h[f])


def test_boxed_rejects_simplex_only_calls():
    v, c = inputs.quad_mesh(3, 0.1, 9)
    plan = api.Plan("quadrilateral", v, c, 2, precisions=("bf16",))
    kd = cuda(inputs.lognormal_kappa(plan.n_cells, plan.n_q, 10))
    w = cuda(np.ones(plan.n_dofs))
    with pytest.raises(api._lib.FeError) as e:
        plan.action(kd, w, prec="bf16")
    assert e.value.status == -2


def test_elements_only_plan():
    # FE_PLAN_ELEMENTS_ONLY: the same element matrices without a dof map or
    # pattern; calls that need them are rejected
    v, c = inputs.hex_mesh(5, 0.15, 11)
    full = api.Plan("hexahedron", v, c, 3, precisions=("bf16",))
    lean = api.Plan("hexahedron", v, c, 3, precisions=("bf16",), elements_only=True)
    assert lean.n_dofs == 0 and lean.nnz == 0
    kd = cuda(inputs.lognormal_kappa(full.n_cells, full.n_q, 12))
    import torch
    for prec in ("bf16", "fp64"):
        a = full.element_matrices(kd, prec=prec)
        b = lean.element_matrices(kd, prec=prec)
        full.sync()
        lean.sync()
        for f in a:
            assert torch.equal(a[f], b[f])
    with pytest.raises(api._lib.FeError) as e:
        lean.assemble(kd, prec="bf16")
    assert e.value.status == -1
