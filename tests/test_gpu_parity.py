"""GPU parity of element matrices and CSR assembly against the FP64 oracle.

FP64 path: max per-cell relative error <= 1e-12 and global <= 1e-12.
Reduced precision: per-cell error within the bound of Theorem 4.8 /
Corollary 4.10 evaluated by the oracle (kappa_q^A per cell), CSR within the
entrywise bound of Corollary 4.11.  Sparsity pattern and dof map: bit-exact.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2410_12614_gb300 import api, inputs

from gpu_util import FP64_TOL, cell_bounds, cell_errors, csr_bound, cuda, make_case, to_np

pytestmark = pytest.mark.gpu

ALL_LOW = ("bf16", "fp16", "tf32", "tf32x3", "e4m3")

SMALL_CASES = [
    ("triangle", 3, 1), ("triangle", 3, 3), ("triangle", 2, 5), ("triangle", 2, 6),
    ("tetrahedron", 2, 1), ("tetrahedron", 2, 2), ("tetrahedron", 3, 3), ("tetrahedron", 2, 4),
    ("tetrahedron", 1, 5),
]


@pytest.mark.parametrize("cell,n,p", SMALL_CASES)
def test_small_meshes_all_precisions(cell, n, p):
    plan, ref, kap = make_case(cell, n, p, 0.15, 11 + p, 12 + p, precisions=ALL_LOW)
    kd = cuda(kap)
    # pattern and dof map bit-exact
    rp, ci = plan.csr_pattern()
    orp, oci = ref.csr_pattern()
    assert np.array_equal(rp.cpu().numpy(), orp) and np.array_equal(ci.cpu().numpy(), oci)
    assert np.array_equal(plan.cell_dofs().cpu().numpy(), ref.cell_dofs()[0])
    for form in ("stiffness", "mass"):
        A = ref.element_matrices(kap, form)
        g_exact = ref.assemble(A)
        for prec in ("fp64",) + ALL_LOW:
            els = plan.element_matrices(kd, forms=(form,), prec=prec)
            vals = plan.assemble(kd, forms=(form,), prec=prec)
            plan.sync()
            got = to_np(els[form])
            err = cell_errors(got, A)
            gv = to_np(vals[form])
            if prec == "fp64":
                assert err.max() <= FP64_TOL, (form, prec, err.max())
                assert np.abs(gv - g_exact).max() <= FP64_TOL * np.abs(g_exact).max()
            else:
                bnd = cell_bounds(ref, kap, form, prec, A)
                assert np.all(err <= bnd), (form, prec, float(err.max()), float(bnd[np.argmax(err / bnd)]))
                gb = csr_bound(ref, A, bnd)
                assert np.all(np.abs(gv - g_exact) <= gb), (form, prec, "csr")
            # assembly of the GPU's own element matrices, checked by the oracle's assembly
            assert np.abs(gv - ref.assemble(got)).max() <= (1e-13 if prec == "fp64" else 1e-5) * np.abs(g_exact).max()


def test_ragged_tail_and_single_cell():
    # 6*3^3 = 162 cells: one full tile of 128 and a ragged tail of 34
    for n_cells_mesh in (3, 1):
        plan, ref, kap = make_case("tetrahedron", n_cells_mesh, 3, 0.15, 5, 6, precisions=("bf16",))
        kd = cuda(kap)
        for form in ("stiffness", "mass"):
            A = ref.element_matrices(kap, form)
            got = to_np(plan.element_matrices(kd, forms=(form,), prec="bf16")[form])
            assert np.all(cell_errors(got, A) <= cell_bounds(ref, kap, form, "bf16", A))
    # a single triangle
    v = np.array([[0.0, 0.0], [1.0, 0.1], [0.2, 0.9]])
    c = np.array([[0, 1, 2]], dtype=np.int32)
    pts, w = api.quadrature_rule("triangle", 3)
    plan = api.Plan("triangle", v, c, 2, pts, w, precisions=("fp16",))
    ref = oracle.Problem(v, c, 2, *oracle.collapsed_rule("triangle", 3))
    kap = inputs.lognormal_kappa(1, plan.n_q, 1)
    for prec in ("fp64", "fp16"):
        got = to_np(plan.element_matrices(cuda(kap), forms=("stiffness",), prec=prec)["stiffness"])
        A = ref.element_matrices(kap, "stiffness")
        tol = FP64_TOL if prec == "fp64" else cell_bounds(ref, kap, "stiffness", prec, A)
        assert np.all(cell_errors(got, A) <= tol)


def test_deterministic_and_host_path_matches():
    plan, ref, kap = make_case("tetrahedron", 4, 3, 0.15, 7, 8, precisions=("bf16",))
    kd = cuda(kap)
    a = plan.assemble(kd, prec="bf16")
    b = plan.assemble(kd, prec="bf16")
    h = plan.assemble_host(torch.from_numpy(kap).pin_memory(), prec="bf16")
    for f in ("stiffness", "mass"):
        assert torch.equal(a[f], b[f])
        assert torch.equal(a[f].cpu(), h[f])


def test_status_codes_for_bad_inputs():
    v, c = inputs.cube_mesh(2, 0.1, 1)
    pts, w = api.quadrature_rule("tetrahedron", 3)
    plan = api.Plan("tetrahedron", v, c, 2, pts, w, precisions=("bf16",))
    kap = inputs.lognormal_kappa(plan.n_cells, plan.n_q, 2)
    kap[5, 3] = np.nan
    plan.element_matrices(cuda(kap), prec="bf16")
    with pytest.raises(api._lib.FeError) as e:
        plan.sync()
    assert e.value.status == -4
    # degenerate cell: collapse one cell's vertices onto a plane through the vertex array override
    verts = torch.from_numpy(v.copy()).cuda()
    cell0 = c[0]
    verts[cell0[3]] = verts[cell0[0]]  # two vertices of cell 0 coincide: det J == 0 exactly
    plan.element_matrices(cuda(inputs.lognormal_kappa(plan.n_cells, plan.n_q, 2)), prec="fp64", vertices=verts)
    with pytest.raises(api._lib.FeError) as e:
        plan.sync()
    assert e.value.status in (-3, -4)
    plan.sync()  # the status word was cleared
    with pytest.raises(ValueError):
        plan.element_matrices(cuda(kap[:, :2].copy()), prec="bf16")
    # precision not prepared by the plan
    with pytest.raises(api._lib.FeError) as e:
        plan.element_matrices(cuda(inputs.lognormal_kappa(plan.n_cells, plan.n_q, 2)), prec="fp16")
    assert e.value.status == -1
