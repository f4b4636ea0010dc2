"""GPU linear forms (Algorithm 2, fe_action) against the oracle.

FP64: cell vectors and the assembled vector within 1e-12 of the oracle's
Algorithm 2.  Mixed (TF32, BF16, FP16): B, the cell coefficients and r_s
rounded once to the storage format (Sec. 4.5: the casting remark and the
theorem on r_s), the rest FP32 -- each cell-vector entry within
(4 u_s + gamma_K(2 u_32)) * M of the exact one, M the magnitude
sum_{s,q} |B_sjq| sum_t |w_q z G_st| sum_k |B_tkq| |w_k| (a componentwise
rounding bound for the two chained sums), and the assembled vector within the
sum of those over its cells plus its own FP32 summation.  The vector assembly is
bitwise deterministic.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2410_12614_gb300 import api, inputs

from gpu_util import cuda, make_case, to_np

pytestmark = pytest.mark.gpu

U_S = {"tf32": 2.0 ** -11, "bf16": 2.0 ** -8, "fp16": 2.0 ** -11}
# thread-per-cell kernel: P1-P8 triangles, P1-P5 tetrahedra (162 cells: a ragged
# last CTA; P3/P5 tetrahedra: several quadrature windows); warp-per-cell
# kernel for the larger elements: P6 tetrahedra, P9 triangles
CASES = [("triangle", 3, 1), ("triangle", 2, 4), ("tetrahedron", 2, 1), ("tetrahedron", 3, 2), ("tetrahedron", 3, 3),
         ("tetrahedron", 1, 5), ("tetrahedron", 1, 6), ("triangle", 2, 9)]


@pytest.mark.parametrize("cell,n,p", CASES)
def test_action_matches_oracle(cell, n, p):
    plan, ref, kap = make_case(cell, n, p, 0.15, 110 + p, 111 + p, precisions=("bf16",))
    w = inputs.gaussian_vector(plan.n_dofs, 112 + p).astype(np.float64)
    kd, wd = cuda(kap), cuda(w)
    dofs, _ = ref.cell_dofs()
    for form in ("stiffness", "mass"):
        b_ex, M = ref.action(kap, w, form, with_magnitude=True)
        v_ex = ref.assemble_vector(b_ex)
        K = ref.n_q * (ref.d if form == "stiffness" else 1) + ref.n_phi
        for prec in ("fp64", "tf32", "bf16", "fp16"):
            v, b = plan.action(kd, wd, forms=(form,), prec=prec, cell_vectors=True)
            plan.sync()
            bg, vg = to_np(b[form]), to_np(v[form])
            if prec == "fp64":
                assert np.abs(bg - b_ex).max() <= 1e-12 * np.abs(b_ex).max()
                assert np.abs(vg - v_ex).max() <= 1e-12 * np.abs(b_ex).max()
            else:
                x = K * 2 * 2.0 ** -23
                # four storage roundings reach b: w^c and B in grad w, r_s, B in b
                tol = (4 * U_S[prec] + x / (1 - x) + 8 * 2.0 ** -24) * M
                assert np.all(np.abs(bg - b_ex) <= tol), (form, prec, float((np.abs(bg - b_ex) / tol).max()))
                vt = ref.assemble_vector(tol) + 32 * 2.0 ** -24 * ref.assemble_vector(np.abs(b_ex))
                assert np.all(np.abs(vg - v_ex) <= vt), (form, prec)
            # the GPU's own vector assembly of its cell vectors
            assert np.abs(vg - ref.assemble_vector(bg)).max() <= (1e-13 if prec == "fp64" else 1e-5) * np.abs(b_ex).max()


def test_action_deterministic_and_outputs():
    plan, ref, kap = make_case("tetrahedron", 3, 2, 0.15, 120, 121, precisions=("bf16",))
    w = cuda(inputs.gaussian_vector(plan.n_dofs, 122).astype(np.float64))
    kd = cuda(kap)
    v1 = plan.action(kd, w, prec="bf16")
    v2 = plan.action(kd, w, prec="bf16")
    plan.sync()
    for f in ("stiffness", "mass"):
        assert torch.equal(v1[f], v2[f])
    with pytest.raises(Exception):
        plan.action(kd, w, prec="e4m3")


def test_action_status_codes():
    # non-finite kappa -> FE_ERR_NONFINITE; a cell of zero volume -> FE_ERR_DEGENERATE_CELL
    v, c = inputs.cube_mesh(2, 0.1, 1)
    pts, w = api.quadrature_rule("tetrahedron", 3)
    plan = api.Plan("tetrahedron", v, c, 2, pts, w, precisions=("bf16",))
    wd = cuda(inputs.gaussian_vector(plan.n_dofs, 130).astype(np.float64))
    for prec in ("bf16", "fp64"):
        kap = inputs.lognormal_kappa(plan.n_cells, plan.n_q, 131)
        kap[7, 2] = np.inf
        plan.action(cuda(kap), wd, prec=prec)
        with pytest.raises(api._lib.FeError) as e:
            plan.sync()
        assert e.value.status == -4
        plan.sync()   # the status word was cleared
        verts = torch.from_numpy(v.copy()).cuda()
        verts[c[0][3]] = verts[c[0][0]]   # two vertices of cell 0 coincide: det J == 0
        plan.action(cuda(inputs.lognormal_kappa(plan.n_cells, plan.n_q, 132)), wd, prec=prec, vertices=verts)
        with pytest.raises(api._lib.FeError) as e:
            plan.sync()
        assert e.value.status in (-3, -4)
        plan.sync()
