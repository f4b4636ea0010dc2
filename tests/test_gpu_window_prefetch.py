"""The builders' window prefetch of the tensor-core element kernel
(fe_plan_set_window_prefetch) changes where a coefficient window is read from,
shared memory filled by asynchronous copies instead of L2, never what is
computed: element matrices with the prefetch forced on are bitwise those with
it off and those of the autotuned choice, in every reduced format, for
tetrahedra whose quadrature points span several windows and for boxed cells,
whose geometry gives every pair its own window.  fe_plan_tc_config confirms
that the forced-on launches really carry the prefetch slot.
"""
import pytest
import torch

from paper_2410_12614_gb300 import api, inputs

from gpu_util import cuda

pytestmark = pytest.mark.gpu

CASES = [
    # P6 tetrahedra: 343 points, 6 windows of 64 (11 of 32 for the TF32 formats)
    ("tetrahedron", 6, ("bf16", "fp16", "e4m3", "tf32", "tf32x3")),
    # Q1 hexahedra: 8 points, but 7 windows per cell (6 pairs and the mass form)
    ("hexahedron", 1, ("bf16", "e4m3", "tf32x3")),
    # Q2 quadrilaterals: 9 points, 4 windows per cell
    ("quadrilateral", 2, ("bf16", "fp16")),
]


def _mesh(cell):
    if cell == "tetrahedron":
        return inputs.cube_mesh(3, 0.15, 3)      # 162 cells: two tiles, the second ragged
    if cell == "hexahedron":
        return inputs.hex_mesh(6, 0.15, 5)       # 216 cells
    return inputs.quad_mesh(14, 0.1, 5)          # 196 cells


@pytest.mark.parametrize("cell,p,precs", CASES)
def test_prefetch_same_bits(cell, p, precs):
    v, c = _mesh(cell)
    pts, w = api.quadrature_rule(cell, p + 1)
    plan = api.Plan(cell, v, c, p, pts, w, precisions=precs, elements_only=True)
    kap = cuda(inputs.lognormal_kappa(plan.n_cells, plan.n_q, 8))
    for prec in precs:
        got = {}
        for mode in (0, 1, -1):
            plan.set_window_prefetch(mode)
            cfg = plan.tc_config(prec=prec)
            if mode == 1:
                assert cfg["win_buf"] == 1, (prec, cfg)
            if mode == 0:
                assert cfg["win_buf"] == 0, (prec, cfg)
            els = plan.element_matrices(kap, prec=prec)
            plan.sync()
            got[mode] = {f: t.clone() for f, t in els.items()}
        for f in ("stiffness", "mass"):
            assert torch.isfinite(got[0][f]).all()
            assert torch.equal(got[1][f], got[0][f]), (prec, f)
            assert torch.equal(got[-1][f], got[0][f]), (prec, f)
