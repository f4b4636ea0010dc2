"""Wide full-row passes of the tensor-core contraction (fe_plan_set_rows_per_pass
with rows * n_phi > 256): both halves of the tensor memory form one 512-column
accumulator and each coefficient chunk feeds two MMAs.  The element matrices
must agree with the narrow whole-row layout (two 256-column accumulators, staged
epilogue) to FP32 accumulation order, and with the FP64 oracle within the
per-cell bound of Corollary 4.10.  Cases: P5 tetrahedra (9 rows, 504 columns),
P6 tetrahedra (6 rows, 504 columns) and Q3 hexahedra (8 rows: exactly 512, the
second MMA 256 columns wide), ragged last tiles.
"""
import numpy as np
import pytest

import oracle
from paper_2410_12614_gb300 import api, inputs

from gpu_util import cell_bounds, cell_errors, cuda, to_np

pytestmark = pytest.mark.gpu

CASES = [("tetrahedron", 5, 9, 4, ("bf16", "e4m3", "tf32x3")),
         ("tetrahedron", 6, 6, 2, ("bf16",)),
         ("hexahedron", 3, 8, 3, ("bf16", "fp16"))]


@pytest.mark.parametrize("cell,p,wide_rows,narrow_rows,precs", CASES)
def test_wide_passes_match(cell, p, wide_rows, narrow_rows, precs):
    if cell == "tetrahedron":
        v, c = inputs.cube_mesh(3, 0.15, 13)        # 162 cells
    else:
        v, c = inputs.hex_mesh(5, 0.15, 13)         # 125 cells
    pts, w = api.quadrature_rule(cell, p + 1)
    plan = api.Plan(cell, v, c, p, pts, w, precisions=precs, elements_only=True)
    kap = inputs.lognormal_kappa(plan.n_cells, plan.n_q, 21)
    kd = cuda(kap)
    ref = oracle.Problem(v, c, p, *oracle.rule_for_degree(cell, p))
    exact = {f: ref.element_matrices(kap, f) for f in ("stiffness", "mass")}
    assert wide_rows * plan.n_phi > 256
    for prec in precs:
        got = {}
        for rows in (narrow_rows, wide_rows):
            plan.set_rows_per_pass(rows, prec=prec)
            cfg = plan.tc_config(prec=prec)
            assert cfg["n_acc"] == (1 if rows == wide_rows else 2), cfg
            els = plan.element_matrices(kd, prec=prec)
            plan.sync()
            got[rows] = {f: to_np(t) for f, t in els.items()}
        for f in ("stiffness", "mass"):
            a, b = got[wide_rows][f], got[narrow_rows][f]
            scale = np.abs(exact[f]).reshape(len(a), -1).max(axis=1)
            diff = np.abs(a - b).reshape(len(a), -1).max(axis=1)
            assert (diff <= 2.0 ** -18 * scale).all(), (prec, f, (diff / scale).max())
            err = cell_errors(a, exact[f])
            bound = cell_bounds(ref, kap, f, prec, exact[f])
            assert (err <= bound).all(), (prec, f, (err / bound).max())
