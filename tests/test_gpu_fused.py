"""Fused assembly (fe_assemble without element-matrix outputs): cells in
slices of one wave of tiles, element matrices in a ring that stays in L2, rows
assembled as soon as their last cell is done.  The CSR values must be bitwise
those of the unfused path (element matrices written out, then assembled) for
every reduced-precision format, on meshes spanning several slices."""
import numpy as np
import pytest
import torch

import oracle
from paper_2410_12614_gb300 import api, inputs

from gpu_util import cell_bounds, csr_bound, cuda, to_np

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cell,n,p", [("tetrahedron", 16, 2), ("tetrahedron", 24, 1), ("triangle", 150, 3),
                                      ("tetrahedron", 12, 3)])
def test_fused_assembly_bitwise_equal_to_unfused(cell, n, p):
    v, c = inputs.structured_mesh(cell, n, 0.15, 500 + p)
    precs = ("bf16", "fp16", "e4m3")
    plan = api.Plan(cell, v, c, p, precisions=precs)
    active = plan.set_fusion(1)
    kap = inputs.lognormal_kappa(plan.n_cells, plan.n_q, 600 + p)
    kd = cuda(kap)
    for prec in precs:
        fused = plan.assemble(kd, prec=prec)
        els = {f: plan.empty_elements(prec) for f in ("stiffness", "mass")}
        unfused = plan.assemble(kd, prec=prec, elements=els)
        plan.sync()
        for f in ("stiffness", "mass"):
            assert torch.equal(fused[f], unfused[f]), (prec, f)
        plan.set_fusion(0)
        off = plan.assemble(kd, prec=prec)
        plan.sync()
        plan.set_fusion(1)
        for f in ("stiffness", "mass"):
            assert torch.equal(off[f], unfused[f]), (prec, f)
    print(cell, n, p, "cells", plan.n_cells, "fused path active:", active)
    if cell == "tetrahedron" and n == 16:
        assert active                          # 24,576 cells, two slices, a 31 MB ring
    if cell == "tetrahedron" and n == 12 and p == 3:
        # the oracle on a sample of rows: the fused values within the bound of Corollary 4.11
        ref = oracle.Problem(v, c, p, *oracle.rule_for_degree(cell, p))
        A = ref.element_matrices(kap, "stiffness")
        bnd = cell_bounds(ref, kap, "stiffness", "bf16", A)
        fused = plan.assemble(kd, forms=("stiffness",), prec="bf16")["stiffness"]
        plan.sync()
        assert np.all(np.abs(to_np(fused) - ref.assemble(A)) <= csr_bound(ref, A, bnd))
