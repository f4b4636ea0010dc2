"""The two assembly algorithms give bitwise the same CSR values: the chunked
segmented reduction (the default) and the row-wise kernel (one warp per CSR
row; fe_plan_set_assembly), both summing every value's element entries
in increasing cell order from zero -- on tetrahedra, triangles with a row
above the row kernel's shared-memory cap (the fan's centre row), boxed cells,
FP64 and reduced precision, and inside a batch."""
import numpy as np
import pytest
import torch

from paper_2410_12614_gb300 import api, inputs

from gpu_util import cuda

pytestmark = pytest.mark.gpu


def _fan(n_tri):
    ang = 2 * np.pi * np.arange(n_tri) / n_tri
    v = np.vstack([[0.0, 0.0], np.c_[np.cos(ang), np.sin(ang)]])
    c = np.array([[0, 1 + i, 1 + (i + 1) % n_tri] for i in range(n_tri)], dtype=np.int32)
    return v, c


@pytest.mark.parametrize("case", ["tet_p3", "tri_fan_p5", "hex_p2", "tet_p1_big", "tet_p5", "hex_p4", "tri_p8"])
def test_row_and_chunked_assembly_bitwise_equal(case):
    if case == "tet_p3":
        v, c = inputs.cube_mesh(8, 0.15, 1)
        cell, p = "tetrahedron", 3
    elif case == "tri_fan_p5":
        v, c = _fan(200)
        cell, p = "triangle", 5
    elif case == "hex_p2":
        v, c = inputs.hex_mesh(6, 0.15, 2)
        cell, p = "hexahedron", 2
    elif case == "tet_p1_big":
        v, c = inputs.cube_mesh(20, 0.15, 3)
        cell, p = "tetrahedron", 1
    elif case == "tet_p5":            # n_phi = 56: two 32-column blocks per element row
        v, c = inputs.cube_mesh(3, 0.15, 4)
        cell, p = "tetrahedron", 5
    elif case == "hex_p4":            # n_phi = 125: four blocks
        v, c = inputs.hex_mesh(3, 0.15, 5)
        cell, p = "hexahedron", 4
    else:                             # n_phi = 45
        v, c = inputs.square_mesh(6, 0.2, 6)
        cell, p = "triangle", 8
    plan = api.Plan(cell, v, c, p, precisions=("bf16",))
    if case == "tri_fan_p5":
        rp, _ = plan.csr_pattern()
        assert int(torch.diff(rp).max()) > 512           # the centre row takes the global path
    kd = cuda(inputs.lognormal_kappa(plan.n_cells, plan.n_q, 9))
    for prec in ("bf16", "fp64"):
        els = plan.element_matrices(kd, prec=prec)
        plan.set_assembly(1)
        rows = plan.assemble_elements(els, prec=prec)
        plan.set_assembly(0)
        chunks = plan.assemble_elements(els, prec=prec)
        plan.set_assembly(0)
        plan.sync()
        for f in ("stiffness", "mass"):
            assert torch.equal(rows[f], chunks[f]), (case, prec, f)


def test_batch_row_assembly_matches_single_plans():
    plans, kaps = [], []
    for i, (cell, n, p) in enumerate([("tetrahedron", 4, 2), ("triangle", 20, 3), ("tetrahedron", 3, 4)]):
        v, c = inputs.structured_mesh(cell, n, 0.15, 20 + i)
        pl = api.Plan(cell, v, c, p, precisions=("bf16",))
        pl.set_assembly(1)
        plans.append(pl)
        kaps.append(cuda(inputs.lognormal_kappa(pl.n_cells, pl.n_q, 30 + i)))
    stream = torch.cuda.Stream()
    b = api.Batch(plans, kaps, prec="bf16", stream=stream)
    b.run()
    b.sync()
    for pl, k, i in zip(plans, kaps, range(len(plans))):
        single = pl.assemble(k, prec="bf16")
        pl.sync()
        for f in ("stiffness", "mass"):
            assert torch.equal(b.values[f][i], single[f]), (i, f)
