"""fe_assemble_host_many: a sequence of host coefficient sets with uploads,
computation and downloads overlapped, bitwise equal to one fe_assemble_host
call per item (including an output buffer reused two items later)."""
import numpy as np
import pytest
import torch

from paper_2410_12614_gb300 import api, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["bf16", "fp64"])
def test_pipelined_host_assembly_matches_single_calls(prec):
    v, c = inputs.cube_mesh(6, 0.15, 31)
    plan = api.Plan("tetrahedron", v, c, 2, precisions=("bf16",))
    kaps = [torch.from_numpy(inputs.lognormal_kappa(plan.n_cells, plan.n_q, 40 + i)).pin_memory() for i in range(5)]
    dt = torch.float64 if prec == "fp64" else torch.float32
    outs = [{f: torch.empty(plan.nnz, dtype=dt, pin_memory=True) for f in ("stiffness", "mass")} for _ in range(3)]
    # items 0..4 write outs[0], outs[1], outs[2], outs[0], outs[1]: the first two are overwritten later
    seq = [outs[i % 3] for i in range(5)]
    plan.assemble_host_many(kaps, seq, prec=prec)
    for i in (2, 3, 4):
        ref = plan.assemble_host(kaps[i], prec=prec)
        for f in ("stiffness", "mass"):
            assert torch.equal(seq[i][f], ref[f]), (i, f)
    # one form only, and a second sequence on the same plan
    only = [{"stiffness": torch.empty(plan.nnz, dtype=dt, pin_memory=True)} for _ in range(2)]
    plan.assemble_host_many(kaps[:2], only, forms=("stiffness",), prec=prec)
    for i in range(2):
        assert torch.equal(only[i]["stiffness"], plan.assemble_host(kaps[i], forms=("stiffness",), prec=prec)["stiffness"])


@pytest.mark.parametrize("cell,n,p,prec,forms", [
    ("tetrahedron", 10, 3, "bf16", ("stiffness", "mass")),
    ("tetrahedron", 8, 2, "fp64", ("stiffness",)),
    ("triangle", 40, 4, "fp16", ("mass",)),
])
def test_single_call_ranges_bitwise(cell, n, p, prec, forms):
    """fe_assemble_host sums the CSR rows in ranges and downloads each range
    while the next is summed: the host values are bitwise those of the device
    call, for both forms or one, in FP64 and the reduced formats."""
    import torch
    v, c = inputs.structured_mesh(cell, n, 0.15, 31)
    pts, w = api.quadrature_rule(cell, p + 1)
    plan = api.Plan(cell, v, c, p, pts, w, precisions=("bf16",) if prec == "fp64" else (prec,))
    kap = inputs.lognormal_kappa(plan.n_cells, plan.n_q, 32)
    dev = plan.assemble(torch.from_numpy(kap).cuda(), forms=forms, prec=prec)
    host = plan.assemble_host(torch.from_numpy(kap).pin_memory(), forms=forms, prec=prec)
    plan.sync()
    for f in forms:
        assert torch.equal(dev[f].cpu(), host[f]), f
