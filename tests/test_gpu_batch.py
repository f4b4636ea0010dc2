"""Batched persistent launch (fe_batch_*): uneven meshes of triangles and
tetrahedra of several degrees in one graph-captured launch, against the FP64
oracle on sampled cells and against the single-plan calls bit for bit.
The full workload is 256 meshes with cell counts log-uniform in 1e3..2e5,
triangles p = 1..6 and tetrahedra p = 1..5, kappa lognormal(0,1), BF16."""
import numpy as np
import pytest
import torch

import oracle
from paper_2410_12614_gb300 import api, inputs

from gpu_util import cell_bounds, cell_errors, cuda, to_np

pytestmark = pytest.mark.gpu


def _plans(descs, precisions=("bf16",)):
    plans, refs, kaps = [], [], []
    for i, x in enumerate(descs):
        v, c = inputs.structured_mesh(x["cell_type"], x["n"], x["alpha"], x["seed"])
        p = x["degree"]
        pts, w = api.quadrature_rule(x["cell_type"], p + 1)
        plan = api.Plan(x["cell_type"], v, c, p, pts, w, precisions=precisions, stream=torch.cuda.current_stream())
        kap = inputs.lognormal_kappa(plan.n_cells, plan.n_q, 500 + i)
        plans.append(plan)
        kaps.append(kap)
        refs.append((v, c, p, x["cell_type"]))
    return plans, refs, kaps


def _check_sampled(ref, kap, got, form, prec, rng, k=4):
    v, c, p, cell = ref
    pr = oracle.Problem(v, c, p, *oracle.rule_for_degree(cell, p))
    ids = np.unique(np.concatenate([rng.choice(len(c), size=min(k, len(c)), replace=False), [0, len(c) - 1]]))
    A = pr.element_matrices_subset(kap, form, ids)
    err = cell_errors(got[ids], A)
    bnd = cell_bounds(pr, kap, form, prec, A, cell_ids=ids)
    assert np.all(err <= bnd), (cell, p, form, float(err.max()), float(bnd.min()))


def test_small_mixed_batch_matches_single_plans_and_oracle():
    descs = [dict(cell_type="triangle", degree=1, n=5, alpha=0.2, seed=1),
             dict(cell_type="tetrahedron", degree=3, n=3, alpha=0.15, seed=2),
             dict(cell_type="triangle", degree=6, n=4, alpha=0.2, seed=3),
             dict(cell_type="tetrahedron", degree=5, n=2, alpha=0.15, seed=4),
             dict(cell_type="tetrahedron", degree=1, n=4, alpha=0.15, seed=5),
             dict(cell_type="triangle", degree=3, n=7, alpha=0.2, seed=6)]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        plans, refs, kaps = _plans(descs, precisions=("bf16", "fp16"))
        kd = [cuda(k) for k in kaps]
        rng = np.random.default_rng(0)
        for prec in ("bf16", "fp16", "fp64"):
            batch = api.Batch(plans, kd, prec=prec, stream=stream)
            batch.run()
            batch.run()
            batch.sync()
            for i, plan in enumerate(plans):
                els = {f: plan.empty_elements(prec) for f in ("stiffness", "mass")}
                single = plan.assemble(kd[i], prec=prec, elements=els)
                plan.sync()
                for f in ("stiffness", "mass"):
                    assert torch.equal(batch.elements[f][i], els[f]), (i, prec, f)
                    assert torch.equal(batch.values[f][i], single[f]), (i, prec, f)
                    if prec != "fp64":
                        _check_sampled(refs[i], kaps[i], to_np(batch.elements[f][i]), f, prec, rng)
            batch.close()


def test_batched_workload_256_meshes_bf16():
    descs = inputs.batched_workload()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        plans, refs, kaps = _plans(descs)
        kd = [cuda(k) for k in kaps]
        batch = api.Batch(plans, kd, prec="bf16", stream=stream)
        assert batch.n_cells == sum(p.n_cells for p in plans) > 9_000_000
        assert batch.launches == 3   # factor, element and assembly kernels
        batch.run()
        batch.sync()
        rng = np.random.default_rng(1)
        for i in rng.choice(len(plans), size=24, replace=False):
            for f in ("stiffness", "mass"):
                _check_sampled(refs[i], kaps[i], to_np(batch.elements[f][i]), f, "bf16", rng, k=3)
        # assembly of a few small meshes against the oracle's assembly of the GPU element matrices
        small = sorted(range(len(plans)), key=lambda i: plans[i].n_cells)[:6]
        for i in small:
            v, c, p, cell = refs[i]
            pr = oracle.Problem(v, c, p, *oracle.rule_for_degree(cell, p))
            for f in ("stiffness", "mass"):
                g = pr.assemble(to_np(batch.elements[f][i]))
                gv = to_np(batch.values[f][i])
                assert np.abs(gv - g).max() <= 24 * 2.0 ** -23 * np.abs(g).max()
        batch.close()
