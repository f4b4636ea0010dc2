"""Parity at the workload sizes: P1 Laplace on 32^2 x 2 triangles (FP64, all
cells), P3 stiffness + mass on 24^3 x 6 tetrahedra (BF16, FP16, FP64; sampled
cells against the oracle, the full CSR against the oracle's assembly of the
GPU element matrices, pattern bit-exact), and the degree sweep p = 1..8 on
16^3 x 6 tetrahedra in every precision on sampled cells.  The launch
configuration is the one the benchmark times."""
import numpy as np
import pytest

import oracle
from paper_2410_12614_gb300 import api, inputs

from gpu_util import FP64_TOL, cell_bounds, cell_errors, cuda, to_np

pytestmark = pytest.mark.gpu


def _sample(n_cells, k, seed):
    rng = np.random.default_rng(seed)
    ids = set(rng.choice(n_cells, size=min(k, n_cells), replace=False).tolist())
    ids |= {0, 1, 127, 128, n_cells - 1, n_cells - 2}  # tile edges and the ragged tail
    return np.array(sorted(i for i in ids if 0 <= i < n_cells))


def test_p1_laplace_triangles_fp64_all_cells():
    v, c = inputs.square_mesh(32, 0.2, 1)
    pts, w = api.quadrature_rule("triangle", 0, family=api._lib.FE_QUAD_TRIANGLE_3POINT)
    plan = api.Plan("triangle", v, c, 1, pts, w, forms=("stiffness",), precisions=("bf16",))
    assert (plan.n_cells, plan.n_vertices, plan.n_dofs, plan.nnz) == (2048, 1089, 1089, 7361)
    ref = oracle.Problem(v, c, 1, *oracle.strang_fix_3())
    kap = np.ones((plan.n_cells, 3))
    el = plan.element_matrices(cuda(kap), forms=("stiffness",), prec="fp64")
    vals = plan.assemble(cuda(kap), forms=("stiffness",), prec="fp64")
    plan.sync()
    A = ref.element_matrices(kap, "stiffness")
    assert cell_errors(to_np(el["stiffness"]), A).max() <= FP64_TOL
    g = ref.assemble(A)
    assert np.abs(to_np(vals["stiffness"]) - g).max() <= FP64_TOL * np.abs(g).max()
    rp, ci = plan.csr_pattern()
    orp, oci = ref.csr_pattern()
    assert np.array_equal(rp.cpu().numpy(), orp) and np.array_equal(ci.cpu().numpy(), oci)


@pytest.fixture(scope="module")
def p3_case():
    v, c = inputs.cube_mesh(24, 0.15, 2)
    pts, w = api.quadrature_rule("tetrahedron", 4)
    plan = api.Plan("tetrahedron", v, c, 3, pts, w, precisions=("bf16", "fp16"))
    kap = inputs.lognormal_kappa(plan.n_cells, plan.n_q, 3)
    ref = oracle.Problem(v, c, 3, *oracle.collapsed_rule("tetrahedron", 4))
    return plan, ref, kap


def test_p3_tets_pattern_and_sizes(p3_case):
    plan, ref, _ = p3_case
    assert (plan.n_cells, plan.n_dofs, plan.nnz, plan.n_phi, plan.n_q) == (82944, 389017, 18388729, 20, 64)
    rp, ci = plan.csr_pattern()
    orp, oci = ref.csr_pattern()
    assert np.array_equal(rp.cpu().numpy(), orp)
    assert np.array_equal(ci.cpu().numpy(), oci)


@pytest.mark.parametrize("prec", ["fp64", "bf16", "fp16"])
def test_p3_tets_parity(p3_case, prec):
    plan, ref, kap = p3_case
    kd = cuda(kap)
    els = {f: plan.empty_elements(prec) for f in ("stiffness", "mass")}
    vals = plan.assemble(kd, prec=prec, elements=els)
    plan.sync()
    ids = _sample(plan.n_cells, 600, 17)
    for form in ("stiffness", "mass"):
        A = ref.element_matrices_subset(kap, form, ids)
        got_all = to_np(els[form])
        got = got_all[ids]
        err = cell_errors(got, A)
        if prec == "fp64":
            assert err.max() <= FP64_TOL, err.max()
        else:
            bnd = cell_bounds(ref, kap, form, prec, A, cell_ids=ids)
            assert np.all(err <= bnd), (float(err.max()), float(bnd.min()))
        # the full CSR against the oracle's assembly of the GPU element matrices
        g = ref.assemble(got_all)
        gv = to_np(vals[form])
        rel = np.abs(gv - g).max() / np.abs(g).max()
        assert rel <= (1e-14 if prec == "fp64" else 24 * 2.0 ** -23), rel


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7, 8])
def test_degree_sweep_sampled_cells(p):
    v, c = inputs.cube_mesh(16, 0.15, 4)
    pts, w = api.quadrature_rule("tetrahedron", p + 1)
    precs = ("tf32x3", "tf32", "bf16", "fp16", "e4m3")
    plan = api.Plan("tetrahedron", v, c, p, pts, w, precisions=precs)
    kap = inputs.lognormal_kappa(plan.n_cells, plan.n_q, 5)
    ref = oracle.Problem(v, c, p, *oracle.collapsed_rule("tetrahedron", p + 1))
    ids = _sample(plan.n_cells, 48 if p <= 5 else 12, 40 + p)
    kd = cuda(kap)
    for form in ("stiffness", "mass"):
        A = ref.element_matrices_subset(kap, form, ids)
        for prec in ("fp64",) + precs:
            got = to_np(plan.element_matrices(kd, forms=(form,), prec=prec)[form])[ids]
            plan.sync()
            err = cell_errors(got, A)
            if prec == "fp64":
                assert err.max() <= FP64_TOL, (p, form, err.max())
            else:
                bnd = cell_bounds(ref, kap, form, prec, A, cell_ids=ids)
                assert np.all(err <= bnd), (p, form, prec, float(err.max()), float(bnd.min()))
