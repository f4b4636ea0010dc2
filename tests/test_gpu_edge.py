"""GPU edge cases of the assembly chunking and of the factor kernel's geometry.

* A fan of 200 P5 triangles around one vertex: that vertex's CSR row sums
  200 * 21 = 4200 element entries, above the 4096-entry assembly chunk, so it
  is summed on the per-row fallback path; its neighbours' rows exercise the
  256-incidence chunk limit.
* Tetrahedra so small (or so large) that det J leaves FP32's normal range:
  the factor kernel must fall back to forming G in FP64.
The oracle decides in every case (FP64 to 1e-12; reduced precision within the
per-cell bound of Corollary 4.10 and the CSR bound of Corollary 4.11).
"""
import numpy as np
import pytest

import oracle
from paper_2410_12614_gb300 import api, inputs

from gpu_util import FP64_TOL, cell_bounds, cell_errors, csr_bound, cuda, to_np

pytestmark = pytest.mark.gpu


def fan_mesh(n_tri, radius=1.0):
    ang = 2 * np.pi * np.arange(n_tri) / n_tri
    v = np.vstack([[0.0, 0.0], np.c_[radius * np.cos(ang), radius * np.sin(ang)]])
    c = np.array([[0, 1 + i, 1 + (i + 1) % n_tri] for i in range(n_tri)], dtype=np.int32)
    return v, c


def _plan_and_ref(cell, v, c, p, precisions):
    pts, w = api.quadrature_rule(cell, p + 1)
    plan = api.Plan(cell, v, c, p, pts, w, precisions=precisions)
    ref = oracle.Problem(v, c, p, *oracle.rule_for_degree(cell, p))
    return plan, ref


def test_fan_row_above_chunk_limit():
    v, c = fan_mesh(200)
    p = 5
    plan, ref = _plan_and_ref("triangle", v, c, p, ("bf16",))
    dofs, _ = ref.cell_dofs()
    # the centre vertex's row really is above the chunk limit
    assert 200 * ref.n_phi > 4096 and np.bincount(dofs.reshape(-1)).max() == 200
    kap = inputs.lognormal_kappa(plan.n_cells, plan.n_q, 5)
    kd = cuda(kap)
    rp, ci = plan.csr_pattern()
    orp, oci = ref.csr_pattern()
    assert np.array_equal(rp.cpu().numpy(), orp) and np.array_equal(ci.cpu().numpy(), oci)
    for form in ("stiffness", "mass"):
        A = ref.element_matrices(kap, form)
        g_exact = ref.assemble(A)
        for prec in ("fp64", "bf16"):
            els = plan.element_matrices(kd, forms=(form,), prec=prec)
            vals = plan.assemble(kd, forms=(form,), prec=prec)
            plan.sync()
            got, gv = to_np(els[form]), to_np(vals[form])
            if prec == "fp64":
                assert cell_errors(got, A).max() <= FP64_TOL
                assert np.abs(gv - g_exact).max() <= FP64_TOL * np.abs(g_exact).max()
            else:
                bnd = cell_bounds(ref, kap, form, prec, A)
                assert np.all(cell_errors(got, A) <= bnd)
                assert np.all(np.abs(gv - g_exact) <= csr_bound(ref, A, bnd))
            # the GPU's assembly of its own element matrices, entry by entry, in
            # particular on the long row
            own = ref.assemble(got)
            centre = slice(int(orp[0]), int(orp[1]))
            assert np.abs(gv - own).max() <= (1e-13 if prec == "fp64" else 1e-5) * np.abs(g_exact).max()
            assert np.abs(gv[centre] - own[centre]).max() <= (1e-13 if prec == "fp64" else 1e-5) * np.abs(own).max()


@pytest.mark.parametrize("scale", [1e-13, 1e13])
def test_geometry_outside_fp32_range(scale):
    # |det J| ~ (scale/2)^3: below FP32's smallest normal number (1e-13) or
    # above its largest (1e13); the stiffness matrices scale like h and stay
    # representable, the mass matrices (~h^3) do not and are not checked.
    v, c = inputs.structured_mesh("tetrahedron", 2, 0.15, 21)
    v = v * scale
    p = 2
    plan, ref = _plan_and_ref("tetrahedron", v, c, p, ("bf16", "fp16", "tf32x3"))
    kap = inputs.lognormal_kappa(plan.n_cells, plan.n_q, 22)
    kd = cuda(kap)
    A = ref.element_matrices(kap, "stiffness")
    for prec in ("bf16", "fp16", "tf32x3"):
        got = to_np(plan.element_matrices(kd, forms=("stiffness",), prec=prec)["stiffness"])
        plan.sync()
        bnd = cell_bounds(ref, kap, "stiffness", prec, A)
        err = cell_errors(got, A)
        assert np.all(err <= bnd), (prec, float(err.max()))


@pytest.mark.parametrize("shape", ["flat", "needle"])
def test_distorted_cells_all_formats(shape):
    """Tetrahedra of aspect ratio ~1e4 (a jittered cube mesh squashed along z,
    or stretched into needles along z): G spans eight orders of magnitude and
    its off-diagonal entries cancel, which the factor kernel detects and forms
    in FP64.  Every format must stay within the per-cell bound (the measured
    error and the bound are printed side by side) and match the
    emulated-precision operands of oracle/emulate.py to FP32 accumulation."""
    from oracle import emulate
    v, c = inputs.structured_mesh("tetrahedron", 3, 0.15, 31)
    v = v.copy()
    if shape == "flat":
        v[:, 2] *= 1e-4
    else:
        v[:, :2] *= 1e-4
    p = 3
    precs = ("bf16", "fp16", "tf32", "tf32x3", "e4m3")
    plan, ref = _plan_and_ref("tetrahedron", v, c, p, precs)
    kap = inputs.lognormal_kappa(plan.n_cells, plan.n_q, 32)
    kd = cuda(kap)
    for form in ("stiffness", "mass"):
        A = ref.element_matrices(kap, form)
        for prec in precs:
            got = to_np(plan.element_matrices(kd, forms=(form,), prec=prec)[form])
            plan.sync()
            bnd = cell_bounds(ref, kap, form, prec, A)
            err = cell_errors(got, A)
            print(shape, form, prec, "max err", float(err.max()), "bound at that cell", float(bnd[err.argmax()]),
                  "worst err/bound", float((err / bnd).max()))
            assert np.all(err <= bnd), (shape, form, prec, float((err / bnd).max()))
            E, M, K, slack = emulate.element_matrices(ref, kap, form, prec)
            x = K * 2 * 2.0 ** -23
            tol = x / (1 - x) * M + 2.0 ** -24 * np.abs(E) + slack
            assert np.all(np.abs(got - E) <= tol), (shape, form, prec, float((np.abs(got - E) / tol).max()))


@pytest.mark.parametrize("p", [3, 5])
def test_misaligned_buffers_same_bits(p):
    """Element matrices written into views that start 4 bytes past a 16-byte
    boundary, from a kappa view 8 bytes past one, are bitwise those of aligned
    buffers: the vector loads and stores are taken only on aligned addresses
    (P3: the staged pair layout; P5: full-row passes)."""
    import torch
    v, c = inputs.cube_mesh(4, 0.15, 3)
    pts, w = api.quadrature_rule("tetrahedron", p + 1)
    plan = api.Plan("tetrahedron", v, c, p, pts, w, precisions=("bf16",), elements_only=True)
    kap = inputs.lognormal_kappa(plan.n_cells, plan.n_q, 5)
    k_al = cuda(kap)
    k_buf = torch.empty(kap.size + 1, dtype=torch.float64, device="cuda")
    k_off = k_buf[1:].view(plan.n_cells, plan.n_q)
    k_off.copy_(k_al)
    assert k_off.data_ptr() % 16 == 8
    ref = plan.element_matrices(k_al, prec="bf16")
    n = plan.n_cells * plan.n_phi * plan.n_phi
    outs = {}
    for f in ("stiffness", "mass"):
        buf = torch.full((n + 1,), float("nan"), dtype=torch.float32, device="cuda")
        outs[f] = buf[1:].view(plan.n_cells, plan.n_phi, plan.n_phi)
        assert outs[f].data_ptr() % 16 == 4
    got = plan.element_matrices(k_off, prec="bf16", out=outs)
    plan.sync()
    for f in ("stiffness", "mass"):
        assert torch.equal(got[f], ref[f]), f
