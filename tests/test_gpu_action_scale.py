"""Linear forms (Algorithm 2) at the size of the P3 workload: 24^3 x 6 Kuhn
tetrahedra (82,944 cells, h = 1/24), every cell against the oracle.

On this mesh r_s = w_q kappa (G grad w)_s is about 1e-4 and the mass r about
2e-7: FP16's smallest normal number is 6.1e-5, so without scaling the mass r
would be rounded in FP16's subnormal range with errors near 10%.  The FP16
path rounds the cell's coefficients and r_s with per-cell powers of two
(exact), so each cell-vector entry must satisfy the componentwise bound

    |b^ - b| <= (4 u_s + gamma_K(2 u_32) + 8 2^-24) M_j + S_j,

M_j = sum_{s,q} |B_sjq| sum_t |w_q kappa G_st| sum_k |B_tkq| |w_k| (four storage
roundings reach b: w^c and B in grad w, r_s, B in b; the casting remark and the
theorem on r_s in Sec. 4.5), and S_j the absolute error of values that still
fall below FP16's normal range after scaling (half the subnormal spacing,
2^-25, in scaled units):

    S_j = 2^-32 max|w^c| M1_j + 2^-26 max|w^c| w_max beta gnorm_c sum_{s,q} |B_sjq|,

M1_j the magnitude with |w_k| = 1, beta = max_{s,q} sum_k |B_skq|, w_max the
largest weight, gnorm_c = max_s sum_t |G_st| (mass: |det J|): the first term
for coefficients below 2^-7 max|w^c| 2^-14 (scaled by 2^e_w with max|w^c| 2^e_w
>= 2^7), the second for r below the scaled bound's 2^-17 (2^e_r puts
max|w^c| 2^e_w w_max beta gnorm_c 2^e_r in [2^3, 2^4) up to a factor two).
BF16 and TF32 share FP32's range: S_j = 0 there.
"""
import numpy as np
import pytest

import oracle
from paper_2410_12614_gb300 import api, inputs

from gpu_util import cuda, to_np

pytestmark = pytest.mark.gpu

U_S = {"tf32": 2.0 ** -11, "bf16": 2.0 ** -8, "fp16": 2.0 ** -11}


def _bounds(ref, kap, w, form, prec):
    b_ex, M = ref.action(kap, w, form, with_magnitude=True)
    K = ref.n_q * (ref.d if form == "stiffness" else 1) + ref.n_phi
    x = K * 2 * 2.0 ** -23
    tol = (4 * U_S[prec] + x / (1 - x) + 8 * 2.0 ** -24) * M
    if prec == "fp16":
        dofs, _ = ref.cell_dofs()
        wmaxc = np.abs(w[dofs]).max(axis=1)                          # max |w^c|
        _, M1 = ref.action(kap, np.ones_like(w), form, with_magnitude=True)
        det, G = oracle.mesh_geometry(ref.vertices, ref.cells)
        B = ref.dphi if form == "stiffness" else ref.phi[None]
        beta = np.abs(B).sum(axis=1).max()                           # max_{s,q} sum_k |B_skq|
        gnorm = np.abs(G).sum(axis=2).max(axis=1) if form == "stiffness" else np.abs(det)
        sumB = np.abs(B).sum(axis=(0, 2))                            # sum_{s,q} |B_sjq|
        S = 2.0 ** -32 * wmaxc[:, None] * M1 + \
            2.0 ** -26 * (wmaxc * ref.weights.max() * beta * gnorm)[:, None] * sumB[None, :]
        tol = tol + S
    return b_ex, tol


@pytest.mark.parametrize("prec", ["fp16", "bf16", "tf32"])
def test_action_p3_tet24_every_cell(prec):
    v, c = inputs.cube_mesh(24, 0.15, 2)
    pts, wts = api.quadrature_rule("tetrahedron", 4)
    plan = api.Plan("tetrahedron", v, c, 3, pts, wts, precisions=("bf16",))
    kap = inputs.lognormal_kappa(plan.n_cells, plan.n_q, 3)
    w = inputs.gaussian_vector(plan.n_dofs, 4).astype(np.float64)
    ref = oracle.Problem(v, c, 3, *oracle.rule_for_degree("tetrahedron", 3))
    vg, bg = plan.action(cuda(kap), cuda(w), prec=prec, cell_vectors=True)
    plan.sync()
    for form in ("stiffness", "mass"):
        b_ex, tol = _bounds(ref, kap, w, form, prec)
        got = to_np(bg[form])
        ratio = np.abs(got - b_ex) / tol
        print(prec, form, "worst |err|/bound", float(ratio.max()),
              "worst rel err", float((np.abs(got - b_ex).max(axis=1) / np.abs(b_ex).max(axis=1)).max()))
        assert np.all(np.abs(got - b_ex) <= tol), (prec, form, float(ratio.max()))
        # the assembled vector: its cells' bounds plus its own FP32 summation
        vt = ref.assemble_vector(tol) + 32 * 2.0 ** -24 * ref.assemble_vector(np.abs(b_ex))
        assert np.all(np.abs(to_np(vg[form]) - ref.assemble_vector(b_ex)) <= vt), (prec, form)


def test_action_fp16_p6_warp_kernel_fine_mesh():
    # the warp-per-cell kernel (n_phi = 84) on h = 1/8 with FP16 scaling
    v, c = inputs.cube_mesh(8, 0.15, 12)
    pts, wts = api.quadrature_rule("tetrahedron", 7)
    plan = api.Plan("tetrahedron", v, c, 6, pts, wts, precisions=("bf16",))
    kap = inputs.lognormal_kappa(plan.n_cells, plan.n_q, 13)
    w = inputs.gaussian_vector(plan.n_dofs, 14).astype(np.float64)
    ref = oracle.Problem(v, c, 6, *oracle.rule_for_degree("tetrahedron", 6))
    _, bg = plan.action(cuda(kap), cuda(w), prec="fp16", cell_vectors=True)
    plan.sync()
    for form in ("stiffness", "mass"):
        b_ex, tol = _bounds(ref, kap, w, form, "fp16")
        got = to_np(bg[form])
        assert np.all(np.abs(got - b_ex) <= tol), (form, float((np.abs(got - b_ex) / tol).max()))
