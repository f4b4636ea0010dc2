"""The paper's error studies on the GPU (fe_geometry, fe_mass_fp16_products).

Sec. 5.2 (geometry errors): the knife tetrahedron with det J = eps, scaled by
3^-1/2 and translated, for eps = 10^-1 ... 10^-6.  The exclusively-FP32
geometry must equal the emulated FP32 arithmetic of oracle/diagnostics.py
bit for bit, and its error must grow linearly with kappa_2(J) (the theorem on
the Poisson geometry, Sec. 4.2); the library's production (mixed) geometry
must equal oracle/emulate.py's specification bit for bit, take FP64 on the
same cells, and stay within 87 units of 2^-24 of the exact G at every
condition number (the per-cell geometry precision of the remark in Sec. 5.2).

Sec. 5.3 (accumulation errors): the FP16-product mass form and action equal
their emulation bit for bit for P1-P4 tetrahedra, and their errors against
the FP64 oracle stay within the accumulation bound for u_q = 2^-11.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import diagnostics as dg
from oracle import emulate
from paper_2410_12614_gb300 import api, inputs

from gpu_util import cuda, to_np

pytestmark = pytest.mark.gpu

IU3 = [(s, t) for s in range(3) for t in range(s, 3)]


def _knife_mesh(eps_list):
    xs, cs = [], []
    for i, eps in enumerate(eps_list):
        x = np.array([[0, 0, 0], [1, 1, 0], [1, 0, 1], [eps, 1, -1]], dtype=np.float64)
        xs.append(x / math.sqrt(3.0) + np.array([1 / 3, 2 / 3, 4 / 3]))
        cs.append(np.arange(4 * i, 4 * i + 4))
    return np.vstack(xs), np.array(cs, dtype=np.int32)


def test_geometry_modes_on_knife_cells_and_a_mesh():
    eps = [10.0 ** (-k / 2) for k in range(2, 13)]
    v, c = _knife_mesh(eps)
    plan = api.Plan("tetrahedron", v, c, 1, precisions=("bf16",))
    det, G64 = oracle.mesh_geometry(v, c)
    g_exact = np.stack([G64[:, s, t] for s, t in IU3], axis=1)
    Gd, ad, _ = plan.geometry("fp64")
    Gf, adf, _ = plan.geometry("fp32")
    Gm, adm, used = plan.geometry("mixed")
    plan.sync()
    Gd, Gf, Gm = to_np(Gd), to_np(Gf), to_np(Gm)
    e32, a32 = dg.geometry_fp32(v, c)
    assert np.array_equal(Gf, e32.astype(np.float64)) and np.array_equal(to_np(adf), a32.astype(np.float64))
    em, am, mask = emulate.geometry32(v, c, g64=False, with_mask=True)
    assert np.array_equal(Gm, em.astype(np.float64)) and np.array_equal(used.cpu().numpy().astype(bool), mask)
    kappa2 = np.array([np.linalg.cond(oracle.geometry(v[4 * i:4 * i + 4])[0], 2) for i in range(len(eps))])
    scale = np.abs(g_exact).max(axis=1)
    err64 = np.abs(Gd - g_exact).max(axis=1) / scale
    err32 = np.abs(Gf - g_exact).max(axis=1) / scale
    errm = np.abs(Gm - g_exact).max(axis=1) / scale
    print("kappa2", kappa2.tolist())
    print("fp32 err / u32", (err32 / 2.0 ** -24).tolist())
    print("mixed err / u32", (errm / 2.0 ** -24).tolist())
    assert np.all(err64 <= 1e-16 * kappa2 * 64)
    slope = np.polyfit(np.log10(kappa2[3:]), np.log10(np.maximum(err32[3:], 1e-12)), 1)[0]
    assert 0.5 < slope < 1.5, slope
    assert np.all(errm <= 87 * 2.0 ** -24)
    # a jittered mesh: the modes agree with their specifications there too
    v2, c2 = inputs.cube_mesh(4, 0.15, 41)
    p2 = api.Plan("tetrahedron", v2, c2, 1, precisions=("bf16",))
    Gf2, _, _ = p2.geometry("fp32")
    Gm2, _, u2 = p2.geometry("mixed")
    p2.sync()
    assert np.array_equal(to_np(Gf2), dg.geometry_fp32(v2, c2)[0].astype(np.float64))
    em2, _, m2 = emulate.geometry32(v2, c2, g64=False, with_mask=True)
    assert np.array_equal(to_np(Gm2), em2.astype(np.float64)) and np.array_equal(u2.cpu().numpy().astype(bool), m2)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_fp16_products_match_emulation_and_bound(p):
    v, c = inputs.cube_mesh(2, 0.15, 50 + p)
    pts, w = api.quadrature_rule("tetrahedron", p + 1)
    plan = api.Plan("tetrahedron", v, c, p, pts, w, precisions=("bf16",))
    ref = oracle.Problem(v, c, p, *oracle.rule_for_degree("tetrahedron", p))
    kap = inputs.lognormal_kappa(plan.n_cells, plan.n_q, 60 + p)
    wv = inputs.gaussian_vector(plan.n_dofs, 70 + p).astype(np.float64)
    A, b = plan.mass_fp16_products(cuda(kap), cuda(wv))
    plan.sync()
    Ae, be = dg.mass_fp16_products(ref, kap, wv)
    assert np.array_equal(to_np(A), Ae)
    assert np.array_equal(to_np(b), be)
    Aex = ref.element_matrices(kap, "mass")
    uq = 2.0 ** -11
    g = ref.n_q * uq / (1 - ref.n_q * uq)
    det, _ = oracle.mesh_geometry(v, c)
    mag = np.einsum("cq,kq,lq->ckl", np.abs(ref.weights[None, :] * kap * det[:, None]), np.abs(ref.phi),
                    np.abs(ref.phi))
    assert np.all(np.abs(to_np(A) - Aex) <= (g + uq + 6 * 2.0 ** -24) * mag)


def test_fp16_products_error_growth_with_n_q():
    """Sec. 5.3: max over cells of ||A - A^||_max / (u_q ||A||_max) (and the
    action's ||b - b^||_inf / (u_q ||b||_inf)) for P1-P8 tetrahedra, n_q =
    (p+1)^3, with the rate of growth in n_q fitted in log-log (the paper finds
    about 0.7 for the bilinear form and about 1 for the action).  Each cell's
    error must stay within the accumulation bound (gamma_{n_q}(u_q) + u_q +
    6 2^-24) sum_q |C_q| |phi_k| |phi_l| relative to ||A||_max."""
    uq = 2.0 ** -11
    rows = []
    for p in range(1, 9):
        v, c = inputs.cube_mesh(2 if p <= 5 else 1, 0.15, 80 + p)
        pts, w = api.quadrature_rule("tetrahedron", p + 1)
        plan = api.Plan("tetrahedron", v, c, p, pts, w, precisions=("bf16",))
        ref = oracle.Problem(v, c, p, *oracle.rule_for_degree("tetrahedron", p))
        kap = inputs.lognormal_kappa(plan.n_cells, plan.n_q, 90 + p)
        wv = inputs.gaussian_vector(plan.n_dofs, 100 + p).astype(np.float64)
        A, b = plan.mass_fp16_products(cuda(kap), cuda(wv))
        plan.sync()
        A, b = to_np(A), to_np(b)
        Aex = ref.element_matrices(kap, "mass")
        bex = ref.action(kap, wv, "mass")
        ea = (np.abs(A - Aex).reshape(len(A), -1).max(1) / np.abs(Aex).reshape(len(A), -1).max(1)).max() / uq
        eb = (np.abs(b - bex).max(1) / np.abs(bex).max(1)).max() / uq
        g = ref.n_q * uq / (1 - ref.n_q * uq)
        det, _ = oracle.mesh_geometry(v, c)
        mag = np.einsum("cq,kq,lq->ckl", np.abs(ref.weights[None, :] * kap * det[:, None]), np.abs(ref.phi),
                        np.abs(ref.phi))
        assert np.all(np.abs(A - Aex) <= (g + uq + 6 * 2.0 ** -24) * mag), p
        rows.append((p, ref.n_q, float(ea), float(eb)))
    nq = np.array([r[1] for r in rows], float)
    rate_a = np.polyfit(np.log10(nq), np.log10([r[2] for r in rows]), 1)[0]
    rate_b = np.polyfit(np.log10(nq), np.log10([r[3] for r in rows]), 1)[0]
    for r in rows:
        print("p=%d n_q=%d bilinear err/u_q=%.3f action err/u_q=%.3f" % r)
    print("fitted rate in n_q: bilinear %.2f, action %.2f" % (rate_a, rate_b))
    assert 0.2 < rate_a < 1.3 and 0.2 < rate_b < 1.3
