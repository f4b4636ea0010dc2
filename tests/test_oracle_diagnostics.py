"""Pins of the emulated arithmetic of the paper's error studies
(oracle/diagnostics.py; Sec. 5.2 geometry errors, Sec. 5.3 FP16 products).

* FP32 geometry: on cells whose coordinates and geometry are exactly
  representable (small integers, the unscaled knife tetrahedron with eps a
  power of two) every FP32 operation is exact, so the result equals the
  closed form; on the scaled and translated knife tetrahedron the error grows
  with kappa_2(J) (Theorem on the Poisson geometry, Sec. 4.2) and stays far
  below 1 for kappa_2(J) << 2^24.
* FP16 products: a scalar re-implementation with Python's own round-half-even
  equals the vectorised emulation bit for bit on a tiny mesh, and the result
  is within the accumulation bound of Theorem 4.8 for u_q = 2^-11:
  |A16 - A| <= (gamma_{n_q}(u_q) + u_q + 6 2^-24) sum_q |C_q phi_kq phi_lq|.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import diagnostics as dg
from paper_2410_12614_gb300 import inputs


def test_fp32_geometry_exact_on_representable_cells():
    kuhn = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [1, 1, 1]], dtype=np.float64)
    G, ad = dg.geometry_fp32(kuhn, np.array([[0, 1, 2, 3]]))
    assert np.array_equal(G[0], [2, -1, 0, 2, -1, 1]) and ad[0] == 1
    eps = 2.0 ** -10
    knife = np.array([[0, 0, 0], [1, 1, 0], [1, 0, 1], [eps, 1, -1]], dtype=np.float64)
    G, ad = dg.geometry_fp32(knife, np.array([[0, 1, 2, 3]]))
    det, G64 = oracle.mesh_geometry(knife, np.array([[0, 1, 2, 3]], dtype=np.int32))
    iu = [(s, t) for s in range(3) for t in range(s, 3)]
    assert ad[0] == abs(det[0]) == eps
    assert np.array_equal(G[0].astype(np.float64), np.array([G64[0, s, t] for s, t in iu]))


def test_fp32_geometry_error_grows_with_condition_number():
    errs, kappas = [], []
    for k in range(2, 12):
        eps = 10.0 ** (-k / 2)
        x = np.array([[0, 0, 0], [1, 1, 0], [1, 0, 1], [eps, 1, -1]], dtype=np.float64)
        x = x / math.sqrt(3.0) + np.array([1 / 3, 2 / 3, 4 / 3])
        cells = np.array([[0, 1, 2, 3]], dtype=np.int32)
        G, _ = dg.geometry_fp32(x, cells)
        _, G64 = oracle.mesh_geometry(x, cells)
        iu = [(s, t) for s in range(3) for t in range(s, 3)]
        g = np.array([G64[0, s, t] for s, t in iu])
        errs.append(np.abs(G[0] - g).max() / (2.0 ** -24 * np.abs(g).max()))
        J, _, _ = oracle.geometry(x)
        kappas.append(np.linalg.cond(J, 2))
    slope = np.polyfit(np.log10(kappas[3:]), np.log10(np.maximum(errs[3:], 1e-3)), 1)[0]
    assert 0.5 < slope < 1.5, (slope, errs)
    assert errs[-1] > 100 * errs[0]


def _rn16_scalar(x):
    if x == 0.0:
        return 0.0
    m, e = math.frexp(abs(x))
    q = max(e - 1, -14) - 10
    return math.copysign(round(abs(x) / 2.0 ** q) * 2.0 ** q, x)


def test_fp16_products_scalar_reimplementation():
    v, c = inputs.cube_mesh(1, 0.0, 0)
    pr = oracle.Problem(v, c[:2], 2, *oracle.rule_for_degree("tetrahedron", 2))
    kap = inputs.lognormal_kappa(pr.n_cells, pr.n_q, 5)
    A, _ = dg.mass_fp16_products(pr, kap)
    f32 = np.float32
    for cc in range(pr.n_cells):
        xv = v[c[cc]].astype(np.float32)
        J = np.array([[xv[j + 1][i] - xv[0][i] for j in range(3)] for i in range(3)], dtype=np.float32)
        c0 = f32(J[1, 1] * J[2, 2]) - f32(J[1, 2] * J[2, 1])
        c1 = f32(J[1, 2] * J[2, 0]) - f32(J[1, 0] * J[2, 2])
        c2 = f32(J[1, 0] * J[2, 1]) - f32(J[1, 1] * J[2, 0])
        ad = abs(f32(f32(J[0, 0] * c0) + f32(J[0, 1] * c1)) + f32(J[0, 2] * c2))
        Cq = [f32(f32(f32(pr.weights[q]) * f32(kap[cc, q])) * ad) for q in range(pr.n_q)]
        s = f32(0)
        for x in Cq:
            s = f32(s + abs(x))
        e = 10 - math.frexp(float(s))[1]
        for k in range(pr.n_phi):
            for l in range(pr.n_phi):
                acc = 0.0
                for q in range(pr.n_q):
                    H = f32(f32(Cq[q] * f32(2.0 ** e)) * f32(pr.phi[k, q]))
                    acc = _rn16_scalar(acc + _rn16_scalar(float(f32(pr.phi[l, q])) * float(H)))
                assert A[cc, k, l] == float(f32(f32(acc) * f32(2.0 ** -e))), (cc, k, l)


@pytest.mark.parametrize("p", [1, 2, 4])
def test_fp16_products_within_accumulation_bound(p):
    v, c = inputs.cube_mesh(2, 0.15, 3)
    pr = oracle.Problem(v, c, p, *oracle.rule_for_degree("tetrahedron", p))
    kap = inputs.lognormal_kappa(pr.n_cells, pr.n_q, 4)
    A16, _ = dg.mass_fp16_products(pr, kap)
    A = pr.element_matrices(kap, "mass")
    uq = 2.0 ** -11
    g = pr.n_q * uq / (1 - pr.n_q * uq)
    det, _ = oracle.mesh_geometry(v, c)
    mag = np.einsum("cq,kq,lq->ckl", np.abs(pr.weights[None, :] * kap * det[:, None]), np.abs(pr.phi), np.abs(pr.phi))
    assert np.all(np.abs(A16 - A) <= (g + uq + 6 * 2.0 ** -24) * mag)
