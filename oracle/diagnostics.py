"""Emulated arithmetic of the paper's error studies (Sec. 5.2, 5.3).

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): it shares no code with
the CUDA library and never calls it.

* ``geometry_fp32`` -- the Poisson geometry tensor G = |det J| J^-1 J^-T
  evaluated exclusively in FP32 (Sec. 5.2, geometry errors), every operation
  a correctly rounded IEEE FP32 operation in the order the library documents
  for its FP32 diagnostic: vertex coordinates rounded to FP32,
  J_ij = x_{j+1,i} - x_{0,i}, cofactors as 2x2 minors fl(fl(a b) - fl(c e)),
  det J = fl(fl(J00 C0 + J01 C1) + J02 C2) (the first cofactor row),
  G_st = fl(fl(sum_r C_rs C_rt) * fl(1/|det J|)) with r increasing.  The
  exact G comes from the LU oracle (``oracle.mesh_geometry``).
* ``mass_fp16_products`` -- the mass bilinear form (Algorithm 1) and the mass
  action (Algorithm 2) with the matrix-matrix / matrix-vector products in
  FP16 and everything else in FP32 (Sec. 5.3: u_s = u_g = u_p = 2^-24,
  u_q = 2^-11): each product of two FP32 values rounded once to FP16, the
  products summed over the quadrature points in increasing order in FP16
  (one rounding per addition), with the per-cell powers of two the library
  documents for the range (exact).
"""
from __future__ import annotations

import numpy as np

from . import emulate


def _f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32)


def _rn16(x):
    """Round FP64 values to FP16 (round to nearest even, gradual underflow)."""
    return emulate.round_format(x, 10, -14, 65504.0)


def _jacobian32(vertices, cells):
    x = _f32(np.asarray(vertices)[np.asarray(cells)])          # [nc, d+1, d]
    d = x.shape[2]
    J = np.empty((x.shape[0], d, d), dtype=np.float32)
    for i in range(d):
        for j in range(d):
            J[:, i, j] = x[:, j + 1, i] - x[:, 0, i]
    return J


def _cofactors32(J):
    d = J.shape[1]
    if d == 2:
        C = np.empty_like(J)
        C[:, 0, 0], C[:, 0, 1] = J[:, 1, 1], -J[:, 1, 0]
        C[:, 1, 0], C[:, 1, 1] = -J[:, 0, 1], J[:, 0, 0]
        det = J[:, 0, 0] * J[:, 1, 1] - J[:, 0, 1] * J[:, 1, 0]
        return C, det
    C = np.empty_like(J)

    def m2(a, b, c, e):
        return (a * b) - (c * e)

    C[:, 0, 0] = m2(J[:, 1, 1], J[:, 2, 2], J[:, 1, 2], J[:, 2, 1])
    C[:, 0, 1] = m2(J[:, 1, 2], J[:, 2, 0], J[:, 1, 0], J[:, 2, 2])
    C[:, 0, 2] = m2(J[:, 1, 0], J[:, 2, 1], J[:, 1, 1], J[:, 2, 0])
    C[:, 1, 0] = m2(J[:, 0, 2], J[:, 2, 1], J[:, 0, 1], J[:, 2, 2])
    C[:, 1, 1] = m2(J[:, 0, 0], J[:, 2, 2], J[:, 0, 2], J[:, 2, 0])
    C[:, 1, 2] = m2(J[:, 0, 1], J[:, 2, 0], J[:, 0, 0], J[:, 2, 1])
    C[:, 2, 0] = m2(J[:, 0, 1], J[:, 1, 2], J[:, 0, 2], J[:, 1, 1])
    C[:, 2, 1] = m2(J[:, 0, 2], J[:, 1, 0], J[:, 0, 0], J[:, 1, 2])
    C[:, 2, 2] = m2(J[:, 0, 0], J[:, 1, 1], J[:, 0, 1], J[:, 1, 0])
    det = (J[:, 0, 0] * C[:, 0, 0] + J[:, 0, 1] * C[:, 0, 1]) + J[:, 0, 2] * C[:, 0, 2]
    return C, det


def geometry_fp32(vertices, cells):
    """(G [nc, d(d+1)/2] in the pair order (s <= t), |det J| [nc]) in FP32."""
    J = _jacobian32(vertices, cells)
    C, det = _cofactors32(J)
    d = J.shape[1]
    ad = np.abs(det)
    inv = np.float32(1.0) / ad
    out = []
    for s in range(d):
        for t in range(s, d):
            acc = C[:, 0, s] * C[:, 0, t]
            for r in range(1, d):
                acc = acc + C[:, r, s] * C[:, r, t]
            out.append(acc * inv)
    return np.stack(out, axis=1), ad


def _scale_exp(x, t):
    x = np.asarray(x, dtype=np.float64)
    _, E = np.frexp(x)
    ok = (x > 0) & np.isfinite(x)
    return np.where(ok, t - E, 0).astype(np.int64)


def mass_fp16_products(problem, kappa, w=None):
    """(A [nc, n_phi, n_phi], b [nc, n_phi] or None) as float64 arrays holding
    the FP32 results of the FP16-product mass form and action."""
    nc, nq, nph = problem.n_cells, problem.n_q, problem.n_phi
    kap = _f32(np.asarray(kappa).reshape(nc, nq))
    wts = _f32(problem.weights)
    phi = _f32(problem.phi)                                       # [nph, nq]
    _, det = _cofactors32(_jacobian32(problem.vertices, problem.cells))
    adet = np.abs(det)
    wk = wts[None, :] * kap                                       # fl32(w_q kappa_cq)
    cq = wk * adet[:, None]                                       # fl32(.. |det J|)
    csum = np.zeros(nc, dtype=np.float32)
    for q in range(nq):
        csum = csum + np.abs(cq[:, q])
    e = _scale_exp(csum, 10)
    sc = np.ldexp(np.float32(1.0), e).astype(np.float32)
    us = np.ldexp(np.float32(1.0), -e).astype(np.float32)
    C = (cq * sc[:, None]).astype(np.float32)                     # exact power of two
    H = (C[:, None, :] * phi[None, :, :]).astype(np.float32)      # [nc, k, q]
    acc = np.zeros((nc, nph, nph))
    for q in range(nq):
        prod = _rn16(H[:, :, q].astype(np.float64)[:, :, None] * phi[:, q].astype(np.float64)[None, None, :])
        acc = _rn16(acc + prod)
    A = (acc.astype(np.float32) * us[:, None, None]).astype(np.float64)
    b = None
    if w is not None:
        dofs, _ = problem.cell_dofs()
        wc = _f32(np.asarray(w)[dofs])                           # [nc, nph]
        ew = _scale_exp(np.abs(wc).max(axis=1), 1)
        sw = np.ldexp(np.float32(1.0), ew).astype(np.float32)
        wcs = (wc * sw[:, None]).astype(np.float32)
        accb = np.zeros((nc, nph))
        for q in range(nq):
            wq = np.zeros(nc, dtype=np.float32)
            for l in range(nph):
                wq = wq + phi[l, q] * wcs[:, l]
            r = C[:, q] * wq
            prod = _rn16(phi[:, q].astype(np.float64)[None, :] * r.astype(np.float64)[:, None])
            accb = _rn16(accb + prod)
        uw = np.ldexp(np.float32(1.0), -ew).astype(np.float32)
        b = ((accb.astype(np.float32) * us[:, None]).astype(np.float32) * uw[:, None]).astype(np.float64)
    return A, b
