"""Emulated-precision oracle for the reduced-precision contraction.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): it shares no code with
the CUDA library and never calls it.

The plain oracle evaluates the quadrature-exact element matrices in FP64; the
error bound of Theorem 4.8 / Corollary 4.10 then allows everything the
mixed strategy of Sec. 4.5 may do.  This module is the tighter pin: it rounds
the two contraction operands to the storage format exactly as the mixed
kernels are specified to, and accumulates their products in FP64, so that a
kernel's result may differ from it only by the FP32 accumulation (and the
FP32 store):

    |A_kernel - A_emulated| <= gamma_K(2 u_acc) * sum |C| |P| + u_out |A_emulated| + slack,

the slack covering the difference between two FP64 tabulations of the basis
(see element_matrices).

The operands (Sec. 3.1 with the pairs (s <= t) folded, mass: one pair):

    P_(st,q),(kl) = RN_s( 2^{e_P} (B_skq B_tlq + [s != t] B_tkq B_slq) )     (FP64, one rounding)
    C_(st,q)      = RN_s( fl32( fl32(kappa32_cq * w32_q) * fl32(G32_st * 2^{e_c}) ) )
    A^c_kl        = 2^{-e_c} 2^{-e_P} sum_{(st),q} C_(st,q) P_(st,q),(kl)      (k <= l, mirrored)

with kappa32 = RN_32(kappa), w32 = RN_32(w), the scale exponents e_P, e_c of
the narrow formats (FP16, e4m3: the largest |P| resp. max_q|kappa32 w32| *
max_st|G32| brought to the format's target binade; powers of two are exact),
and the geometry factor G32 formed from the FP64 cofactor matrix C of J
(J^{-1} = C^T / det J, Sec. 4.2):

    BF16, FP16, TF32, e4m3:  c32 = RN_32(C), a32 = RN_32(|det J|),
                             G32_st = fl32( fma32(c0s, c0t, fma32(c1s, c1t, fl32(c2s c2t))) * fl32(1 / a32) )
                             (a cell whose off-diagonal sums cancel by more than a
                             factor 16 takes the TF32x3 form; see geometry32)
    TF32x3:                  G32_st = RN_32( sum_i C_is C_it / |det J| )  (FP64 first)

(mass: G32 = a32).  TF32x3 splits both operands into TF32 hi and lo parts and
keeps hi.hi + hi.lo + lo.hi.  All roundings are round-to-nearest-even with
gradual underflow; e4m3 saturates at 448.
"""
from __future__ import annotations

import numpy as np

# (explicit mantissa bits, smallest normal exponent, largest finite value)
FORMATS = {
    "bf16": (7, -126, 3.3895313892515355e38),
    "fp16": (10, -14, 65504.0),
    "tf32": (10, -126, 3.4028234663852886e38),
    "tf32x3": (10, -126, 3.4028234663852886e38),
    "e4m3": (3, -6, 448.0),
}
# target binade of the per-cell / per-operand power-of-two scales (1: no scaling)
TARGET_EXP = {"bf16": 1, "fp16": 15, "tf32": 1, "tf32x3": 1, "e4m3": 8}


def round_format(x, mbits: int, emin: int, maxfinite: float):
    """Round to nearest even into a binary format with `mbits` explicit mantissa
    bits, smallest normal exponent `emin` (gradual underflow below it) and
    largest finite value `maxfinite` (saturating)."""
    x = np.asarray(x, dtype=np.float64)
    ax = np.abs(x)
    _, E = np.frexp(ax)                     # ax = m 2^E, m in [0.5, 1): leading bit 2^(E-1)
    q = np.maximum(E - 1, emin) - mbits     # the quantum is 2^q
    r = np.ldexp(np.rint(np.ldexp(ax, -q)), q)
    r = np.minimum(r, maxfinite)
    return np.where(ax == 0, 0.0, np.copysign(r, x))


def quantum(x, mbits: int, emin: int):
    """The spacing 2^q of the format's values around |x| (q as in round_format)."""
    _, E = np.frexp(np.abs(np.asarray(x, dtype=np.float64)))
    return np.ldexp(1.0, np.maximum(E - 1, emin) - mbits)


def near_midpoint(y, mbits: int, emin: int, rel: float = 2.0 ** -40):
    """Entries whose rounding could go either way under a relative perturbation `rel`."""
    y = np.asarray(y, dtype=np.float64)
    r = round_format(y, mbits, emin, np.inf)
    return np.abs(np.abs(y - r) - 0.5 * quantum(y, mbits, emin)) <= rel * np.abs(y)


def f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32)


def fma32(a, b, c):
    """fl32(a b + c) for FP32 inputs: the product is exact in FP64."""
    return f32(np.float64(1.0) * np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64))


def pairs(d: int):
    return [(s, t) for s in range(d) for t in range(s, d)]


def cofactors(vertices, cells):
    """FP64 J, cofactor matrix C (C[i, s] with J^{-1} = C^T / det J) and det J per cell."""
    x = np.asarray(vertices, np.float64)[np.asarray(cells)]      # [nc, d+1, d]
    d = x.shape[2]
    J = np.transpose(x[:, 1:, :] - x[:, :1, :], (0, 2, 1))      # J[i][j] = x^{j+1}_i - x^0_i
    if d == 3:
        C = np.empty_like(J)
        for i in range(3):
            for s in range(3):
                r = [a for a in range(3) if a != i]
                c = [b for b in range(3) if b != s]
                minor = J[:, r[0], c[0]] * J[:, r[1], c[1]] - J[:, r[0], c[1]] * J[:, r[1], c[0]]
                C[:, i, s] = minor if (i + s) % 2 == 0 else -minor
        det = J[:, 0, 0] * C[:, 0, 0] + J[:, 0, 1] * C[:, 0, 1] + J[:, 0, 2] * C[:, 0, 2]
    else:
        C = np.empty_like(J)
        C[:, 0, 0], C[:, 0, 1] = J[:, 1, 1], -J[:, 1, 0]
        C[:, 1, 0], C[:, 1, 1] = -J[:, 0, 1], J[:, 0, 0]
        det = J[:, 0, 0] * J[:, 1, 1] - J[:, 0, 1] * J[:, 1, 0]
    return J, C, det


def geometry32(vertices, cells, g64: bool, with_mask: bool = False):
    """G32 [nc, n_pairs] in the pair order (s <= t) and |det J| in FP32.

    FP32 cells: G32 from the rounded cofactors as in the module docstring,
    except that a cell where some off-diagonal pair cancels -- the FP32 sum
    m_st = fma32(|c0s|,|c0t|, fma32(|c1s|,|c1t|, |fl32(c2s c2t)|)) of the
    magnitudes exceeding 16 |acc_st| (an exact zero counts) -- takes the FP64
    G rounded once, as the TF32x3 cells do (the kernels' guard against
    sheared cells, whose FP32 off-diagonals would lose their relative
    accuracy)."""
    _, C, det = cofactors(vertices, cells)
    d = C.shape[1]
    adet = np.abs(det)
    G64 = np.stack([np.einsum("ci,ci->c", C[:, :, s], C[:, :, t]) / adet for s, t in pairs(d)], axis=1)
    if g64:
        return (f32(G64), f32(adet), np.ones(len(adet), bool)) if with_mask else (f32(G64), f32(adet))
    c32 = f32(C)
    a32 = f32(adet)
    inv = (np.float32(1.0) / a32).astype(np.float32)
    out = []
    cancel = np.zeros(C.shape[0], dtype=bool)
    for s, t in pairs(d):
        if d == 3:
            acc = fma32(c32[:, 1, s], c32[:, 1, t], (c32[:, 2, s] * c32[:, 2, t]).astype(np.float32))
            mag = fma32(np.abs(c32[:, 1, s]), np.abs(c32[:, 1, t]),
                        np.abs((c32[:, 2, s] * c32[:, 2, t]).astype(np.float32)))
        else:
            acc = (c32[:, 1, s] * c32[:, 1, t]).astype(np.float32)
            mag = np.abs(acc)
        acc = fma32(c32[:, 0, s], c32[:, 0, t], acc)
        mag = fma32(np.abs(c32[:, 0, s]), np.abs(c32[:, 0, t]), mag)
        if s != t:
            cancel |= ~(mag <= np.float32(16.0) * np.abs(acc))
        out.append((acc * inv).astype(np.float32))
    G = np.stack(out, axis=1)
    G[cancel] = f32(G64[cancel])
    return (G, a32, cancel) if with_mask else (G, a32)


def operand_P(problem, form: str):
    """P [n_q, n_pairs, n_sym] in FP64 and the sym index list (k, l), k <= l."""
    d, nph, nq = problem.d, problem.n_phi, problem.n_q
    sym = [(k, l) for k in range(nph) for l in range(k, nph)]
    ks = np.array([k for k, _ in sym])
    ls = np.array([l for _, l in sym])
    if form == "mass":
        P = (problem.phi[ks, :] * problem.phi[ls, :]).T[:, None, :]
    else:
        B = problem.dphi
        cols = []
        for s, t in pairs(d):
            v = B[s][ks, :] * B[t][ls, :]
            if s != t:
                v = v + B[t][ks, :] * B[s][ls, :]
            cols.append(v.T)
        P = np.stack(cols, axis=1)
    return P, ks, ls


def _scale_exp(maxabs, target):
    """e such that maxabs 2^e lies in [2^(target-1), 2^target) (0 where maxabs is 0 or not finite)."""
    maxabs = np.asarray(maxabs)
    _, E = np.frexp(maxabs)
    ok = (maxabs > 0) & np.isfinite(maxabs)
    return np.where(ok, target - E, 0).astype(np.int64)


def element_matrices(problem, kappa, form: str, prec: str, exact: bool = False):
    """Emulated element matrices [nc, n_phi, n_phi], the magnitude sum |C||P|
    (unscaled, same shape), the number of accumulated products per entry, and
    the slack that the FP64 tabulation leaves (same shape): another FP64
    tabulation of the same basis differs by a few units of 2^-53, which moves
    P entries near zero by ~2^-46 max|P| and may flip the storage rounding of
    entries lying within 2^-40 of a rounding midpoint (one storage unit).

    exact=True skips every rounding (FP64 throughout): the result is then the
    quadrature-exact element matrix, computed through the folded P-form.
    """
    mbits, emin, maxf = FORMATS[prec]
    target = TARGET_EXP[prec]
    nc, nq, nph = problem.n_cells, problem.n_q, problem.n_phi
    kap = np.asarray(kappa, np.float64).reshape(nc, nq)
    rnd = (lambda v: v) if exact else (lambda v: round_format(v, mbits, emin, maxf))
    # the tabulated operand
    P, ks, ls = operand_P(problem, form)
    eP = 0 if exact else int(_scale_exp(np.abs(P).max(), target)) if target > 1 else 0
    Ps = np.ldexp(P, eP)
    P_hi = rnd(Ps)
    P_lo = rnd(Ps - P_hi) if prec == "tf32x3" and not exact else None
    # the per-cell factor
    if exact:
        _, C, det = cofactors(problem.vertices, problem.cells)
        adet = np.abs(det)
        if form == "mass":
            g = adet[:, None]
        else:
            g = np.stack([np.einsum("ci,ci->c", C[:, :, s], C[:, :, t]) / adet for s, t in pairs(problem.d)], axis=1)
        win = kap * problem.weights[None, :]
        Cv = win[:, :, None] * g[:, None, :]
        ec = np.zeros(nc, dtype=np.int64)
    else:
        G32, a32 = geometry32(problem.vertices, problem.cells, g64=(prec == "tf32x3"))
        g = a32[:, None] if form == "mass" else G32
        win = (f32(kap) * f32(problem.weights)[None, :]).astype(np.float32)
        if target > 1:
            wmax = np.abs(win).max(axis=1)
            gmax = np.abs(g).max(axis=1)
            ec = _scale_exp((wmax * gmax).astype(np.float32), target)
        else:
            ec = np.zeros(nc, dtype=np.int64)
        gj = np.ldexp(g.astype(np.float64), ec[:, None]).astype(np.float32)
        Cv = (win[:, :, None] * gj[:, None, :]).astype(np.float32).astype(np.float64)
    C_hi = rnd(Cv)
    if prec == "tf32x3" and not exact:
        C_lo = rnd((Cv.astype(np.float32) - C_hi.astype(np.float32)).astype(np.float64))
        terms = [(C_hi, P_hi), (C_hi, P_lo), (C_lo, P_hi)]
    else:
        terms = [(C_hi, P_hi)]
    Asym = sum(np.einsum("cqj,qjk->ck", a, b) for a, b in terms)
    mag = sum(np.einsum("cqj,qjk->ck", np.abs(a), np.abs(b)) for a, b in terms)
    if exact:
        slack = np.zeros_like(mag)
    else:
        amb = near_midpoint(Ps, mbits, emin) * quantum(Ps, mbits, emin)
        sumC = sum(np.abs(a) for a, _ in terms)
        slack = np.einsum("cqj,qjk->ck", sumC, amb) + 2.0 ** -46 * np.abs(Ps).max() * sumC.sum(axis=(1, 2))[:, None]
    unscale = np.ldexp(1.0, -(ec + eP))[:, None]
    Asym *= unscale
    mag *= unscale
    slack = slack * unscale
    A = np.zeros((nc, nph, nph))
    M = np.zeros((nc, nph, nph))
    Sl = np.zeros((nc, nph, nph))
    for dst, src in ((A, Asym), (M, mag), (Sl, slack)):
        dst[:, ks, ls] = src
        dst[:, ls, ks] = src
    K = nq * P.shape[1] * len(terms)
    return A, M, K, Sl
