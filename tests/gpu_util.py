"""Shared helpers of the GPU parity tests (no method arithmetic: bounds come
from the oracle's kappa_q and error_bound)."""
import numpy as np
import torch

import oracle
from paper_2410_12614_gb300 import api, inputs

# Per-format constants of oracle.error_bound (see its docstring):
# U_S, ROUNDINGS -- each product of two stored operands carries (1 + u)^r - 1:
#   one rounding of C and one of the tabulated operand (r = 2, u = u_s); for
#   the split TF32x3 each operand is hi + lo with |x - hi - lo| <= 2^-22 |x| and
#   the dropped lo.lo product adds 2^-22 more: r = 3, u = 2^-22;
# U_PRE -- the relative error of C before its storage rounding: the FP32
#   coefficient window (kappa and the weight rounded to FP32, their product:
#   3 roundings), the FP32 product with the geometry factor (1), and the
#   geometry factor itself: FP32 G from FP64 cofactors with the cancellation
#   guard, (5 * 16 + 3) roundings for an off-diagonal entry, or FP64 G rounded
#   once (TF32x3: 1);
# FORMAT -- mantissa bits, smallest normal exponent and scale target binade of
#   the gradual-underflow term (oracle.subnormal_term).
U_S = {"bf16": 2.0 ** -8, "fp16": 2.0 ** -11, "tf32": 2.0 ** -11, "tf32x3": 2.0 ** -22, "e4m3": 2.0 ** -4}
ROUNDINGS = {"bf16": 2, "fp16": 2, "tf32": 2, "tf32x3": 3, "e4m3": 2}
U_PRE = {"bf16": 87 * 2.0 ** -24, "fp16": 87 * 2.0 ** -24, "tf32": 87 * 2.0 ** -24, "tf32x3": 5 * 2.0 ** -24,
         "e4m3": 87 * 2.0 ** -24}
FORMAT = {"bf16": (7, -126, 1), "fp16": (10, -14, 15), "tf32": (10, -126, 1), "tf32x3": (10, -126, 1),
          "e4m3": (3, -6, 8)}
FP64_TOL = 1e-12


def make_case(cell, n, p, alpha, seed_mesh, seed_kappa, precisions=("bf16",)):
    v, c = inputs.structured_mesh(cell, n, alpha, seed_mesh)
    pts, w = api.quadrature_rule(cell, p + 1)
    plan = api.Plan(cell, v, c, p, pts, w, precisions=precisions)
    kap = inputs.lognormal_kappa(plan.n_cells, plan.n_q, seed_kappa)
    ref = oracle.Problem(v, c, p, *oracle.rule_for_degree(cell, p))
    return plan, ref, kap


def contraction_length(ref, form):
    d = ref.d
    return ref.n_q * (d * (d + 1) // 2 if form == "stiffness" else 1)


def cell_errors(got, exact):
    """Per-cell max-norm relative error ||A^ - A||_max / ||A||_max (the paper's metric)."""
    num = np.abs(got - exact).reshape(len(exact), -1).max(axis=1)
    den = np.abs(exact).reshape(len(exact), -1).max(axis=1)
    return num / den


def cell_bounds(ref, kap, form, prec, exact, cell_ids=None):
    kq = ref.kappa_q(kap, form, exact, cell_ids=cell_ids)
    sub = oracle.subnormal_term(ref, kap, form, exact, *FORMAT[prec], cell_ids=cell_ids)
    return oracle.error_bound(kq, U_S[prec], contraction_length(ref, form), storage_roundings=ROUNDINGS[prec],
                              u_pre=U_PRE[prec], abs_rel=sub)


def csr_bound(ref, exact_elems, per_cell_err, m_K=None):
    """Entrywise bound of Corollary 4.11: L|D^-D|L^T + 2 m_K u_q L|D|L^T,
    with |D^-D| <= err_c ||A^c||_max on every entry of cell c."""
    nph = ref.n_phi
    amax = np.abs(exact_elems).reshape(len(exact_elems), -1).max(axis=1)
    E = np.broadcast_to((per_cell_err * amax)[:, None, None], exact_elems.shape).copy()
    bnd = ref.assemble(E, absval=True)
    if m_K is None:
        dofs, _ = ref.cell_dofs()
        m_K = int(np.bincount(dofs.reshape(-1)).max())
    bnd += 2 * m_K * 2.0 ** -24 * ref.assemble(exact_elems, absval=True)
    return bnd


def to_np(t):
    return t.double().cpu().numpy()


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()
