"""Shared helpers of the GPU parity tests (no method arithmetic: bounds come
from the oracle's kappa_q and error_bound)."""
import numpy as np
import torch

import oracle
from paper_2410_12614_gb300 import api, inputs

U_S = {"bf16": 2.0 ** -8, "fp16": 2.0 ** -11, "tf32": 2.0 ** -11, "tf32x3": 2.0 ** -21, "e4m3": 2.0 ** -4}
# operand roundings charged per cell: C and the tabulated product operand (2);
# e4m3 gets a doubled constant for the gradual-underflow range of its 3-bit mantissa.
ROUNDINGS = {"bf16": 2, "fp16": 2, "tf32": 2, "tf32x3": 2, "e4m3": 4}
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
    return oracle.error_bound(kq, U_S[prec], contraction_length(ref, form), storage_roundings=ROUNDINGS[prec])


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
