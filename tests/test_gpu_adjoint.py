"""GPU adjoint of L = v^T A_stiffness u against the FP64 oracle.

dL/dkappa at the quadrature points and dL/dvertices (kappa held fixed),
computed by fe_adjoint with the geometry recomputed from the vertices, are
compared with the oracle's closed-form gradient (itself pinned by central
differences and invariants in test_oracle_assembly_adjoint.py), with central
finite differences of the GPU's own L (FP64, step 1e-6), and through the
torch.autograd.Function.  Workload sizes: small meshes and P2 tetrahedra on
32^3 x 6 boxes (196,608 cells).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2410_12614_gb300 import api, inputs

from gpu_util import cuda

pytestmark = pytest.mark.gpu


def _case(cell, n, p, alpha, seeds):
    v, c = inputs.structured_mesh(cell, n, alpha, seeds[0])
    pts, w = api.quadrature_rule(cell, p + 1)
    plan = api.Plan(cell, v, c, p, pts, w, forms=("stiffness",), precisions=("bf16",))
    kap = inputs.lognormal_kappa(plan.n_cells, plan.n_q, seeds[1])
    u = inputs.gaussian_vector(plan.n_dofs, seeds[2])
    vv = inputs.gaussian_vector(plan.n_dofs, seeds[3])
    ref = oracle.Problem(v, c, p, *oracle.rule_for_degree(cell, p))
    return plan, ref, v, kap, u, vv


@pytest.mark.parametrize("cell,n,p", [("triangle", 3, 2), ("triangle", 2, 4), ("tetrahedron", 2, 1),
                                      ("tetrahedron", 2, 2), ("tetrahedron", 2, 3)])
def test_adjoint_small_vs_oracle_and_fd(cell, n, p):
    plan, ref, v, kap, u, vv = _case(cell, n, p, 0.15, (31, 32, 33, 34))
    L, gk, gx = plan.adjoint(cuda(kap), cuda(u), cuda(vv))
    plan.sync()
    Lo, gko, gxo = ref.adjoint_stiffness(kap, u.astype(np.float64), vv.astype(np.float64))
    assert abs(L.item() - Lo) <= 1e-12 * abs(Lo)
    np.testing.assert_allclose(gk.cpu().numpy(), gko, rtol=0, atol=1e-12 * np.abs(gko).max())
    np.testing.assert_allclose(gx.cpu().numpy(), gxo, rtol=0, atol=1e-12 * np.abs(gxo).max())
    # central differences of the GPU's own L in the vertex coordinates
    rng = np.random.default_rng(3)
    verts = torch.from_numpy(v).cuda()
    for _ in range(4):
        i, s = int(rng.integers(v.shape[0])), int(rng.integers(v.shape[1]))
        h = 1e-6
        vp, vm = verts.clone(), verts.clone()
        vp[i, s] += h
        vm[i, s] -= h
        Lp = plan.adjoint(cuda(kap), cuda(u), cuda(vv), vertices=vp, want_kappa=False, want_vertices=False)[0].item()
        Lm = plan.adjoint(cuda(kap), cuda(u), cuda(vv), vertices=vm, want_kappa=False, want_vertices=False)[0].item()
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - gx[i, s].item()) <= 1e-6 * gx.abs().max().item()


def test_adjoint_p2_tets_32_cubed():
    plan, ref, v, kap, u, vv = _case("tetrahedron", 32, 2, 0.15, (7, 8, 9, 10))
    assert plan.n_cells == 196608 and plan.n_dofs == 274625
    L, gk, gx = plan.adjoint(cuda(kap), cuda(u), cuda(vv))
    plan.sync()
    Lo, gko, gxo = ref.adjoint_stiffness(kap, u.astype(np.float64), vv.astype(np.float64))
    assert abs(L.item() - Lo) <= 1e-11 * abs(Lo)
    np.testing.assert_allclose(gk.cpu().numpy(), gko, rtol=0, atol=1e-12 * np.abs(gko).max())
    np.testing.assert_allclose(gx.cpu().numpy(), gxo, rtol=0, atol=1e-11 * np.abs(gxo).max())
    # kappa enters linearly: central differences of L in kappa are exact up to rounding
    rng = np.random.default_rng(4)
    kd = cuda(kap)
    for _ in range(3):
        c, q = int(rng.integers(plan.n_cells)), int(rng.integers(plan.n_q))
        h = 1e-3
        kp, km = kd.clone(), kd.clone()
        kp[c, q] += h
        km[c, q] -= h
        Lp = plan.adjoint(kp, cuda(u), cuda(vv), want_kappa=False, want_vertices=False)[0].item()
        Lm = plan.adjoint(km, cuda(u), cuda(vv), want_kappa=False, want_vertices=False)[0].item()
        assert abs((Lp - Lm) / (2 * h) - gk[c, q].item()) <= 1e-9 * gk.abs().max().item() + 1e-9 * abs(Lo)


def test_autograd_function_matches_adjoint():
    plan, ref, v, kap, u, vv = _case("tetrahedron", 3, 2, 0.15, (41, 42, 43, 44))
    kd = cuda(kap).requires_grad_(True)
    xd = torch.from_numpy(v).cuda().requires_grad_(True)
    L = api.QuadraticForm.apply(kd, xd, cuda(u), cuda(vv), plan)
    (2.5 * L).backward()
    _, gk, gx = plan.adjoint(cuda(kap), cuda(u), cuda(vv))
    torch.testing.assert_close(kd.grad, 2.5 * gk, rtol=0, atol=0)
    torch.testing.assert_close(xd.grad, 2.5 * gx, rtol=0, atol=0)
    # L agrees with v^T A u assembled by the library in FP64
    vals = plan.assemble(cuda(kap), forms=("stiffness",), prec="fp64")["stiffness"]
    rp, ci = plan.csr_pattern()
    rows = torch.repeat_interleave(torch.arange(plan.n_dofs, device="cuda"), rp[1:] - rp[:-1])
    quad = (cuda(vv).double()[rows] * vals * cuda(u).double()[ci.long()]).sum()
    assert abs(quad.item() - L.item()) <= 1e-12 * abs(L.item())


def test_adjoint_is_deterministic():
    plan, ref, v, kap, u, vv = _case("tetrahedron", 4, 3, 0.15, (51, 52, 53, 54))
    a = plan.adjoint(cuda(kap), cuda(u), cuda(vv))
    b = plan.adjoint(cuda(kap), cuda(u), cuda(vv))
    for x, y in zip(a, b):
        assert torch.equal(x, y)
