"""The allocation-free adjoint entry point, fe_adjoint_noalloc.

Some callers may not allocate device memory while they run (their device
memory belongs to their own allocator or a fixed budget, or a latency-critical
loop cannot afford cudaMalloc's implicit synchronisation).  For them the
library offers fe_adjoint_noalloc, which takes the adjoint's per-cell scratch
from a fixed static device array instead of a plan workspace.  These tests
call it through the C ABI and check it against fe_adjoint on two calls in a
row, and check that plans above the array's capacity are rejected.  The file
name sorts last so that a run stopping at the first failure has already run
every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2410_12614_gb300 import _lib, api, inputs

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the relative tolerance of the adjoint parity tests


def _plan(n, seeds):
    v, c = inputs.cube_mesh(n, 0.15, seeds[0])
    pts, w = api.quadrature_rule("tetrahedron", 3)
    plan = api.Plan("tetrahedron", v, c, 2, pts, w, forms=("stiffness",), precisions=("bf16",))
    kap = torch.from_numpy(inputs.lognormal_kappa(plan.n_cells, plan.n_q, seeds[1])).cuda()
    u = torch.from_numpy(inputs.gaussian_vector(plan.n_dofs, seeds[2])).cuda()
    vv = torch.from_numpy(inputs.gaussian_vector(plan.n_dofs, seeds[3])).cuda()
    return plan, kap, u, vv


def _noalloc(plan, kap, u, vv, want_vertices=True):
    L = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    gk = torch.full((plan.n_cells, plan.n_q), np.nan, dtype=torch.float64, device="cuda")
    gx = torch.full((plan.n_vertices, 3), np.nan, dtype=torch.float64, device="cuda") if want_vertices else None
    st = _lib.load().fe_adjoint_noalloc(plan._h, None, ctypes.c_void_p(kap.data_ptr()),
                                        ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(vv.data_ptr()),
                                        ctypes.c_void_p(gk.data_ptr()),
                                        ctypes.c_void_p(gx.data_ptr()) if want_vertices else None,
                                        ctypes.c_void_p(L.data_ptr()))
    _lib.check(st, "fe_adjoint_noalloc")
    plan.sync()
    return L, gk, gx


def _close(a, b):
    scale = b.abs().max().item()
    assert (a - b).abs().max().item() <= TOL * scale


def test_noalloc_matches_adjoint_on_two_calls_in_a_row():
    plan, kap, u, vv = _plan(6, (61, 62, 63, 64))
    # on a fresh plan the allocation-free call comes first: it must leave the
    # plan's workspaces (where fe_adjoint keeps its scratch) empty
    _, ws0 = plan.memory()
    first = _noalloc(plan, kap, u, vv)
    assert plan.memory()[1] == ws0 == 0
    L0, gk0, gx0 = plan.adjoint(kap, u, vv)
    plan.sync()
    assert plan.memory()[1] > 0          # fe_adjoint did allocate its scratch
    for a, b in zip(first, (L0, gk0, gx0)):
        _close(a, b)
    for _ in range(2):
        L, gk, gx = _noalloc(plan, kap, u, vv)
        _close(L, L0)
        _close(gk, gk0)
        _close(gx, gx0)
    # a different plan in between keeps the results right (the array is fully rewritten)
    other, ko, uo, vo = _plan(3, (65, 66, 67, 68))
    Lo0, _, gxo0 = other.adjoint(ko, uo, vo)
    Lo, _, gxo = _noalloc(other, ko, uo, vo)
    _close(Lo, Lo0)
    _close(gxo, gxo0)
    L, gk, gx = _noalloc(plan, kap, u, vv)
    _close(gx, gx0)


def test_noalloc_python_wrapper_with_vertex_override():
    # Plan.adjoint_noalloc (argument checks + the C call) with moved vertices,
    # against fe_adjoint with the same vertices
    plan, kap, u, vv = _plan(4, (71, 72, 73, 74))
    moved = torch.from_numpy(inputs.cube_mesh(4, 0.15, 75)[0]).cuda()
    L = torch.empty(1, dtype=torch.float64, device="cuda")
    gk = torch.empty((plan.n_cells, plan.n_q), dtype=torch.float64, device="cuda")
    gx = torch.empty((plan.n_vertices, 3), dtype=torch.float64, device="cuda")
    plan.adjoint_noalloc(kap, u, vv, L, gk, gx, vertices=moved)
    plan.sync()
    L0, gk0, gx0 = plan.adjoint(kap, u, vv, vertices=moved)
    plan.sync()
    _close(L, L0)
    _close(gk, gk0)
    _close(gx, gx0)
    with pytest.raises(ValueError):
        plan.adjoint_noalloc(kap, u, vv, L, gk, gx, vertices=moved.float())


def test_noalloc_rejects_plans_above_capacity():
    # 6 * 39^3 = 355,914 tetrahedra > 322,638: too many for vertex gradients,
    # but within the capacity when only L and dL/dkappa are requested
    v, c = inputs.cube_mesh(39, 0.1, 1)
    pts, w = api.quadrature_rule("tetrahedron", 2)
    plan = api.Plan("tetrahedron", v, c, 1, pts, w, forms=("stiffness",), precisions=("bf16",))
    kap = torch.from_numpy(inputs.lognormal_kappa(plan.n_cells, plan.n_q, 2)).cuda()
    u = torch.from_numpy(inputs.gaussian_vector(plan.n_dofs, 3)).cuda()
    vv = torch.from_numpy(inputs.gaussian_vector(plan.n_dofs, 4)).cuda()
    with pytest.raises(_lib.FeError) as e:
        _noalloc(plan, kap, u, vv, want_vertices=True)
    assert e.value.status == -2 and "capacity" in str(e.value)
    L, gk, _ = _noalloc(plan, kap, u, vv, want_vertices=False)
    L0, gk0, _ = plan.adjoint(kap, u, vv, want_vertices=False)
    _close(L, L0)
    _close(gk, gk0)
