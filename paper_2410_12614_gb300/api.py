"""PyTorch-facing binding of the C ABI.

PyTorch provides device memory, streams and autograd plumbing only; every
step of the computation runs in the library's CUDA kernels.  All names follow
include/fe_gb300.h.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import FE_FORM_MASS, FE_FORM_STIFFNESS, PRECISIONS, check, load

FORMS = {"stiffness": FE_FORM_STIFFNESS, "mass": FE_FORM_MASS}


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def quadrature_rule(cell_type: str, m: int, family: int | None = None):
    """Reference rule from the library's host helper: (points [n_q, d], weights [n_q]) float64 numpy.
    Default family: collapsed Gauss-Jacobi on simplices, tensor Gauss-Legendre on boxed cells."""
    lib = load()
    t, d = _lib.CELL_TYPES[cell_type]
    if family is None:
        boxed = t in (_lib.FE_QUADRILATERAL, _lib.FE_HEXAHEDRON)
        family = _lib.FE_QUAD_GAUSS_LEGENDRE_TENSOR if boxed else _lib.FE_QUAD_COLLAPSED_GAUSS_JACOBI
    nq = ctypes.c_int32(0)
    check(lib.fe_quadrature_rule(t, family, m, ctypes.byref(nq), None, None), "fe_quadrature_rule")
    pts = np.zeros((nq.value, d))
    wts = np.zeros(nq.value)
    check(lib.fe_quadrature_rule(t, family, m, ctypes.byref(nq), pts.ctypes.data, wts.ctypes.data),
          "fe_quadrature_rule")
    return pts, wts


class Pattern:
    """Host-only dof map and CSR pattern (fe_pattern_*)."""

    def __init__(self, cell_type: str, n_vertices: int, cells, degree: int):
        lib = load()
        cells = np.ascontiguousarray(cells, dtype=np.int32)
        t, _ = _lib.CELL_TYPES[cell_type]
        h = ctypes.c_void_p()
        check(lib.fe_pattern_create(ctypes.byref(h), t, n_vertices, cells.shape[0], cells.ctypes.data, degree),
              "fe_pattern_create")
        self._h = h
        nd, nnz = ctypes.c_int64(), ctypes.c_int64()
        nph, mr = ctypes.c_int32(), ctypes.c_int32()
        check(lib.fe_pattern_sizes(h, ctypes.byref(nd), ctypes.byref(nnz), ctypes.byref(nph), ctypes.byref(mr)))
        self.n_dofs, self.nnz, self.n_phi, self.max_row = nd.value, nnz.value, nph.value, mr.value
        self.n_cells = cells.shape[0]

    def arrays(self):
        dofs = np.zeros((self.n_cells, self.n_phi), dtype=np.int32)
        rp = np.zeros(self.n_dofs + 1, dtype=np.int64)
        ci = np.zeros(self.nnz, dtype=np.int32)
        check(load().fe_pattern_copy(self._h, dofs.ctypes.data, rp.ctypes.data, ci.ctypes.data), "fe_pattern_copy")
        return dofs, rp, ci

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            load().fe_pattern_destroy(h)
            self._h = None


class Plan:
    """One mesh, degree and quadrature rule on the current CUDA device (fe_plan_*)."""

    def __init__(self, cell_type: str, vertices, cells, degree: int, points=None, weights=None,
                 forms=("stiffness", "mass"), precisions=("bf16",), stream: torch.cuda.Stream | None = None,
                 elements_only: bool = False):
        lib = load()
        t, self.d = _lib.CELL_TYPES[cell_type]
        self.cell_type = {_lib.FE_TRIANGLE: "triangle", _lib.FE_TETRAHEDRON: "tetrahedron",
                          _lib.FE_QUADRILATERAL: "quadrilateral", _lib.FE_HEXAHEDRON: "hexahedron"}[t]
        self.boxed = t in (_lib.FE_QUADRILATERAL, _lib.FE_HEXAHEDRON)
        vertices = np.ascontiguousarray(np.asarray(vertices, dtype=np.float64))
        cells = np.ascontiguousarray(np.asarray(cells, dtype=np.int32))
        if points is None:
            points, weights = quadrature_rule(self.cell_type, degree + 1)
        points = np.ascontiguousarray(points, dtype=np.float64)
        weights = np.ascontiguousarray(weights, dtype=np.float64)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        mesh = _lib.FeMesh(t, vertices.shape[0], vertices.ctypes.data, cells.shape[0], cells.ctypes.data)
        rule = _lib.FeQuadrature(weights.shape[0], points.ctypes.data, weights.ctypes.data)
        fmask = 0
        for f in forms:
            fmask |= FORMS[f]
        if elements_only:
            fmask |= 0x100   # FE_PLAN_ELEMENTS_ONLY
        pmask = 0
        for p in precisions:
            pmask |= 1 << PRECISIONS[p]
        h = ctypes.c_void_p()
        check(lib.fe_plan_create(ctypes.byref(h), ctypes.byref(mesh), degree, ctypes.byref(rule), fmask, pmask,
                                 ctypes.c_void_p(self.stream.cuda_stream)), "fe_plan_create")
        self._h = h
        nc, nv, nd, nnz = (ctypes.c_int64() for _ in range(4))
        nph, nq = ctypes.c_int32(), ctypes.c_int32()
        check(lib.fe_plan_sizes(h, ctypes.byref(nc), ctypes.byref(nv), ctypes.byref(nd), ctypes.byref(nnz),
                                ctypes.byref(nph), ctypes.byref(nq)))
        self.n_cells, self.n_vertices, self.n_dofs, self.nnz = nc.value, nv.value, nd.value, nnz.value
        self.n_phi, self.n_q = nph.value, nq.value
        self.degree = degree
        self.forms = tuple(forms)
        self.precisions = tuple(precisions)
        self.device = torch.device("cuda", torch.cuda.current_device())

    # -- helpers ----------------------------------------------------------
    def _dtype(self, prec):
        return torch.float64 if prec == "fp64" else torch.float32

    def _forms_mask(self, forms):
        m = 0
        for f in forms:
            m |= FORMS[f]
        return m

    def _check_dev(self, t, dtype, shape, name):
        if t is None:
            return
        if not t.is_cuda or t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor of shape {tuple(shape)}")

    def empty_elements(self, prec):
        return torch.empty((self.n_cells, self.n_phi, self.n_phi), dtype=self._dtype(prec), device=self.device)

    def empty_values(self, prec):
        return torch.empty(self.nnz, dtype=self._dtype(prec), device=self.device)

    # -- queries ------------------------------------------------------------
    def csr_pattern(self):
        rp = torch.empty(self.n_dofs + 1, dtype=torch.int64, device=self.device)
        ci = torch.empty(self.nnz, dtype=torch.int32, device=self.device)
        check(load().fe_csr_pattern(self._h, _ptr(rp), _ptr(ci)), "fe_csr_pattern")
        return rp, ci

    def cell_dofs(self):
        out = torch.empty((self.n_cells, self.n_phi), dtype=torch.int32, device=self.device)
        check(load().fe_cell_dofs(self._h, _ptr(out)), "fe_cell_dofs")
        return out

    # -- compute ------------------------------------------------------------
    def element_matrices(self, kappa, forms=("stiffness", "mass"), prec="bf16", vertices=None, out=None):
        self._check_dev(kappa, torch.float64, (self.n_cells, self.n_q), "kappa")
        self._check_dev(vertices, torch.float64, (self.n_vertices, self.d), "vertices")
        out = dict(out or {})
        for f in forms:
            if f not in out:
                out[f] = self.empty_elements(prec)
            self._check_dev(out[f], self._dtype(prec), (self.n_cells, self.n_phi, self.n_phi), f)
        check(load().fe_element_matrices(self._h, self._forms_mask(forms), PRECISIONS[prec], _ptr(vertices),
                                         _ptr(kappa), _ptr(out.get("stiffness")), _ptr(out.get("mass"))),
              "fe_element_matrices")
        return out

    def assemble(self, kappa, forms=("stiffness", "mass"), prec="bf16", vertices=None, elements=None, out=None):
        """CSR values per form; ``elements`` (dict) receives the element matrices if given."""
        self._check_dev(kappa, torch.float64, (self.n_cells, self.n_q), "kappa")
        self._check_dev(vertices, torch.float64, (self.n_vertices, self.d), "vertices")
        out = dict(out or {})
        for f in forms:
            if f not in out:
                out[f] = self.empty_values(prec)
            self._check_dev(out[f], self._dtype(prec), (self.nnz,), f)
        el = elements or {}
        check(load().fe_assemble(self._h, self._forms_mask(forms), PRECISIONS[prec], _ptr(vertices), _ptr(kappa),
                                 _ptr(el.get("stiffness")), _ptr(el.get("mass")), _ptr(out.get("stiffness")),
                                 _ptr(out.get("mass"))), "fe_assemble")
        return out

    def assemble_elements(self, elements, prec="bf16", out=None):
        forms = tuple(elements.keys())
        out = dict(out or {})
        for f in forms:
            if f not in out:
                out[f] = self.empty_values(prec)
        check(load().fe_assemble_elements(self._h, self._forms_mask(forms), PRECISIONS[prec],
                                          _ptr(elements.get("stiffness")), _ptr(elements.get("mass")),
                                          _ptr(out.get("stiffness")), _ptr(out.get("mass"))), "fe_assemble_elements")
        return out

    def assemble_host(self, kappa_host, forms=("stiffness", "mass"), prec="bf16", out=None):
        """End to end with host buffers: kappa (CPU float64, pinned preferred) -> CSR values (CPU)."""
        if kappa_host.is_cuda or kappa_host.dtype != torch.float64 or not kappa_host.is_contiguous():
            raise ValueError("kappa_host must be a contiguous CPU float64 tensor")
        out = dict(out or {})
        for f in forms:
            if f not in out:
                out[f] = torch.empty(self.nnz, dtype=self._dtype(prec), pin_memory=True)
        check(load().fe_assemble_host(self._h, self._forms_mask(forms), PRECISIONS[prec], _ptr(kappa_host),
                                      _ptr(out.get("stiffness")), _ptr(out.get("mass"))), "fe_assemble_host")
        return out

    def assemble_host_many(self, kappas_host, outs, forms=("stiffness", "mass"), prec="bf16"):
        """fe_assemble_host_many: a sequence of host coefficient sets (contiguous
        CPU float64 tensors, pinned preferred) -> their CSR values in the host
        tensors outs[i][form]; uploads, computation and downloads overlap."""
        n = len(kappas_host)
        for k in kappas_host:
            if k.is_cuda or k.dtype != torch.float64 or not k.is_contiguous():
                raise ValueError("kappa_host entries must be contiguous CPU float64 tensors")
        kap = (ctypes.c_void_p * n)(*[ctypes.c_void_p(k.data_ptr()) for k in kappas_host])
        arrs = {}
        for f in ("stiffness", "mass"):
            arrs[f] = (ctypes.c_void_p * n)(*[ctypes.c_void_p(o[f].data_ptr()) for o in outs]) if f in forms else None
        check(load().fe_assemble_host_many(self._h, self._forms_mask(forms), PRECISIONS[prec], n, kap,
                                           arrs["stiffness"], arrs["mass"]), "fe_assemble_host_many")
        return outs

    def action(self, kappa, w, forms=("stiffness", "mass"), prec="fp64", vertices=None, cell_vectors=False,
               out=None):
        """Algorithm 2: v^g = L b with b^c_j = a_K(w, phi_j) for the FE function with
        coefficients w (fe_action).  Returns {form: v [n_dofs]} (and, with
        cell_vectors, {form: b [n_cells, n_phi]} as a second value)."""
        self._check_dev(kappa, torch.float64, (self.n_cells, self.n_q), "kappa")
        self._check_dev(w, torch.float64, (self.n_dofs,), "w")
        self._check_dev(vertices, torch.float64, (self.n_vertices, self.d), "vertices")
        dt = torch.float64 if prec == "fp64" else torch.float32
        v = out if out is not None else {f: torch.empty(self.n_dofs, dtype=dt, device=self.device) for f in forms}
        b = {f: torch.empty((self.n_cells, self.n_phi), dtype=dt, device=self.device) for f in forms} \
            if cell_vectors else {}
        check(load().fe_action(self._h, self._forms_mask(forms), PRECISIONS[prec], _ptr(vertices), _ptr(kappa),
                               _ptr(w), _ptr(b.get("stiffness")), _ptr(b.get("mass")), _ptr(v.get("stiffness")),
                               _ptr(v.get("mass"))), "fe_action")
        return (v, b) if cell_vectors else v

    def adjoint(self, kappa, u, v, vertices=None, want_kappa=True, want_vertices=True, want_L=True):
        """(L, dL/dkappa, dL/dvertices) for L = v^T A_stiffness u, computed in FP64."""
        self._check_dev(kappa, torch.float64, (self.n_cells, self.n_q), "kappa")
        self._check_dev(u, torch.float32, (self.n_dofs,), "u")
        self._check_dev(v, torch.float32, (self.n_dofs,), "v")
        self._check_dev(vertices, torch.float64, (self.n_vertices, self.d), "vertices")
        gk = torch.empty((self.n_cells, self.n_q), dtype=torch.float64, device=self.device) if want_kappa else None
        gx = torch.empty((self.n_vertices, self.d), dtype=torch.float64, device=self.device) if want_vertices else None
        L = torch.empty(1, dtype=torch.float64, device=self.device) if want_L else None
        check(load().fe_adjoint(self._h, _ptr(vertices), _ptr(kappa), _ptr(u), _ptr(v), _ptr(gk), _ptr(gx), _ptr(L)),
              "fe_adjoint")
        return L, gk, gx

    def adjoint_values(self, kappa, grad_values, vertices=None, want_kappa=True, want_vertices=True, want_L=True):
        """(L, dL/dkappa, dL/dvertices) for L = sum_e g_e A^g_e (stiffness) with the
        gradient g (grad_values, [nnz], any float dtype) on the CSR values; FP64."""
        self._check_dev(kappa, torch.float64, (self.n_cells, self.n_q), "kappa")
        self._check_dev(vertices, torch.float64, (self.n_vertices, self.d), "vertices")
        g = grad_values.detach().to(torch.float64).contiguous()
        if g.device.type != "cuda" or g.numel() != self.nnz:
            raise ValueError(f"grad_values: expected a CUDA tensor of {self.nnz} values")
        gk = torch.empty((self.n_cells, self.n_q), dtype=torch.float64, device=self.device) if want_kappa else None
        gx = torch.empty((self.n_vertices, self.d), dtype=torch.float64, device=self.device) if want_vertices else None
        L = torch.empty(1, dtype=torch.float64, device=self.device) if want_L else None
        check(load().fe_adjoint_values(self._h, _ptr(vertices), _ptr(kappa), _ptr(g), _ptr(gk), _ptr(gx), _ptr(L)),
              "fe_adjoint_values")
        return L, gk, gx

    def adjoint_noalloc(self, kappa, u, v, out_L, out_kappa=None, out_vertices=None, vertices=None):
        """fe_adjoint_noalloc: the adjoint without any device allocation by the
        library; the caller provides every output buffer."""
        self._check_dev(kappa, torch.float64, (self.n_cells, self.n_q), "kappa")
        self._check_dev(u, torch.float32, (self.n_dofs,), "u")
        self._check_dev(v, torch.float32, (self.n_dofs,), "v")
        self._check_dev(out_L, torch.float64, (1,), "out_L")
        self._check_dev(out_kappa, torch.float64, (self.n_cells, self.n_q), "out_kappa")
        self._check_dev(out_vertices, torch.float64, (self.n_vertices, self.d), "out_vertices")
        self._check_dev(vertices, torch.float64, (self.n_vertices, self.d), "vertices")
        check(load().fe_adjoint_noalloc(self._h, _ptr(vertices), _ptr(kappa), _ptr(u), _ptr(v), _ptr(out_kappa),
                                        _ptr(out_vertices), _ptr(out_L)), "fe_adjoint_noalloc")

    def sync(self):
        check(load().fe_sync_status(self._h), "fe_sync_status")

    # -- diagnostics (the paper's error studies) -------------------------------
    GEOMETRY_MODES = {"fp64": 0, "fp32": 1, "mixed": 2}

    def geometry(self, mode="fp64", vertices=None, cells=None):
        """fe_geometry: (G [n, d(d+1)/2], |det J| [n], used_fp64 [n]) of the
        cells range(*cells) (default: all) as float64 / int32 CUDA tensors."""
        self._check_dev(vertices, torch.float64, (self.n_vertices, self.d), "vertices")
        c0, c1 = cells if cells is not None else (0, self.n_cells)
        n = c1 - c0
        G = torch.empty((n, self.d * (self.d + 1) // 2), dtype=torch.float64, device=self.device)
        ad = torch.empty(n, dtype=torch.float64, device=self.device)
        used = torch.zeros(n, dtype=torch.int32, device=self.device)
        check(load().fe_geometry(self._h, self.GEOMETRY_MODES[mode], _ptr(vertices), c0, c1, _ptr(G), _ptr(ad),
                                 _ptr(used)), "fe_geometry")
        return G, ad, used

    def mass_fp16_products(self, kappa, w=None, cells=None, matrices=True):
        """fe_mass_fp16_products: the mass matrices (and, with w, the mass
        action) of the cells range(*cells) with FP16 products and sums."""
        self._check_dev(kappa, torch.float64, (self.n_cells, self.n_q), "kappa")
        self._check_dev(w, torch.float64, (self.n_dofs,), "w")
        c0, c1 = cells if cells is not None else (0, self.n_cells)
        n = c1 - c0
        A = torch.empty((n, self.n_phi, self.n_phi), dtype=torch.float32, device=self.device) if matrices else None
        b = torch.empty((n, self.n_phi), dtype=torch.float32, device=self.device) if w is not None else None
        check(load().fe_mass_fp16_products(self._h, _ptr(kappa), _ptr(w), c0, c1, _ptr(A), _ptr(b)),
              "fe_mass_fp16_products")
        return A, b

    def set_wait_limit(self, limit_ns: int = 0):
        """fe_plan_set_wait_limit: the longest one bounded wait inside the
        plan's kernels may see no progress (0 restores the default)."""
        check(load().fe_plan_set_wait_limit(self._h, int(limit_ns)), "fe_plan_set_wait_limit")

    def set_fusion(self, mode: int = 1) -> bool:
        """fe_plan_set_fusion: 1 on, 0 off (the default); returns whether
        fe_assemble without element-matrix outputs takes the fused path."""
        act = ctypes.c_int32()
        check(load().fe_plan_set_fusion(self._h, int(mode), ctypes.byref(act)), "fe_plan_set_fusion")
        return bool(act.value)

    def set_assembly(self, algo: int = 0):
        """fe_plan_set_assembly: 0 the chunked segmented reduction (default), 1
        one warp per CSR row; the CSR values are bitwise the same."""
        check(load().fe_plan_set_assembly(self._h, int(algo)), "fe_plan_set_assembly")

    def set_window_prefetch(self, mode: int = -1):
        """fe_plan_set_window_prefetch: -1 as autotuned (default), 0 off, 1 on; the
        element matrices are bitwise the same."""
        check(load().fe_plan_set_window_prefetch(self._h, int(mode)), "fe_plan_set_window_prefetch")

    def set_rows_per_pass(self, rows: int, forms=("stiffness", "mass"), prec="bf16"):
        """fe_plan_set_rows_per_pass: whole-row passes of `rows` rows (wide above
        256 columns) for these forms in this precision, instead of the tuned layout."""
        check(load().fe_plan_set_rows_per_pass(self._h, PRECISIONS[prec], self._forms_mask(forms), int(rows)),
              "fe_plan_set_rows_per_pass")

    def tc_config(self, forms=("stiffness", "mass"), prec="bf16"):
        """fe_plan_tc_config: the tensor-core launch shape for these forms and
        precision, as a dict (ring_a, ring_b, win_buf, staged, n_acc)."""
        v = [ctypes.c_int32() for _ in range(5)]
        check(load().fe_plan_tc_config(self._h, self._forms_mask(forms), PRECISIONS[prec],
                                       *[ctypes.byref(x) for x in v]), "fe_plan_tc_config")
        return dict(zip(("ring_a", "ring_b", "win_buf", "staged", "n_acc"), (x.value for x in v)))

    def memory(self):
        """(plan_bytes, workspace_bytes) of device memory the plan holds (fe_plan_memory)."""
        pb, wb = ctypes.c_int64(), ctypes.c_int64()
        check(load().fe_plan_memory(self._h, ctypes.byref(pb), ctypes.byref(wb)), "fe_plan_memory")
        return pb.value, wb.value

    def enable_timing(self, on=True):
        check(load().fe_plan_enable_timing(self._h, int(on)))

    def stage_times(self):
        ms = (ctypes.c_float * 4)()
        check(load().fe_plan_stage_times(self._h, ms, 4))
        return list(ms)

    def last_launches(self):
        n = ctypes.c_int32()
        check(load().fe_plan_last_launches(self._h, ctypes.byref(n)))
        return n.value

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            load().fe_plan_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several plans run as one persistent launch + one assembly launch, captured
    in a CUDA graph (fe_batch_*).  Buffers are fixed at creation and reused by
    every run()."""

    def __init__(self, plans, kappas, forms=("stiffness", "mass"), prec="bf16", elements=True, assemble=True,
                 stream: torch.cuda.Stream | None = None):
        lib = load()
        self.plans = list(plans)
        n = len(self.plans)
        self.forms = tuple(forms)
        self.prec = prec
        self.stream = stream if stream is not None else self.plans[0].stream
        for p, k in zip(self.plans, kappas):
            p._check_dev(k, torch.float64, (p.n_cells, p.n_q), "kappa")
        self.kappas = list(kappas)
        self.elements = {f: [p.empty_elements(prec) for p in self.plans] if elements else None for f in forms}
        self.values = {f: [p.empty_values(prec) for p in self.plans] if assemble else None for f in forms}
        arr = lambda xs: (ctypes.c_void_p * n)(*[ctypes.c_void_p(x.data_ptr()) for x in xs]) if xs is not None else None
        self._keep = [(ctypes.c_void_p * n)(*[p._h for p in self.plans])]
        kap = (ctypes.c_void_p * n)(*[ctypes.c_void_p(k.data_ptr()) for k in self.kappas])
        a_s = arr(self.elements.get("stiffness")) if "stiffness" in forms and elements else None
        a_m = arr(self.elements.get("mass")) if "mass" in forms and elements else None
        c_s = arr(self.values.get("stiffness")) if "stiffness" in forms and assemble else None
        c_m = arr(self.values.get("mass")) if "mass" in forms and assemble else None
        self._keep += [kap, a_s, a_m, c_s, c_m]
        mask = 0
        for f in forms:
            mask |= FORMS[f]
        h = ctypes.c_void_p()
        check(lib.fe_batch_create(ctypes.byref(h), self._keep[0], n, mask, PRECISIONS[prec], kap, a_s, a_m, c_s, c_m,
                                  ctypes.c_void_p(self.stream.cuda_stream)), "fe_batch_create")
        self._h = h
        nc, nnz = ctypes.c_int64(), ctypes.c_int64()
        nl = ctypes.c_int32()
        check(lib.fe_batch_sizes(h, ctypes.byref(nc), ctypes.byref(nnz), ctypes.byref(nl)))
        self.n_cells, self.nnz, self.launches = nc.value, nnz.value, nl.value

    def run(self):
        check(load().fe_batch_run(self._h), "fe_batch_run")

    def sync(self):
        check(load().fe_batch_sync(self._h), "fe_batch_sync")

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            load().fe_batch_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class AssembleStiffness(torch.autograd.Function):
    """values = assemble(kappa, vertices): the CSR values of the stiffness form
    (fe_assemble in the given precision).  The backward takes any gradient on
    the values and returns dL/dkappa and dL/dvertices from the FP64 adjoint
    fe_adjoint_values (kappa at the quadrature points held fixed when the
    vertices move), i.e. the gradient of the exact quadrature form."""

    @staticmethod
    def forward(ctx, kappa, vertices, plan, prec="fp64"):
        vals = plan.assemble(kappa, forms=("stiffness",), prec=prec, vertices=vertices)["stiffness"]
        ctx.save_for_backward(kappa, vertices)
        ctx.plan = plan
        return vals

    @staticmethod
    def backward(ctx, grad_values):
        kappa, vertices = ctx.saved_tensors
        _, gk, gx = ctx.plan.adjoint_values(kappa, grad_values, vertices=vertices, want_L=False,
                                            want_kappa=ctx.needs_input_grad[0],
                                            want_vertices=ctx.needs_input_grad[1])
        return gk, gx, None, None


class QuadraticForm(torch.autograd.Function):
    """L = v^T A(kappa, vertices) u for the stiffness form of a plan.

    Forward and backward both run the library's FP64 adjoint kernels
    (fe_adjoint); the backward recomputes the geometry from the vertices.
    Gradients flow to kappa and to the vertex coordinates (kappa at the
    quadrature points held fixed when the vertices move); u and v are treated
    as constants.
    """

    @staticmethod
    def forward(ctx, kappa, vertices, u, v, plan):
        L, _, _ = plan.adjoint(kappa, u, v, vertices=vertices, want_kappa=False, want_vertices=False)
        ctx.save_for_backward(kappa, vertices, u, v)
        ctx.plan = plan
        return L[0]

    @staticmethod
    def backward(ctx, grad_L):
        kappa, vertices, u, v = ctx.saved_tensors
        _, gk, gx = ctx.plan.adjoint(kappa, u, v, vertices=vertices, want_L=False,
                                     want_kappa=ctx.needs_input_grad[0], want_vertices=ctx.needs_input_grad[1])
        gk = gk * grad_L if gk is not None else None
        gx = gx * grad_L if gx is not None else None
        return gk, gx, None, None, None
