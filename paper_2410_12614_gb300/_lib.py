"""ctypes loader for libfe_gb300.so (the C ABI in include/fe_gb300.h).

Argument marshalling only.  If the compiled library is missing the import of
the package still works, but every call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libfe_gb300.so")

FE_OK = 0
STATUS_NAMES = {
    0: "FE_OK",
    -1: "FE_ERR_INVALID_ARG",
    -2: "FE_ERR_UNSUPPORTED",
    -3: "FE_ERR_DEGENERATE_CELL",
    -4: "FE_ERR_NONFINITE",
    -5: "FE_ERR_OOM",
    -6: "FE_ERR_CUDA",
    -7: "FE_ERR_TIMEOUT",
    -8: "FE_ERR_NO_DEVICE",
}
FE_TRIANGLE, FE_TETRAHEDRON, FE_QUADRILATERAL, FE_HEXAHEDRON = 2, 3, 4, 5
FE_FORM_MASS, FE_FORM_STIFFNESS = 1, 2
PRECISIONS = {"fp64": 0, "tf32x3": 1, "tf32": 2, "bf16": 3, "fp16": 4, "e4m3": 5}
FE_QUAD_COLLAPSED_GAUSS_JACOBI, FE_QUAD_TRIANGLE_3POINT, FE_QUAD_GAUSS_LEGENDRE_TENSOR = 0, 1, 2
CELL_TYPES = {"triangle": (FE_TRIANGLE, 2), "tri": (FE_TRIANGLE, 2), "tetrahedron": (FE_TETRAHEDRON, 3),
              "tet": (FE_TETRAHEDRON, 3), "quadrilateral": (FE_QUADRILATERAL, 2), "quad": (FE_QUADRILATERAL, 2),
              "hexahedron": (FE_HEXAHEDRON, 3), "hex": (FE_HEXAHEDRON, 3)}

# every exported symbol, with (restype, argtypes)
_vp, _i32, _i64, _u32, _dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_void_p
_pi32, _pi64 = ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)


class FeMesh(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("n_vertices", ctypes.c_int64), ("vertices", ctypes.c_void_p),
                ("n_cells", ctypes.c_int64), ("cells", ctypes.c_void_p)]


class FeQuadrature(ctypes.Structure):
    _fields_ = [("n_q", ctypes.c_int32), ("points", ctypes.c_void_p), ("weights", ctypes.c_void_p)]


SIGNATURES = {
    "fe_quadrature_rule": [ctypes.c_int, ctypes.c_int, ctypes.c_int, _pi32, _vp, _vp],
    "fe_pattern_create": [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, _i64, _i64, _vp, ctypes.c_int],
    "fe_pattern_sizes": [_vp, _pi64, _pi64, _pi32, _pi32],
    "fe_pattern_copy": [_vp, _vp, _vp, _vp],
    "fe_pattern_destroy": [_vp],
    "fe_last_error": [],
    "fe_plan_create": [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(FeMesh), ctypes.c_int,
                       ctypes.POINTER(FeQuadrature), ctypes.c_uint, ctypes.c_uint, _vp],
    "fe_plan_destroy": [_vp],
    "fe_plan_set_stream": [_vp, _vp],
    "fe_plan_set_wait_limit": [_vp, ctypes.c_uint64],
    "fe_plan_set_fusion": [_vp, ctypes.c_int, _pi32],
    "fe_plan_set_assembly": [_vp, ctypes.c_int],
    "fe_plan_set_window_prefetch": [_vp, ctypes.c_int],
    "fe_plan_set_rows_per_pass": [_vp, ctypes.c_int, ctypes.c_uint, ctypes.c_int],
    "fe_plan_tc_config": [_vp, ctypes.c_uint, ctypes.c_int, _pi32, _pi32, _pi32, _pi32, _pi32],
    "fe_plan_memory": [_vp, _pi64, _pi64],
    "fe_plan_sizes": [_vp, _pi64, _pi64, _pi64, _pi64, _pi32, _pi32],
    "fe_csr_pattern": [_vp, _vp, _vp],
    "fe_cell_dofs": [_vp, _vp],
    "fe_element_matrices": [_vp, ctypes.c_uint, ctypes.c_int, _vp, _vp, _vp, _vp],
    "fe_assemble": [_vp, ctypes.c_uint, ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _vp],
    "fe_assemble_host": [_vp, ctypes.c_uint, ctypes.c_int, _vp, _vp, _vp],
    "fe_assemble_host_many": [_vp, ctypes.c_uint, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp],
    "fe_assemble_elements": [_vp, ctypes.c_uint, ctypes.c_int, _vp, _vp, _vp, _vp],
    "fe_adjoint": [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "fe_adjoint_values": [_vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "fe_action": [_vp, ctypes.c_uint, ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "fe_adjoint_noalloc": [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "fe_geometry": [_vp, ctypes.c_int, _vp, _i64, _i64, _vp, _vp, _vp],
    "fe_mass_fp16_products": [_vp, _vp, _vp, _i64, _i64, _vp, _vp],
    "fe_sync_status": [_vp],
    "fe_batch_create": [ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p, ctypes.c_int, ctypes.c_uint, ctypes.c_int,
                        _vp, _vp, _vp, _vp, _vp, _vp],
    "fe_batch_run": [_vp],
    "fe_batch_sync": [_vp],
    "fe_batch_sizes": [_vp, _pi64, _pi64, _pi32],
    "fe_batch_destroy": [_vp],
    "fe_plan_enable_timing": [_vp, ctypes.c_int],
    "fe_plan_stage_times": [_vp, ctypes.POINTER(ctypes.c_float), ctypes.c_int],
    "fe_plan_last_launches": [_vp, _pi32],
}

_lock = threading.Lock()
_lib = None


class FeError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load(path: str | None = None):
    """Load (once) and return the CDLL with typed signatures."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise FeError(-6, f"{p} is missing: build it with __graft_entry__.build() "
                                  "(the GPU path has no fallback)")
            lib = ctypes.CDLL(p)
            for name, args in SIGNATURES.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = ctypes.c_char_p if name == "fe_last_error" else ctypes.c_int
            _lib = lib
    return _lib


def check(status: int, what: str = ""):
    if status != FE_OK:
        msg = load().fe_last_error().decode(errors="replace")
        raise FeError(status, f"{what}: {msg}" if what else msg)
