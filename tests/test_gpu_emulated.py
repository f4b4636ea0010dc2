"""The tensor-core kernels against the emulated-precision oracle.

oracle/emulate.py rounds C and P to the storage format as the mixed kernels
are specified to and accumulates in FP64; the kernels may then differ from it
only by their FP32 accumulation and the FP32 store:

    |A_gpu - A_emul| <= gamma_K(2 u_acc) sum |C||P| + u_out |A_emul| + slack,

the slack covering the difference between two FP64 tabulations of P (~2^-46
max|P| on entries near zero, one storage unit where an entry lies within 2^-40
of a rounding midpoint),

a tolerance orders of magnitude below the error bound of Corollary 4.10.  A
wrong rounding mode, scale, split or operand layout shows up here even where
it would hide inside the bound.
"""
import numpy as np
import pytest

from oracle import emulate

from gpu_util import cuda, make_case, to_np

pytestmark = pytest.mark.gpu

ALL_LOW = ("bf16", "fp16", "tf32", "tf32x3", "e4m3")
CASES = [("triangle", 3, 1), ("triangle", 2, 3), ("triangle", 2, 5), ("tetrahedron", 2, 1),
         ("tetrahedron", 2, 2), ("tetrahedron", 3, 3), ("tetrahedron", 1, 5)]


@pytest.mark.parametrize("cell,n,p", CASES)
def test_kernels_match_emulated_operands(cell, n, p):
    plan, ref, kap = make_case(cell, n, p, 0.15, 60 + p, 61 + p, precisions=ALL_LOW)
    kd = cuda(kap)
    worst = {}
    for form in ("stiffness", "mass"):
        for prec in ALL_LOW:
            got = to_np(plan.element_matrices(kd, forms=(form,), prec=prec)[form])
            plan.sync()
            E, M, K, slack = emulate.element_matrices(ref, kap, form, prec)
            x = K * 2 * 2.0 ** -23
            tol = x / (1 - x) * M + 2.0 ** -24 * np.abs(E) + slack
            ratio = np.abs(got - E) / np.maximum(tol, 1e-300)
            worst[(form, prec)] = float(ratio.max())
            assert np.all(np.abs(got - E) <= tol), (form, prec, float(ratio.max()))
    print({k: round(v, 4) for k, v in worst.items()})
