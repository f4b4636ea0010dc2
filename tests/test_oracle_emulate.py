"""Pins of the emulated-precision oracle (oracle/emulate.py), on the CPU.

* the rounding function against closed-form cases and against numpy's own
  float16 / float32 conversions (round to nearest even);
* with every rounding switched off, the folded P-form contraction reproduces
  the literal FP64 oracle (pins the pair folding, the [s != t] term, the
  mirroring and the scale bookkeeping);
* with rounding on, the emulated matrices sit within the paper's error bound
  of the exact ones (Corollary 4.10) and the FP32 geometry factor within a few
  FP32 units of the FP64 one.
"""
import numpy as np
import pytest

import oracle
from oracle import emulate
from paper_2410_12614_gb300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def test_round_format_closed_forms():
    bf = emulate.FORMATS["bf16"]
    assert emulate.round_format(1 + 2.0 ** -8, *bf) == 1.0                       # tie -> even
    assert emulate.round_format(1 + 3 * 2.0 ** -8, *bf) == 1 + 2.0 ** -6         # tie -> even (up)
    assert emulate.round_format(-(1 + 2.0 ** -7), *bf) == -(1 + 2.0 ** -7)      # representable
    e4 = emulate.FORMATS["e4m3"]
    assert emulate.round_format(17.0, *e4) == 16.0                               # tie -> even
    assert emulate.round_format(19.0, *e4) == 20.0
    assert emulate.round_format(500.0, *e4) == 448.0                             # saturates
    assert emulate.round_format(0.003, *e4) == 2 * 2.0 ** -9                     # subnormal quantum 2^-9
    assert emulate.round_format(2.0 ** -10, *e4) == 0.0                          # tie to even zero
    assert emulate.round_format(0.0, *e4) == 0.0
    # midpoints: 1 + 2^-8 is one for BF16, 1 + 2^-9 is not
    assert emulate.near_midpoint(1 + 2.0 ** -8, 7, -126) and not emulate.near_midpoint(1 + 2.0 ** -9, 7, -126)
    assert emulate.quantum(1.5, 7, -126) == 2.0 ** -7 and emulate.quantum(2.0 ** -130, 7, -126) == 2.0 ** -133


def test_round_format_matches_numpy_casts():
    rng = np.random.default_rng(7)
    x = (rng.standard_normal(200000) * np.exp(rng.uniform(-30, 30, 200000))).astype(np.float32)
    # FP16 (gradual underflow, finite range only)
    xs = x[np.abs(x) < 65000].astype(np.float64)
    assert np.array_equal(emulate.round_format(xs, *emulate.FORMATS["fp16"]), xs.astype(np.float16).astype(np.float64))
    # FP32 itself: rounding FP64 values with 23 mantissa bits equals numpy's cast
    y = rng.standard_normal(200000) * np.exp(rng.uniform(-60, 60, 200000))
    assert np.array_equal(emulate.round_format(y, 23, -126, 3.4028234663852886e38), y.astype(np.float32).astype(np.float64))
    # TF32: 10 bits by integer rounding of the FP32 pattern
    u = x.view(np.uint32).astype(np.uint64)
    t = ((u + 0xFFF + ((u >> 13) & 1)) & 0xFFFFE000).astype(np.uint32).view(np.float32).astype(np.float64)
    fin = np.isfinite(t) & (np.abs(x) > 2.0 ** -126)
    assert np.array_equal(emulate.round_format(x.astype(np.float64), *emulate.FORMATS["tf32"])[fin], t[fin])


CASES = [("triangle", 3, 1), ("triangle", 2, 3), ("tetrahedron", 2, 1), ("tetrahedron", 2, 2), ("tetrahedron", 1, 3)]


def _problem(cell, n, p, seed):
    v, c = inputs.structured_mesh(cell, n, 0.15, seed)
    ref = oracle.Problem(v, c, p, *oracle.rule_for_degree(cell, p))
    kap = inputs.lognormal_kappa(ref.n_cells, ref.n_q, seed + 1)
    return ref, kap


@pytest.mark.parametrize("cell,n,p", CASES)
def test_exact_mode_is_the_literal_oracle(cell, n, p):
    ref, kap = _problem(cell, n, p, 30 + p)
    for form in ("stiffness", "mass"):
        A = ref.element_matrices(kap, form)
        E, M, K, _ = emulate.element_matrices(ref, kap, form, "bf16", exact=True)
        assert np.abs(E - A).max() <= 1e-12 * np.abs(A).max()
        assert K == ref.n_q * (ref.d * (ref.d + 1) // 2 if form == "stiffness" else 1)


@pytest.mark.parametrize("cell,n,p", CASES)
def test_rounded_operands_within_the_bound(cell, n, p):
    ref, kap = _problem(cell, n, p, 40 + p)
    u_s = {"bf16": 2.0 ** -8, "fp16": 2.0 ** -11, "tf32": 2.0 ** -11, "tf32x3": 2.0 ** -21, "e4m3": 2.0 ** -4}
    for form in ("stiffness", "mass"):
        A = ref.element_matrices(kap, form)
        kq = ref.kappa_q(kap, form, A)
        for prec in ("bf16", "fp16", "tf32", "tf32x3", "e4m3"):
            E, _, K, _ = emulate.element_matrices(ref, kap, form, prec)
            err = np.abs(E - A).reshape(len(A), -1).max(1) / np.abs(A).reshape(len(A), -1).max(1)
            r = 4 if prec == "e4m3" else 2
            # no accumulation error here (FP64 sums): only the operand roundings and the FP32 factor
            bnd = (r * u_s[prec] + 8 * 2.0 ** -24) * kq
            assert np.all(err <= bnd), (form, prec, float(err.max()))


def test_fp32_geometry_factor_close_to_fp64():
    ref, _ = _problem("tetrahedron", 3, 1, 50)
    det, G = oracle.mesh_geometry(ref.vertices, ref.cells)
    G32, a32 = emulate.geometry32(ref.vertices, ref.cells, g64=False)
    iu = [(s, t) for s in range(3) for t in range(s, 3)]
    Gp = np.stack([G[:, s, t] for s, t in iu], axis=1)
    scale = np.abs(Gp).max(axis=1, keepdims=True)
    assert np.abs(G32 - Gp).max() <= 8 * 2.0 ** -24 * scale.max()
    assert np.allclose(a32, np.abs(det), rtol=2.0 ** -23, atol=0)
