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
    """The emulated operands (FP64 sums, so no accumulation error) within the
    derived bound of oracle.error_bound with gamma = 0: (1+u)^r (1+u_pre) - 1
    times kappa_q^A plus the gradual-underflow term."""
    from gpu_util import FORMAT, ROUNDINGS, U_PRE, U_S
    ref, kap = _problem(cell, n, p, 40 + p)
    for form in ("stiffness", "mass"):
        A = ref.element_matrices(kap, form)
        kq = ref.kappa_q(kap, form, A)
        for prec in ("bf16", "fp16", "tf32", "tf32x3", "e4m3"):
            E, _, K, _ = emulate.element_matrices(ref, kap, form, prec)
            err = np.abs(E - A).reshape(len(A), -1).max(1) / np.abs(A).reshape(len(A), -1).max(1)
            sub = oracle.subnormal_term(ref, kap, form, A, *FORMAT[prec])
            bnd = oracle.error_bound(kq, U_S[prec], K, u_acc=0.0, u_out=0.0, storage_roundings=ROUNDINGS[prec],
                                     u_pre=U_PRE[prec], abs_rel=sub)
            assert np.all(err <= bnd), (form, prec, float((err / bnd).max()))


def test_gradual_underflow_needs_the_absolute_term():
    """In e4m3 (3 mantissa bits, smallest normal 2^-6, subnormal spacing 2^-9)
    a value in gradual underflow is rounded with an absolute error up to half
    the spacing, 2^-10, which relative to the value can exceed u = 2^-4 many
    times over: fl(1.4 * 2^-9) = 2^-9.  A contraction whose products fall
    there breaks the bound without the absolute term of subnormal_term and
    keeps it with that term."""
    mbits, emin, maxf = emulate.FORMATS["e4m3"]
    u, h = 2.0 ** -4, 2.0 ** (emin - mbits - 1)
    x = np.array([1.4, 1.6, 2.7, 3.5, 5.5]) * 2.0 ** -9
    r = emulate.round_format(x, mbits, emin, maxf)
    assert np.all(np.abs(r - x) <= h) and np.any(np.abs(r - x) > u * np.abs(x))
    # sum_i fl(C_i) fl(P_i): C normal (scaled to [2^7, 2^8)), P entries of one
    # column in gradual underflow
    rng = np.random.default_rng(3)
    C = rng.uniform(128, 256, 64)
    P = rng.uniform(1.1, 1.45, 64) * 2.0 ** -9
    exact = np.sum(C * P)
    got = np.sum(emulate.round_format(C, mbits, emin, maxf) * emulate.round_format(P, mbits, emin, maxf))
    rho = (1 + u) ** 2 - 1
    mag = np.sum(np.abs(C) * np.abs(P))
    assert abs(got - exact) > rho * mag                                  # the relative terms alone fail
    a_P = h                                                              # P unscaled: its eta bound
    assert abs(got - exact) <= rho * mag + (1 + u) * a_P * np.sum(np.abs(C))


def test_fp32_geometry_factor_close_to_fp64():
    ref, _ = _problem("tetrahedron", 3, 1, 50)
    det, G = oracle.mesh_geometry(ref.vertices, ref.cells)
    G32, a32 = emulate.geometry32(ref.vertices, ref.cells, g64=False)
    iu = [(s, t) for s in range(3) for t in range(s, 3)]
    Gp = np.stack([G[:, s, t] for s, t in iu], axis=1)
    scale = np.abs(Gp).max(axis=1, keepdims=True)
    assert np.abs(G32 - Gp).max() <= 8 * 2.0 ** -24 * scale.max()
    assert np.allclose(a32, np.abs(det), rtol=2.0 ** -23, atol=0)
