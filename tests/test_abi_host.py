"""CPU tests of the C ABI library: it loads, exports every declared symbol,
and its host-side logic (quadrature helper, dof map, CSR pattern) matches the
oracle bit for bit.  No GPU call is made here."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2410_12614_gb300 import _lib, api, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2410_12614_gb300 import build
    build.build()
    oracle.build()


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^\s*(?:fe_status|const char \*)\s*(fe_\w+)\s*\(", src, re.M))
    return names


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert names == set(_lib.SIGNATURES), names ^ set(_lib.SIGNATURES)


def test_last_error_reports_invalid_arguments():
    lib = _lib.load()
    nq = ctypes.c_int32()
    st = lib.fe_quadrature_rule(7, 0, 3, ctypes.byref(nq), None, None)
    assert st == -1 and b"cell type" in lib.fe_last_error()
    st = lib.fe_quadrature_rule(3, 0, 99, ctypes.byref(nq), None, None)
    assert st == -2


@pytest.mark.parametrize("cell", ["triangle", "tetrahedron"])
@pytest.mark.parametrize("m", [1, 2, 3, 4, 7, 9, 12])
def test_quadrature_helper_matches_oracle(cell, m):
    p1, w1 = api.quadrature_rule(cell, m)
    p2, w2 = oracle.collapsed_rule(cell, m)
    np.testing.assert_allclose(p1, p2, rtol=4e-15, atol=1e-16)
    np.testing.assert_allclose(w1, w2, rtol=4e-14, atol=0)


def test_three_point_rule():
    p, w = api.quadrature_rule("triangle", 0, family=_lib.FE_QUAD_TRIANGLE_3POINT)
    p2, w2 = oracle.strang_fix_3()
    np.testing.assert_array_equal(p, p2)
    np.testing.assert_array_equal(w, w2)


@pytest.mark.parametrize("cell,n,p", [("triangle", 4, 1), ("triangle", 3, 4), ("triangle", 2, 10),
                                      ("tetrahedron", 3, 1), ("tetrahedron", 2, 3), ("tetrahedron", 2, 5),
                                      ("tetrahedron", 1, 8)])
def test_pattern_bit_exact_vs_oracle(cell, n, p):
    v, c = inputs.structured_mesh(cell, n, 0.1, 1)
    pat = api.Pattern(cell, v.shape[0], c, p)
    dofs, rp, ci = pat.arrays()
    pr = oracle.Problem(v, c, p, *oracle.rule_for_degree(cell, min(p, 2)))
    odofs, nd = pr.cell_dofs()
    orp, oci = pr.csr_pattern()
    assert pat.n_dofs == nd
    assert np.array_equal(dofs, odofs)
    assert np.array_equal(rp, orp)
    assert np.array_equal(ci, oci)
    assert pat.max_row == int(np.diff(orp).max())


def test_pattern_rejects_bad_connectivity():
    v, c = inputs.cube_mesh(1)
    bad = c.copy()
    bad[0, 0] = 10 ** 6
    with pytest.raises(_lib.FeError) as e:
        api.Pattern("tetrahedron", v.shape[0], bad, 2)
    assert e.value.status == -1
    with pytest.raises(_lib.FeError) as e:
        api.Pattern("tetrahedron", v.shape[0], c, 9)
    assert e.value.status == -2


@pytest.mark.parametrize("cell", ["quadrilateral", "hexahedron"])
@pytest.mark.parametrize("m", [1, 2, 4, 7])
def test_tensor_rule_helper_matches_oracle(cell, m):
    p1, w1 = api.quadrature_rule(cell, m)
    p2, w2 = oracle.tensor_rule(cell, m)
    np.testing.assert_allclose(p1, p2, rtol=4e-15, atol=1e-16)
    np.testing.assert_allclose(w1, w2, rtol=4e-14, atol=0)


@pytest.mark.parametrize("cell,n,p", [("quadrilateral", 4, 1), ("quadrilateral", 3, 3), ("quadrilateral", 2, 8),
                                      ("hexahedron", 3, 1), ("hexahedron", 2, 2), ("hexahedron", 2, 4),
                                      ("hexahedron", 1, 5)])
def test_box_pattern_bit_exact_vs_oracle(cell, n, p):
    # the library numbers boxed-cell dofs entity by entity; the oracle sorts
    # the nodes' Q1-weight keys: the two must agree bit for bit
    v, c = inputs.structured_mesh(cell, n, 0.1, 2)
    pat = api.Pattern(cell, v.shape[0], c, p)
    dofs, rp, ci = pat.arrays()
    pr = oracle.Problem(v, c, p, *oracle.rule_for_degree(cell, 1))
    odofs, nd = pr.cell_dofs()
    orp, oci = pr.csr_pattern()
    assert pat.n_dofs == nd == (p * n + 1) ** pr.d
    assert np.array_equal(dofs, odofs)
    assert np.array_equal(rp, orp)
    assert np.array_equal(ci, oci)


def test_box_pattern_on_a_permuted_mesh():
    # renumbered vertices and cells with every cell's corners in tensor order
    # but the mesh numbering scrambled: entity orientations now differ between
    # neighbours, and the numbering must still agree with the oracle's keys
    v, c = inputs.hex_mesh(3, 0.1, 3)
    rng = np.random.default_rng(4)
    perm = rng.permutation(len(v))
    inv = np.argsort(perm)
    v2 = v[perm]
    c2 = inv[c][rng.permutation(len(c))].astype(np.int32)
    for p in (2, 3):
        pat = api.Pattern("hexahedron", v2.shape[0], c2, p)
        dofs, rp, ci = pat.arrays()
        pr = oracle.Problem(v2, c2, p, *oracle.rule_for_degree("hexahedron", 1))
        odofs, nd = pr.cell_dofs()
        assert np.array_equal(dofs, odofs)
        assert np.array_equal(rp, pr.csr_pattern()[0]) and np.array_equal(ci, pr.csr_pattern()[1])
