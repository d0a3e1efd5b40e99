"""Host-side checks of libfe that need no GPU: exports, reference tables, the
weak-form compiler and argument validation."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2107_04121_gb300 import fe

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "fe.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+char\s*\*|fe_status|int)\s*(fe_\w+)\s*\(", src, flags=re.M)))


def test_every_declared_symbol_is_exported(libfe):
    names = _declared_functions()
    assert len(names) >= 17
    for n in names:
        assert hasattr(libfe, n), n
    assert set(names) == set(fe.EXPORTED)


def test_status_strings(libfe):
    for code in range(9):
        assert libfe.fe_status_str(code).decode().startswith("FE_")
    assert libfe.fe_version() >= 100


@pytest.mark.parametrize("p,nq", [(1, 2), (2, 3), (3, 4), (2, 2), (3, 3), (4, 5)])
def test_refbasis_matches_oracle_tables(libfe, p, nq):
    pts, w, phi, dphi = fe.refbasis_hex(p, nq)
    opts, ow = oracle.hex_quadrature(nq)
    ophi, odphi = oracle.hex_basis(p, opts)
    np.testing.assert_allclose(pts, opts, atol=1e-15)
    np.testing.assert_allclose(w, ow, rtol=1e-14, atol=1e-16)
    np.testing.assert_allclose(phi, ophi, atol=1e-13)
    np.testing.assert_allclose(dphi, odphi, atol=1e-12)


@pytest.mark.parametrize("p,nq", [(1, 2), (2, 3), (3, 4), (2, 5)])
def test_refbasis_1d_factors_reproduce_3d_tables(libfe, p, nq):
    pts, w, phi, dphi = fe.refbasis_hex(p, nq)
    b, d = fe.refbasis_hex_1d(p, nq)
    n1 = p + 1
    want_phi = np.einsum("zk,yj,xi->zyxkji", b, b, b).reshape(nq ** 3, n1 ** 3)
    np.testing.assert_allclose(phi, want_phi, atol=1e-14)
    want_dx = np.einsum("zk,yj,xi->zyxkji", b, b, d).reshape(nq ** 3, n1 ** 3)
    np.testing.assert_allclose(dphi[:, 0, :], want_dx, atol=1e-13)


@pytest.mark.parametrize("n", range(1, 11))
def test_library_gauss_rule_matches_leggauss(libfe, n):
    pts, w, _, _ = fe.refbasis_hex(1, n)
    x, wr = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(pts[:n, 0], 0.5 * (x + 1), atol=1e-15)
    np.testing.assert_allclose(w.reshape(n, n, n)[0, 0, :] / w[0], wr / wr[0], rtol=1e-13)


def test_refbasis_rejects_unsupported(libfe):
    dp = ctypes.POINTER(ctypes.c_double)
    assert libfe.fe_refbasis_hex(0, 2, None, None, None, None) == fe.FE_ERR_SHAPE
    assert libfe.fe_refbasis_hex(5, 2, None, None, None, None) == fe.FE_ERR_SHAPE
    assert libfe.fe_refbasis_hex(2, 11, None, None, None, None) == fe.FE_ERR_SHAPE


V, S, M, PA = fe.VIRTUAL, fe.STATE, fe.MATERIAL, fe.PARAMETER
NONE, SC, LAME, D66 = fe.MAT_NONE, fe.MAT_SCALAR, fe.MAT_LAME, fe.MAT_D66


@pytest.mark.parametrize("expr,ops,shape", [
    ("0.i,0.i", [(V, 1, NONE), (S, 1, NONE)], 8),
    ("0.j, 0.j", [(V, 1, NONE), (S, 1, NONE)], 8),
    ("0,0.i,0.i", [(M, 1, SC), (V, 1, NONE), (S, 1, NONE)], 8),
    ("i,i", [(V, 3, NONE), (S, 3, NONE)], 24),
    ("i,i", [(V, 1, NONE), (S, 1, NONE)], 8),
    ("0,0", [(V, 1, NONE), (S, 1, NONE)], 8),
    ("0,i,i", [(M, 1, SC), (V, 3, NONE), (S, 3, NONE)], 24),
    ("IK,s(i:j)->I,s(k:l)->K", [(M, 1, LAME), (V, 3, NONE), (S, 3, NONE)], 24),
    ("IK,s(i:j)->I,s(k:l)->K", [(M, 1, D66), (V, 3, NONE), (S, 3, NONE)], 24),
    ("AB,s(p:q)->A,s(r:t)->B", [(M, 1, D66), (V, 3, NONE), (S, 3, NONE)], 24),
    ("KI,s(i:j)->I,s(k:l)->K", [(M, 1, D66), (V, 3, NONE), (S, 3, NONE)], 24),
    ("s(k:l)->K,IK,s(i:j)->I", [(S, 3, NONE), (M, 1, LAME), (V, 3, NONE)], 24),
    ("i,i.j,j", [(V, 3, NONE), (S, 3, NONE), (S, 3, NONE)], 24),
    ("i,i.j,j", [(V, 3, NONE), (S, 3, NONE), (PA, 3, NONE)], 24),
    ("i,i.j,j", [(V, 3, NONE), (PA, 3, NONE), (S, 3, NONE)], 24),
    ("a,b,a.b", [(V, 3, NONE), (S, 3, NONE), (S, 3, NONE)], 24),
    ("ij,i,j", [(M, 1, fe.MAT_M33), (V, 3, NONE), (S, 3, NONE)], 24),
    ("ji,i,j", [(M, 1, fe.MAT_M33), (V, 3, NONE), (S, 3, NONE)], 24),
])
def test_form_compile_accepts_tab_ewfd_forms(libfe, expr, ops, shape):
    f = fe.form_compile(expr, ops)
    assert f.shape(8) == (shape, shape)


@pytest.mark.parametrize("expr,ops,shape", [
    ("i.i,0", [(V, 3, NONE), (S, 1, NONE)], (24, 8)),          # Stokes coupling (v, p)
    ("i.i,0", [(S, 3, NONE), (V, 1, NONE)], (8, 24)),          # transposed coupling (u, q)
    ("0,i.i", [(V, 1, NONE), (S, 3, NONE)], (8, 24)),
    ("i.i", [(V, 3, NONE)], (24, 0)),                          # divergence: residual only
    # eval forms: no test function
    ("0.i,0.i", [(PA, 1, NONE), (PA, 1, NONE)], (1, 0)),
    ("i,i", [(S, 3, NONE), (PA, 3, NONE)], (1, 0)),
    ("IK,s(i:j)->I,s(k:l)->K", [(M, 1, LAME), (PA, 3, NONE), (PA, 3, NONE)], (1, 0)),
    ("IK,s(k:l)->K", [(M, 1, D66), (PA, 3, NONE)], (6, 0)),    # Cauchy stress
    ("i.i", [(PA, 3, NONE)], (1, 0)),
    ("i,i.j,j", [(PA, 3, NONE), (PA, 3, NONE), (PA, 3, NONE)], (1, 0)),
])
def test_form_compile_accepts_mixed_and_eval_forms(libfe, expr, ops, shape):
    f = fe.form_compile(expr, ops)
    assert f.shape(8) == shape
@pytest.mark.parametrize("expr,ops,code", [
    # valid notation, no kernel
    ("i,i.j,j", [(V, 3, NONE), (PA, 3, NONE), (PA, 3, NONE)], fe.FE_ERR_UNSUPPORTED_SPEC),  # no unknown
    ("i,i.j,i", [(V, 3, NONE), (S, 3, NONE), (S, 3, NONE)], fe.FE_ERR_UNSUPPORTED_SPEC),
    ("j,i.j,i", [(V, 3, NONE), (S, 3, NONE), (S, 3, NONE)], fe.FE_ERR_UNSUPPORTED_SPEC),
    ("i,i.i,i", [(V, 3, NONE), (S, 3, NONE), (S, 3, NONE)], fe.FE_ERR_UNSUPPORTED_SPEC),
    ("i,i,i", [(V, 3, NONE), (S, 3, NONE), (PA, 3, NONE)], fe.FE_ERR_UNSUPPORTED_SPEC),
    ("ij,i,j", [(M, 1, D66), (V, 3, NONE), (S, 3, NONE)], fe.FE_ERR_UNSUPPORTED_SPEC),  # needs M33
    ("ij,i,j", [(M, 1, fe.MAT_M33), (V, 3, NONE), (PA, 3, NONE)], fe.FE_ERR_UNSUPPORTED_SPEC),  # no unknown
    ("i.j,0", [(V, 3, NONE), (S, 1, NONE)], fe.FE_ERR_UNSUPPORTED_SPEC),
    ("i.i", [(V, 1, NONE)], fe.FE_ERR_UNSUPPORTED_SPEC),
    ("IK,s(k:l)->K", [(M, 1, D66), (V, 3, NONE)], fe.FE_ERR_UNSUPPORTED_SPEC),  # Cauchy stress: eval only
    ("0.i,0.j", [(V, 1, NONE), (S, 1, NONE)], fe.FE_ERR_UNSUPPORTED_SPEC),
    ("IK,s(i:j)->I,s(i:j)->K", [(M, 1, LAME), (V, 3, NONE), (S, 3, NONE)], fe.FE_ERR_UNSUPPORTED_SPEC),
    # malformed
    ("0.i,0.", [(V, 1, NONE), (S, 1, NONE)], fe.FE_ERR_INVALID_ARG),
    ("0.i", [(V, 1, NONE), (S, 1, NONE)], fe.FE_ERR_INVALID_ARG),
    ("s(i:j->I,s(k:l)->K", [(V, 3, NONE), (S, 3, NONE)], fe.FE_ERR_INVALID_ARG),
    ("0.i,0.i", [(V, 3, NONE), (S, 3, NONE)], fe.FE_ERR_INVALID_ARG),  # scalar symbol on a vector field
    ("i,i", [(V, 2, NONE), (S, 2, NONE)], fe.FE_ERR_INVALID_ARG),
    ("i,i.j,0", [(V, 3, NONE), (S, 3, NONE), (S, 3, NONE)], fe.FE_ERR_INVALID_ARG),  # scalar symbol, vector field
    ("0.i,0.i", [(V, 1, LAME), (S, 1, NONE)], fe.FE_ERR_INVALID_ARG),
])
def test_form_compile_rejects(libfe, expr, ops, code):
    with pytest.raises(fe.FEError) as ei:
        fe.form_compile(expr, ops)
    assert ei.value.status == code


def test_null_arguments_are_rejected(libfe):
    h = ctypes.c_void_p()
    assert libfe.fe_create(0, None) == fe.FE_ERR_INVALID_ARG
    assert libfe.fe_form_compile(None, None, None, 0, ctypes.byref(h)) == fe.FE_ERR_INVALID_ARG
    assert libfe.fe_eval_matrix(None, None, None, None, 0, 0, None, None) == fe.FE_ERR_INVALID_ARG
    assert libfe.fe_eval_residual(None, None, None, None, 0, None, None) == fe.FE_ERR_INVALID_ARG
    assert libfe.fe_assemble_vector(None, None, 1, None, 0, None, 0, None) == fe.FE_ERR_INVALID_ARG
    assert libfe.fe_geometry(None, None, None, None, 0, ctypes.byref(h), None) == fe.FE_ERR_INVALID_ARG
    assert libfe.fe_destroy(None) == fe.FE_ERR_INVALID_ARG
    assert libfe.fe_geometry_free(None) == fe.FE_ERR_INVALID_ARG
    assert libfe.fe_assembly_free(None) == fe.FE_ERR_INVALID_ARG
    # every entry point rejects a NULL context or handle before touching the device
    v = ctypes.c_int()
    assert libfe.fe_geometry_view(None, None, 0, 0, ctypes.byref(h)) == fe.FE_ERR_INVALID_ARG
    assert libfe.fe_geometry_update(None, None, None) == fe.FE_ERR_INVALID_ARG
    assert libfe.fe_geometry_get(None, None, 0, 0, None, None) == fe.FE_ERR_INVALID_ARG
    assert libfe.fe_assembly_create(None, None, ctypes.byref(h), None) == fe.FE_ERR_INVALID_ARG
    assert libfe.fe_assemble_vector_noalloc(None, None, 3, None, 0, None, 0, None) == fe.FE_ERR_INVALID_ARG
    assert libfe.fe_batch_create(None, None, 0, 0, ctypes.byref(h), None) == fe.FE_ERR_INVALID_ARG
    assert libfe.fe_batch_run(None, None, None) == fe.FE_ERR_INVALID_ARG
    assert libfe.fe_batch_describe(None, 0, None, None, None) == fe.FE_ERR_INVALID_ARG
    assert libfe.fe_batch_schedule(None, ctypes.byref(v)) == fe.FE_ERR_INVALID_ARG
    assert libfe.fe_batch_free(None) == fe.FE_ERR_INVALID_ARG
    assert libfe.fe_round_f32(None, None, None, 0, None) == fe.FE_ERR_INVALID_ARG
    assert libfe.fe_debug_hold_next_matrix(None) == fe.FE_ERR_INVALID_ARG


def test_header_flag_values_match_the_binding():
    """Every flag the header defines (#define FE_<NAME> <value>u) that the Python
    binding also names (<NAME>) has the same value there, so that the binding passes
    what the library reads."""
    import re

    from paper_2107_04121_gb300 import fe
    text = open(HEADER).read()
    defs = dict(re.findall(r"#define\s+FE_(\w+)\s+(\d+)u?\b", text))
    shared = {k: int(v) for k, v in defs.items() if hasattr(fe, k)}
    for name in ("BATCH_GEOMETRY", "BATCH_AUTOTUNE", "BATCH_GRAPH", "BATCH_PERSISTENT", "BATCH_LAUNCHES",
                 "BATCH_SHARED_GRAM", "GEOM_STORE_F64", "GEOM_STORE_F32", "GEOM_DEFERRED"):
        assert name in shared, name
    for name, value in shared.items():
        assert getattr(fe, name) == value, (name, getattr(fe, name), value)
