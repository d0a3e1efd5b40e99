"""GPU parity: libfe (through the C ABI) against the FP64 oracle, element by
element, on seeded meshes that span several CTA tiles and a ragged tail."""
import time

import numpy as np
import pytest

import oracle
from paper_2107_04121_gb300 import fe, meshgen
from tests.parity import TOL, Problem, rel_matrix_error, rel_vector_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(libfe):
    c = fe.Context(0)
    yield c
    c.close()


def _t(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)


# ---- geometry ------------------------------------------------------------------

# (p, nq): n1 == nq takes the collocation kernel (x at the points, then the
# derivative on the points), n1 != nq the three-stage sum factorisation
@pytest.mark.parametrize("p,nq,n", [(1, 2, (5, 4, 3)), (2, 3, (4, 3, 3)), (3, 4, (2, 2, 3)),
                                    (1, 3, (4, 3, 3)), (2, 4, (3, 3, 2))])
def test_geometry_matches_oracle(ctx, p, nq, n):
    mesh = meshgen.structured_hex(*n, p, 0.15, 21)
    P = Problem(ctx, mesh, p, nq)
    wdetJ, G, Jinv = oracle.geometry(mesh.coords, mesh.conn, P.ref, want_Jinv=True)
    g_w = P.geom.get(fe.GEOM_WDETJ, "f64").cpu().numpy()
    g_J = P.geom.get(fe.GEOM_JINV, "f64").cpu().numpy()
    g_G = P.geom.get(fe.GEOM_G, "f64").cpu().numpy()
    ctx.check()
    assert np.abs(g_w - wdetJ).max() <= 1e-14 * np.abs(wdetJ).max()
    assert np.abs(g_J - Jinv).max() <= 1e-13 * np.abs(Jinv).max()
    assert np.abs(g_G - G).max() <= 1e-12 * np.abs(G).max()
    # float32 copies are the float64 values rounded once
    np.testing.assert_array_equal(P.geom.get(fe.GEOM_WDETJ, "f32").cpu().numpy(), g_w.astype(np.float32))
    np.testing.assert_array_equal(P.geom.get(fe.GEOM_JINV, "f32").cpu().numpy(), g_J.astype(np.float32))


@pytest.mark.parametrize("p,nq", [(1, 2), (2, 3), (3, 4), (2, 4)])
def test_direct_and_sum_factorised_geometry_agree(ctx, p, nq):
    """The generic kernel (tables only) and the tensor-product kernels compute the same map."""
    mesh = meshgen.structured_hex(3, 2, 3, p, 0.15, 24)
    P = Problem(ctx, mesh, p, nq)  # tensor-product path
    pts, w, phi, dphi = fe.refbasis_hex(p, nq)
    g_direct = fe.geometry(ctx, P.m, phi, dphi, w)
    wdetJ, G, Jinv = oracle.geometry(mesh.coords, mesh.conn, P.ref, want_Jinv=True)
    for g in (P.geom, g_direct):
        assert np.abs(g.get(fe.GEOM_JINV, "f64").cpu().numpy() - Jinv).max() <= 1e-13 * np.abs(Jinv).max()
        assert np.abs(g.get(fe.GEOM_WDETJ, "f64").cpu().numpy() - wdetJ).max() <= 1e-14 * np.abs(wdetJ).max()
    ctx.check()


def test_float32_rounding_of_the_geometry_matches_ieee(ctx):
    """The integer float64 -> float32 rounding of the geometry kernels gives the
    IEEE nearest-even result (numpy's conversion) bit for bit: ties either way,
    carries into the exponent, the ends of the normal range, and the values that
    take the hardware path (zero, subnormal results, overflow, inf, NaN)."""
    rng = np.random.default_rng(98)
    one_ulp32 = 2.0 ** -23
    edge = [0.0, -0.0, 1.0, -1.0, 1.5, 1.0 + one_ulp32 / 2, 1.0 + 3 * one_ulp32 / 2, 1.0 + one_ulp32 / 2 + 2.0 ** -40,
            1.0 + one_ulp32 / 2 - 2.0 ** -40, 2.0 - 2.0 ** -30, np.nextafter(2.0, 0.0),
            float(np.finfo(np.float32).tiny), float(np.finfo(np.float32).tiny) * (1 - 2.0 ** -30),
            float(np.finfo(np.float32).tiny) / 3, 1e-40, 1e-46, 2.0 ** -149, 2.0 ** -150, 3 * 2.0 ** -151,
            float(np.finfo(np.float32).max), float(np.finfo(np.float32).max) * (1 + 2.0 ** -25),
            float(np.finfo(np.float32).max) * (1 + 2.0 ** -23), 1e39, -1e39, 1e300, -1e-300, np.inf, -np.inf]
    rand = [rng.standard_normal(20000) * 10.0 ** rng.uniform(-40, 40, 20000),
            # float32 values plus exactly half their spacing: ties, to the even neighbour
            (lambda f: f.astype(np.float64) + np.spacing(f).astype(np.float64) / 2)(
                (rng.standard_normal(5000) * 10.0 ** rng.uniform(-30, 30, 5000)).astype(np.float32)),
            rng.uniform(-1, 1, 20000)]
    x = np.concatenate([np.array(edge)] + rand)
    with np.errstate(over="ignore"):
        want = x.astype(np.float32)
    got = fe.round_f32(ctx, _t(x, torch.float64)).cpu().numpy()
    ctx.check()
    np.testing.assert_array_equal(got.view(np.uint32), want.view(np.uint32))
    nan = fe.round_f32(ctx, _t(np.array([np.nan, -np.nan]), torch.float64)).cpu().numpy()
    assert np.all(np.isnan(nan))


def test_meshes_past_the_32_bit_index_range_are_rejected(ctx):
    """Node indices and the (element, local node) incidences of the assembly lists
    are 32-bit: a mesh whose node count or n_elems * N exceeds 2^31 - 1 is rejected
    on the host before any launch (here the descriptor overstates its sizes, and
    nothing past the real arrays is read); the same descriptor with its true
    sizes is accepted."""
    mesh = meshgen.structured_hex(1, 1, 1, 2, 0.0, 0)
    m = fe.Mesh(torch.from_numpy(mesh.coords).cuda(), torch.from_numpy(mesh.conn).cuda())
    for field, value in (("n_elems", (2 ** 31 - 1) // 27 + 1), ("n_nodes", 2 ** 31)):
        saved = getattr(m.struct, field)
        setattr(m.struct, field, value)
        for call in (lambda: fe.assembly_create(ctx, m), lambda: fe.hex_geometry(ctx, m, 2, 3)):
            with pytest.raises(fe.FEError) as ei:
                call()
            assert ei.value.status == fe.FE_ERR_INVALID_ARG
        setattr(m.struct, field, saved)
    fe.hex_geometry(ctx, m, 2, 3)
    fe.assembly_create(ctx, m)
    ctx.check()


def test_inconsistent_tensor_factors_are_rejected(ctx):
    mesh = meshgen.structured_hex(2, 2, 2, 2, 0.0, 0)
    P = Problem(ctx, mesh, 2, 3)
    pts, w, phi, dphi = fe.refbasis_hex(2, 3)
    b1d, d1d = fe.refbasis_hex_1d(2, 3)
    d1d = d1d.copy()
    d1d[1, 2] += 1e-6
    with pytest.raises(fe.FEError) as ei:
        fe.geometry(ctx, P.m, phi, dphi, w, b1d=b1d, d1d=d1d)
    assert ei.value.status == fe.FE_ERR_INVALID_ARG
    assert "1-D factors" in str(ei.value)
    # the next failing call reports its own problem, not this message
    asm = fe.assembly_create(ctx, P.m)
    r = torch.zeros((mesh.n_elems, 2 * 27), dtype=torch.float64, device="cuda")
    with pytest.raises(fe.FEError) as ei:
        fe.assemble_vector(ctx, asm, 2, r, "f64")
    assert ei.value.status == fe.FE_ERR_INVALID_ARG
    assert "1-D factors" not in str(ei.value)


def test_geometry_update_follows_moved_nodes(ctx):
    mesh = meshgen.structured_hex(3, 3, 3, 2, 0.1, 22)
    P = Problem(ctx, mesh, 2, 3)
    rng = np.random.default_rng(23)
    new = mesh.coords * np.array([1.5, 0.8, 1.1]) + 0.01 * rng.standard_normal(mesh.coords.shape)
    P.coords_d.copy_(torch.from_numpy(new))
    P.geom.update()
    wdetJ, G, _ = oracle.geometry(new, mesh.conn, P.ref)
    ctx.check()
    g_G = P.geom.get(fe.GEOM_G, "f64").cpu().numpy()
    assert np.abs(P.geom.get(fe.GEOM_WDETJ, "f64").cpu().numpy() - wdetJ).max() <= 1e-14 * np.abs(wdetJ).max()
    assert np.abs(g_G - G).max() <= 1e-12 * np.abs(G).max()


def test_nonpositive_detj_is_reported(ctx):
    mesh = meshgen.structured_hex(3, 3, 2, 1, 0.0, 0)
    mesh.conn[7, [0, 1]] = mesh.conn[7, [1, 0]]  # mirrored element
    mesh.conn[12, [2, 3]] = mesh.conn[12, [3, 2]]
    P = Problem(ctx, mesh, 1, 2)
    st, bad = ctx.status()
    assert st == fe.FE_ERR_NONPOSITIVE_DETJ and bad == 7
    assert ctx.status() == (fe.FE_OK, -1)  # cleared


@pytest.mark.parametrize("path", ["geometry", "residual", "matrix"])
def test_degenerate_and_nonfinite_geometry_are_reported(ctx, path):
    """det J = 0 exactly (an element collapsed to a point) and a NaN coordinate, from
    the geometry kernel and from the residual and tensor-core matrix kernels that
    compute a stale geometry."""
    mesh = meshgen.structured_hex(1, 1, 1, 2, 0.0, 0)
    lm = _t(np.ones((1, 2)), torch.float64)
    u = _t(np.zeros(3 * mesh.n_nodes), torch.float32)
    for value, code in ((None, fe.FE_ERR_NONPOSITIVE_DETJ), (np.nan, fe.FE_ERR_NONFINITE)):
        coords = mesh.coords.copy()
        if value is None:
            coords[:] = coords[0]
        else:
            coords[13, 1] = value
        m = fe.Mesh(_t(coords, torch.float64), _t(mesh.conn, torch.int32))
        ctx.status()
        if path == "geometry":
            fe.hex_geometry(ctx, m, 2, 3, flags=fe.GEOM_STORE_F32)
        elif path == "residual":
            lazy = fe.hex_geometry(ctx, m, 2, 3, flags=fe.GEOM_STORE_F32 | fe.GEOM_DEFERRED)
            fe.eval_residual(ctx, fe.elasticity_form(), lazy, [lm, None, u], "f32")
        else:
            lazy = fe.hex_geometry(ctx, m, 2, 3, flags=fe.GEOM_STORE_F32 | fe.GEOM_DEFERRED)
            fe.eval_matrix(ctx, fe.elasticity_form(), lazy, [lm, None, None], "bf16x3")
        assert ctx.status() == (code, 0)


# ---- matrix and residual modes ----------------------------------------------------

def _case(ctx, kind, p, n, seed, material=fe.MAT_LAME):
    mesh = meshgen.structured_hex(*n, p, 0.15, seed)
    lam, mu = meshgen.lame_materials(mesh)
    P = Problem(ctx, mesh, p, p + 1)
    wdetJ, G, _ = P.oracle_geometry()
    rng = np.random.default_rng(seed + 100)
    E = mesh.n_elems
    if kind == "laplace":
        coef = rng.uniform(0.5, 2.0, E)
        form = fe.laplace_form(weighted=True)
        mat = coef
        K = oracle.matrix_laplace(wdetJ, G, coef)
        u = rng.standard_normal(mesh.n_nodes)
        r = oracle.residual_laplace(mesh.conn, wdetJ, G, u, coef)
        ncomp = 1
    elif kind in ("mass1", "mass3"):
        ncomp = 1 if kind == "mass1" else 3
        coef = rng.uniform(0.5, 2.0, E)
        form = fe.mass_form(ncomp, weighted=True)
        mat = coef
        K = oracle.matrix_mass(wdetJ, P.ref.phi, ncomp, coef)
        u = rng.standard_normal(mesh.n_nodes * ncomp)
        r = oracle.residual_mass(mesh.conn, wdetJ, P.ref.phi, u, ncomp, coef)
    else:
        ncomp = 3
        form = fe.elasticity_form(material)
        if material == fe.MAT_LAME:
            mat = np.stack([lam, mu], 1)
            D = oracle.lame_to_D(lam, mu)
        else:  # general symmetric positive definite D per element
            A = rng.standard_normal((E, 6, 6))
            D = np.einsum("eij,ekj->eik", A, A) + 6 * np.eye(6)
            mat = D
        K = oracle.matrix_elasticity(wdetJ, G, D)
        u = rng.standard_normal(mesh.n_nodes * 3)
        r = oracle.residual_elasticity(mesh.conn, wdetJ, G, D, u)
    return P, form, mat, u, K, r, ncomp


CASES = [
    ("laplace", 1, (5, 4, 3)), ("laplace", 2, (4, 3, 3)), ("laplace", 3, (2, 2, 3)),
    ("mass1", 1, (5, 4, 3)), ("mass3", 2, (4, 3, 3)), ("mass1", 3, (2, 2, 3)),
    ("elasticity", 1, (5, 4, 3)), ("elasticity", 2, (4, 4, 4)), ("elasticity", 3, (2, 2, 3)),
]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("kind,p,n", CASES)
def test_matrix_and_residual_match_oracle(ctx, kind, p, n, prec):
    P, form, mat, u, Kref, rref, ncomp = _case(ctx, kind, p, n, 31 + p)
    dt = torch.float64 if prec == "f64" else torch.float32
    args = [None] * len(form.operands)
    args[form.state_op] = _t(u, dt)
    args[0] = _t(mat, torch.float64)  # the material is operand 0 in the named forms
    K = fe.eval_matrix(ctx, form, P.geom, args, prec)
    r = fe.eval_residual(ctx, form, P.geom, args, prec)
    ctx.check()
    ek = rel_matrix_error(K.cpu().numpy(), Kref)
    er = rel_vector_error(r.cpu().numpy(), rref)
    assert ek <= TOL[prec], ek
    assert er <= TOL[prec], er


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_elasticity_general_D_and_transposed_spec(ctx, prec):
    P, form, D, u, Kref, rref, _ = _case(ctx, "elasticity", 2, (3, 3, 2), 41, fe.MAT_D66)
    dt = torch.float64 if prec == "f64" else torch.float32
    K = fe.eval_matrix(ctx, form, P.geom, [_t(D, torch.float64), None, None], prec)
    r = fe.eval_residual(ctx, form, P.geom, [_t(D, torch.float64), None, _t(u, dt)], prec)
    assert rel_matrix_error(K.cpu().numpy(), Kref) <= TOL[prec]
    assert rel_vector_error(r.cpu().numpy(), rref) <= TOL[prec]
    # 'KI,...' names the material indices as (u, v): the kernel must use D^T
    ft = fe.form_compile("KI,s(i:j)->I,s(k:l)->K", [(fe.MATERIAL, 1, fe.MAT_D66), (fe.VIRTUAL, 3, 0),
                                                      (fe.STATE, 3, 0)])
    Dt = np.ascontiguousarray(D.transpose(0, 2, 1))
    Kt = fe.eval_matrix(ctx, ft, P.geom, [_t(Dt, torch.float64), None, None], prec)
    assert rel_matrix_error(Kt.cpu().numpy(), Kref) <= TOL[prec]


# raw BF16 (8-bit significands, no split) is below the 1e-5 bar by design: its
# error is a stated figure (2.4e-3 measured at the 48^3 workload), gated at 5e-3
TC_TOL = [("tf32x3", TOL["tf32x3"]), ("bf16x3", TOL["bf16x3"]), ("bf16", 5e-3)]


@pytest.mark.parametrize("prec,tol", TC_TOL)
def test_tensor_core_elasticity_matches_oracle(ctx, prec, tol):
    """tcgen05 split-precision paths (Q2, Lame): TF32x3 and BF16x3 within the 1e-5
    bar on every element; raw BF16 against its stated figure."""
    P, form, mat, u, Kref, rref, _ = _case(ctx, "elasticity", 2, (4, 4, 5), 81)
    args = [_t(mat, torch.float64), None, None]
    K = fe.eval_matrix(ctx, form, P.geom, args, prec)
    K32 = fe.eval_matrix(ctx, form, P.geom, args, "f32")
    ctx.check()
    err = rel_matrix_error(K.cpu().numpy(), Kref)
    assert err <= tol, err
    assert rel_matrix_error(K32.cpu().numpy(), Kref) <= TOL["f32"]
    # symmetric like the exact matrix
    Kh = K.cpu().numpy()
    assert np.abs(Kh - Kh.transpose(0, 2, 1)).max() <= 10 * tol * np.abs(Kh).max()


@pytest.mark.parametrize("prec,tol", TC_TOL)
def test_tensor_core_pipeline_many_elements_per_cta(ctx, prec, tol):
    """2,352 elements: every persistent CTA of the tensor-core kernel runs 5 or 6
    elements through its two operand buffers and its accumulator (buffer reuse,
    accumulator hand-back, ragged split over the CTAs).  Every element against the
    oracle, in the benchmark's step: deferred geometry computed by the residual
    kernel, then K_e."""
    P, form, mat, u, Kref, rref, _ = _case(ctx, "elasticity", 2, (14, 14, 12), 83)
    E = P.mesh.n_elems
    assert E == 2352 and E > 5 * 152 * 3
    geom = fe.hex_geometry(ctx, P.m, 2, 3, flags=fe.GEOM_STORE_F32 | fe.GEOM_DEFERRED)
    args = [_t(mat, torch.float64), None, _t(u, torch.float32)]
    geom.update()
    r = fe.eval_residual(ctx, form, geom, args, prec)
    K = fe.eval_matrix(ctx, form, geom, args, prec)
    ctx.check()
    err = rel_matrix_error(K.cpu().numpy(), Kref)
    assert err <= tol, err
    assert rel_vector_error(r.cpu().numpy(), rref) <= TOL["f32"]


@pytest.mark.parametrize("prec,tol", TC_TOL)
def test_tensor_core_kernel_computes_stale_geometry(ctx, prec, tol):
    """fe_eval_matrix first on a stale float32-only deferred handle: the geometry
    warp of the tensor-core kernel computes the FP64 geometry (5,184 elements, 11-12
    per CTA, so that the ring of geometry slots wraps around).  The stored float32
    copy equals the geometry kernel's bit for bit, K_e equals the kernel on the
    eager geometry bit for bit and matches the oracle, and the residual that follows
    on the now computed handle equals the eager path's."""
    P, form, mat, u, Kref, rref, _ = _case(ctx, "elasticity", 2, (18, 18, 16), 87)
    E = P.mesh.n_elems
    assert E == 5184 and E > 11 * 152 * 3
    eager = fe.hex_geometry(ctx, P.m, 2, 3, flags=fe.GEOM_STORE_F32)
    lazy = fe.hex_geometry(ctx, P.m, 2, 3, flags=fe.GEOM_STORE_F32 | fe.GEOM_DEFERRED)
    args = [_t(mat, torch.float64), None, _t(u, torch.float32)]
    for _ in range(2):  # a second update re-marks the handle stale
        lazy.update()
        K_l = fe.eval_matrix(ctx, form, lazy, args, prec)
    r_l = fe.eval_residual(ctx, form, lazy, args, "f32")
    K_e = fe.eval_matrix(ctx, form, eager, args, prec)
    r_e = fe.eval_residual(ctx, form, eager, args, "f32")
    ctx.check()
    np.testing.assert_array_equal(lazy.get(fe.GEOM_WDETJ, "f32").cpu().numpy(),
                                  eager.get(fe.GEOM_WDETJ, "f32").cpu().numpy())
    np.testing.assert_array_equal(lazy.get(fe.GEOM_JINV, "f32").cpu().numpy(),
                                  eager.get(fe.GEOM_JINV, "f32").cpu().numpy())
    assert torch.equal(K_l, K_e)
    assert torch.equal(r_l, r_e)
    assert rel_matrix_error(K_l.cpu().numpy(), Kref) <= tol
    assert rel_vector_error(r_l.cpu().numpy(), rref) <= TOL["f32"]


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3", "bf16"])
def test_deferred_geometry_matches_eager(ctx, prec):
    """A deferred float32-only geometry is computed by the first call that reads it;
    its stored copy, K_e and the following residual equal the eager path's."""
    P, form, mat, u, Kref, rref, _ = _case(ctx, "elasticity", 2, (5, 4, 3), 91)
    eager = fe.hex_geometry(ctx, P.m, 2, 3, flags=fe.GEOM_STORE_F32)
    lazy = fe.hex_geometry(ctx, P.m, 2, 3, flags=fe.GEOM_STORE_F32 | fe.GEOM_DEFERRED)
    args = [_t(mat, torch.float64), None, _t(u, torch.float32)]
    for _ in range(2):  # a second update re-marks the handle stale
        lazy.update()
        K_l = fe.eval_matrix(ctx, form, lazy, args, prec)
        r_l = fe.eval_residual(ctx, form, lazy, args, "f32")
    K_e = fe.eval_matrix(ctx, form, eager, args, prec)
    r_e = fe.eval_residual(ctx, form, eager, args, "f32")
    ctx.check()
    # the deferred handle is settled by the same kernel: identical bits throughout
    np.testing.assert_array_equal(lazy.get(fe.GEOM_WDETJ, "f32").cpu().numpy(),
                                  eager.get(fe.GEOM_WDETJ, "f32").cpu().numpy())
    np.testing.assert_array_equal(lazy.get(fe.GEOM_JINV, "f32").cpu().numpy(),
                                  eager.get(fe.GEOM_JINV, "f32").cpu().numpy())
    assert torch.equal(K_l, K_e)
    assert torch.equal(r_l, r_e)
    assert rel_vector_error(r_l.cpu().numpy(), rref) <= TOL["f32"]


@pytest.mark.parametrize("kind,material", [("laplace", None), ("mass1", None), ("mass3", None),
                                           ("elasticity", fe.MAT_LAME), ("elasticity", fe.MAT_D66)])
@pytest.mark.parametrize("p,n", [(1, (5, 4, 3)), (2, (4, 3, 3)), (3, (2, 2, 3))])
def test_residual_computes_stale_geometry(ctx, kind, material, p, n):
    """fe_eval_residual on a stale float32-only deferred handle computes the FP64
    geometry in the residual kernel: r, the stored copy and the matrix that
    follows equal the eager path's bit for bit, and r matches the oracle."""
    P, form, mat, u, Kref, rref, _ = _case(ctx, kind, p, n, 95 + p, material or fe.MAT_LAME)
    eager = fe.hex_geometry(ctx, P.m, p, p + 1, flags=fe.GEOM_STORE_F32)
    lazy = fe.hex_geometry(ctx, P.m, p, p + 1, flags=fe.GEOM_STORE_F32 | fe.GEOM_DEFERRED)
    args = [None] * len(form.operands)
    args[form.state_op] = _t(u, torch.float32)
    args[0] = _t(mat, torch.float64)  # the material is operand 0 in the named forms
    r_e = fe.eval_residual(ctx, form, eager, args, "f32")
    for _ in range(2):
        lazy.update()
        r_l = fe.eval_residual(ctx, form, lazy, args, "f32")
    ctx.check()
    assert torch.equal(r_l, r_e)
    assert torch.equal(lazy.get(fe.GEOM_JINV, "f32"), eager.get(fe.GEOM_JINV, "f32"))
    assert torch.equal(lazy.get(fe.GEOM_WDETJ, "f32"), eager.get(fe.GEOM_WDETJ, "f32"))
    assert torch.equal(fe.eval_matrix(ctx, form, lazy, args, "f32"), fe.eval_matrix(ctx, form, eager, args, "f32"))
    assert rel_vector_error(r_l.cpu().numpy(), rref) <= TOL["f32"]


def test_residual_computes_stale_geometry_many_groups_per_cta(ctx):
    """60,800 Q2 elements: the residual kernel's grid is capped at four waves of
    resident CTAs (4 x 7 x 152 of 7 elements on GB300), so every CTA takes at
    least two groups of elements; the last group is ragged."""
    mesh = meshgen.structured_hex(40, 40, 38, 2, 0.15, 96)
    P = Problem(ctx, mesh, 2, 3)
    lam, mu = meshgen.lame_materials(mesh)
    lm = _t(np.stack([lam, mu], 1), torch.float64)
    u = _t(np.random.default_rng(97).standard_normal(3 * mesh.n_nodes), torch.float32)
    form = fe.elasticity_form()
    eager = fe.hex_geometry(ctx, P.m, 2, 3, flags=fe.GEOM_STORE_F32)
    lazy = fe.hex_geometry(ctx, P.m, 2, 3, flags=fe.GEOM_STORE_F32 | fe.GEOM_DEFERRED)
    r_l = fe.eval_residual(ctx, form, lazy, [lm, None, u], "f32")
    r_e = fe.eval_residual(ctx, form, eager, [lm, None, u], "f32")
    ctx.check()
    assert torch.equal(r_l, r_e)
    assert torch.equal(lazy.get(fe.GEOM_JINV, "f32"), eager.get(fe.GEOM_JINV, "f32"))
    assert torch.equal(lazy.get(fe.GEOM_WDETJ, "f32"), eager.get(fe.GEOM_WDETJ, "f32"))
    # the tensor-core precisions name the same float32 residual kernel
    lazy.update()
    r_b = fe.eval_residual(ctx, form, lazy, [lm, None, u], "bf16x3")
    K_b = fe.eval_matrix(ctx, form, lazy, [lm, None, None], "bf16x3")
    ctx.check()
    assert torch.equal(r_b, r_e)
    assert torch.equal(K_b, fe.eval_matrix(ctx, form, eager, [lm, None, None], "bf16x3"))


def test_residual_with_stale_geometry_reports_nonpositive_detj(ctx):
    mesh = meshgen.structured_hex(3, 2, 2, 2, 0.0, 0)
    mesh.conn[7] = mesh.conn[7].reshape(3, 3, 3)[:, ::-1, :].reshape(-1)  # mirror element 7 in y
    P = Problem(ctx, mesh, 2, 3)
    ctx.status()  # the eager geometry of Problem reported it already: clear
    lazy = fe.hex_geometry(ctx, P.m, 2, 3, flags=fe.GEOM_STORE_F32 | fe.GEOM_DEFERRED)
    lm = _t(np.ones((mesh.n_elems, 2)), torch.float64)
    u = _t(np.zeros(3 * mesh.n_nodes), torch.float32)
    fe.eval_residual(ctx, fe.elasticity_form(), lazy, [lm, None, u], "f32")
    assert ctx.status() == (fe.FE_ERR_NONPOSITIVE_DETJ, 7)


def test_deferred_geometry_settles_for_other_kernels(ctx):
    P, form, mat, u, Kref, rref, _ = _case(ctx, "elasticity", 2, (3, 3, 2), 92)
    lazy = fe.hex_geometry(ctx, P.m, 2, 3, flags=fe.GEOM_DEFERRED)  # both copies: no fusion
    args = [_t(mat, torch.float64), None, None]
    K = fe.eval_matrix(ctx, form, lazy, args, "f64")
    ctx.check()
    assert rel_matrix_error(K.cpu().numpy(), Kref) <= TOL["f64"]
    lazy32 = fe.hex_geometry(ctx, P.m, 2, 3, flags=fe.GEOM_STORE_F32 | fe.GEOM_DEFERRED)
    wd = lazy32.get(fe.GEOM_WDETJ, "f32")  # settles before copying out
    ctx.check()
    wref, _, _ = P.oracle_geometry()
    np.testing.assert_allclose(wd.cpu().numpy(), wref, rtol=1e-6)


def test_deferred_geometry_reports_nonpositive_detj(ctx):
    mesh = meshgen.structured_hex(3, 2, 2, 2, 0.0, 0)
    mesh.conn[5] = mesh.conn[5].reshape(3, 3, 3)[:, :, ::-1].reshape(-1)  # mirror element 5 in x
    P = Problem(ctx, mesh, 2, 3)
    ctx.status()  # the eager geometry of Problem reported it already: clear
    lazy = fe.hex_geometry(ctx, P.m, 2, 3, flags=fe.GEOM_STORE_F32 | fe.GEOM_DEFERRED)
    lm = _t(np.ones((mesh.n_elems, 2)), torch.float64)
    fe.eval_matrix(ctx, fe.elasticity_form(), lazy, [lm, None, None], "bf16x3")
    assert ctx.status() == (fe.FE_ERR_NONPOSITIVE_DETJ, 5)


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_tensor_core_wait_timeout_is_reported_and_the_context_recovers(ctx, prec):
    """A tensor-core launch whose consumers wait on a flag that nothing sets: the
    bounded wait runs out (about two seconds), every CTA drains its MMAs and leaves,
    FE_ERR_TIMEOUT is reported, and the next launch on the context is a normal one."""
    # 1,000 elements: two or three per CTA, so the producers also run into their
    # bounded waits and drain the MMAs already issued
    P, form, mat, u, Kref, rref, _ = _case(ctx, "elasticity", 2, (10, 10, 10), 97)
    args = [_t(mat, torch.float64), None, None]
    ctx.status()
    fe.debug_hold_next_matrix(ctx)
    t0 = time.time()
    fe.eval_matrix(ctx, form, P.geom, args, prec)
    st, bad = ctx.status()
    assert st == fe.FE_ERR_TIMEOUT and bad >= 0
    assert time.time() - t0 < 60
    K = fe.eval_matrix(ctx, form, P.geom, args, prec)
    ctx.check()
    assert rel_matrix_error(K.cpu().numpy(), Kref) <= TOL[prec]


def test_tensor_core_timeout_with_the_geometry_warp(ctx):
    """The same bounded wait in the kernel that computes a stale geometry: the
    consumers wait on a flag that nothing sets, the geometry warp and the producers
    give up too, FE_ERR_TIMEOUT is reported; after fe_geometry_update (the aborted
    launch left the deferred geometry undefined) the next launch is a normal one."""
    P, form, mat, u, Kref, rref, _ = _case(ctx, "elasticity", 2, (10, 10, 10), 98)
    args = [_t(mat, torch.float64), None, None]
    lazy = fe.hex_geometry(ctx, P.m, 2, 3, flags=fe.GEOM_STORE_F32 | fe.GEOM_DEFERRED)
    ctx.status()
    fe.debug_hold_next_matrix(ctx)
    t0 = time.time()
    fe.eval_matrix(ctx, form, lazy, args, "bf16x3")
    st, bad = ctx.status()
    assert st == fe.FE_ERR_TIMEOUT and bad >= 0
    assert time.time() - t0 < 60
    lazy.update()
    K = fe.eval_matrix(ctx, form, lazy, args, "bf16x3")
    ctx.check()
    assert rel_matrix_error(K.cpu().numpy(), Kref) <= TOL["bf16x3"]


@pytest.mark.parametrize("prec,tol", TC_TOL)
def test_tensor_core_laplacian_matches_oracle(ctx, prec, tol):
    """The weighted scalar Laplacian of Q2 hexahedra on the tensor cores, as the
    sum of the diagonal blocks of the elasticity Gram matrix: every element of a
    2,352-element mesh (5 or 6 elements per persistent CTA) against the oracle,
    the zero row sums of the exact matrix, and the unweighted form (c = 1)."""
    P, form, mat, u, Kref, rref, _ = _case(ctx, "laplace", 2, (14, 14, 12), 87)
    K = fe.eval_matrix(ctx, form, P.geom, [_t(mat, torch.float64), None, None], prec)
    ctx.check()
    assert K.shape == (2352, 27, 27) and K.dtype == torch.float32
    Kh = K.cpu().numpy()
    err = rel_matrix_error(Kh, Kref)
    assert err <= tol, err
    scale = np.abs(Kref).max(axis=(1, 2))
    assert (np.abs(Kh.sum(axis=2)).max(axis=1) / scale).max() <= 30 * tol
    K1 = fe.eval_matrix(ctx, fe.laplace_form(), P.geom, [None, None], prec)
    ctx.check()
    wdetJ, G, _ = P.oracle_geometry()
    assert rel_matrix_error(K1.cpu().numpy(), oracle.matrix_laplace(wdetJ, G)) <= tol


def test_tensor_core_q3_elasticity_matches_oracle(ctx):
    """Q3 Lame elasticity (64-node hexahedra, 4 x 4 x 4 points) on the tensor cores in
    TF32x3: the 192-row Gram in two MMA tiles, K_e staged by 64-row blocks; every
    element of a 384-element mesh (two or three elements per persistent CTA) against
    the oracle, symmetry, and BF16 precisions rejected for this element."""
    P, form, mat, u, Kref, rref, _ = _case(ctx, "elasticity", 3, (8, 8, 6), 89)
    args = [_t(mat, torch.float64), None, None]
    K = fe.eval_matrix(ctx, form, P.geom, args, "tf32x3")
    ctx.check()
    assert K.shape == (384, 192, 192) and K.dtype == torch.float32
    Kh = K.cpu().numpy()
    err = rel_matrix_error(Kh, Kref)
    assert err <= TOL["tf32x3"], err
    assert np.abs(Kh - Kh.transpose(0, 2, 1)).max() <= 10 * TOL["tf32x3"] * np.abs(Kh).max()
    for prec in ("bf16x3", "bf16"):
        with pytest.raises(fe.FEError) as ei:
            fe.eval_matrix(ctx, form, P.geom, args, prec)
        assert ei.value.status == fe.FE_ERR_UNSUPPORTED_SPEC


@pytest.mark.parametrize("kind", ["laplace", "mass1"])
def test_tensor_core_q3_scalar_forms_match_oracle(ctx, kind):
    """The weighted scalar Laplacian (diagonal Gram blocks only) and mass matrix
    (Gram of sqrt(w det J) phi) of Q3 hexahedra on the tensor cores in TF32x3: every
    element of a 384-element mesh against the oracle, and symmetry."""
    P, form, mat, u, Kref, rref, _ = _case(ctx, kind, 3, (8, 8, 6), 91)
    K = fe.eval_matrix(ctx, form, P.geom, [_t(mat, torch.float64), None, None], "tf32x3")
    ctx.check()
    assert K.shape == (384, 64, 64) and K.dtype == torch.float32
    Kh = K.cpu().numpy()
    err = rel_matrix_error(Kh, Kref)
    assert err <= TOL["tf32x3"], err
    assert np.abs(Kh - Kh.transpose(0, 2, 1)).max() <= 10 * TOL["tf32x3"] * np.abs(Kh).max()


def test_tensor_core_paths_reject_other_forms(ctx):
    mesh = meshgen.structured_hex(2, 2, 2, 2, 0.0, 0)
    P = Problem(ctx, mesh, 2, 3)
    D = np.tile(np.eye(6), (mesh.n_elems, 1, 1))
    with pytest.raises(fe.FEError) as ei:
        fe.eval_matrix(ctx, fe.elasticity_form(fe.MAT_D66), P.geom, [_t(D, torch.float64), None, None], "tf32x3")
    assert ei.value.status == fe.FE_ERR_UNSUPPORTED_SPEC
    mesh1 = meshgen.structured_hex(2, 2, 2, 1, 0.0, 0)
    P1 = Problem(ctx, mesh1, 1, 2)
    lm = np.ones((mesh1.n_elems, 2))
    with pytest.raises(fe.FEError) as ei:
        fe.eval_matrix(ctx, fe.elasticity_form(), P1.geom, [_t(lm, torch.float64), None, None], "bf16x3")
    assert ei.value.status == fe.FE_ERR_UNSUPPORTED_SPEC


def test_laplace_q1_cube_config(ctx):
    """Plain method, Laplace stiffness on the 8^3 Q1 cube (+-0.1h, seed 0), c = 1."""
    mesh, u = meshgen.laplace_q1_cube(8, 0)
    P = Problem(ctx, mesh, 1, 2)
    wdetJ, G, _ = P.oracle_geometry()
    form = fe.laplace_form()
    K = fe.eval_matrix(ctx, form, P.geom, [None, None], "f64")
    r = fe.eval_residual(ctx, form, P.geom, [None, _t(u, torch.float64)], "f64")
    ctx.check()
    assert K.shape == (512, 8, 8) and K.dtype == torch.float64 and r.shape == (512, 8)
    assert rel_matrix_error(K.cpu().numpy(), oracle.matrix_laplace(wdetJ, G)) <= 1e-12
    assert rel_vector_error(r.cpu().numpy(), oracle.residual_laplace(mesh.conn, wdetJ, G, u)) <= 1e-12


def test_empty_mesh_is_a_no_op(ctx):
    mesh = meshgen.structured_hex(2, 2, 2, 2, 0.0, 0)
    coords = _t(mesh.coords, torch.float64)
    conn = torch.zeros((0, 27), dtype=torch.int32, device="cuda")
    m = fe.Mesh(coords, conn)
    g = fe.hex_geometry(ctx, m, 2, 3)
    K = fe.eval_matrix(ctx, fe.elasticity_form(), g, [torch.zeros((0, 2), dtype=torch.float64, device="cuda"),
                                                       None, None], "f32")
    ctx.check()
    assert K.shape == (0, 81, 81)
    # the step of the benchmark on no elements: deferred geometry computed by the
    # residual kernel, tensor-core matrix, assembly of nothing
    lazy = fe.hex_geometry(ctx, m, 2, 3, flags=fe.GEOM_STORE_F32 | fe.GEOM_DEFERRED)
    lazy.update()
    lm0 = torch.zeros((0, 2), dtype=torch.float64, device="cuda")
    u = torch.zeros(3 * mesh.n_nodes, dtype=torch.float32, device="cuda")
    r = fe.eval_residual(ctx, fe.elasticity_form(), lazy, [lm0, None, u], "bf16x3")
    K = fe.eval_matrix(ctx, fe.elasticity_form(), lazy, [lm0, None, None], "bf16x3")
    gv = fe.assemble_vector(ctx, fe.assembly_create(ctx, m), 3, r, "f32", flags=fe.ASSEMBLE_COMPENSATED)
    ctx.check()
    assert r.shape == (0, 81) and K.shape == (0, 81, 81)
    assert gv.shape == (3 * mesh.n_nodes,) and not torch.any(gv)


def test_argument_errors(ctx):
    mesh = meshgen.structured_hex(2, 2, 2, 2, 0.0, 0)
    P = Problem(ctx, mesh, 2, 3)
    form = fe.laplace_form()
    with pytest.raises(fe.FEError) as ei:
        fe.eval_matrix(ctx, form, P.geom, [None, None], "f64", diff_op=0)  # not the state operand
    assert ei.value.status == fe.FE_ERR_INVALID_ARG
    with pytest.raises(fe.FEError) as ei:  # no tensor-core kernel for the mass matrix
        fe.eval_matrix(ctx, fe.mass_form(), P.geom, [None, None], "bf16x3")
    assert ei.value.status == fe.FE_ERR_UNSUPPORTED_SPEC
    # unsupported (N, Q) pair
    pts, w, phi, dphi = fe.refbasis_hex(2, 2)
    with pytest.raises(fe.FEError) as ei:
        fe.geometry(ctx, P.m, phi, dphi, w)
    assert ei.value.status == fe.FE_ERR_SHAPE
    # a geometry without the float32 copy cannot feed the float32 kernels
    pts, w, phi, dphi = fe.refbasis_hex(2, 3)
    g64 = fe.geometry(ctx, P.m, phi, dphi, w, flags=fe.GEOM_STORE_F64)
    with pytest.raises(fe.FEError) as ei:
        fe.eval_matrix(ctx, form, g64, [None, None], "f32")
    assert ei.value.status == fe.FE_ERR_INVALID_ARG
    ctx.check()


# ---- assembly -------------------------------------------------------------------------

@pytest.mark.parametrize("p,ncomp", [(1, 1), (2, 3)])
def test_assembly_fp64_is_bit_exact(ctx, p, ncomp):
    mesh = meshgen.structured_hex(5, 4, 3, p, 0.1, 51)
    rng = np.random.default_rng(52)
    r = rng.standard_normal((mesh.n_elems, ncomp * mesh.nodes_per_elem))
    want = oracle.assemble(mesh.conn, r, mesh.n_nodes, ncomp)
    m = fe.Mesh(_t(mesh.coords, torch.float64), _t(mesh.conn, torch.int32))
    asm = fe.assembly_create(ctx, m)
    got = fe.assemble_vector(ctx, asm, ncomp, _t(r, torch.float64), "f64").cpu().numpy()
    np.testing.assert_array_equal(got, want)
    g0 = rng.standard_normal(mesh.n_nodes * ncomp)
    out = _t(g0, torch.float64)
    fe.assemble_vector(ctx, asm, ncomp, _t(r, torch.float64), "f64", out=out, flags=fe.ASSEMBLE_ACCUMULATE)
    np.testing.assert_array_equal(out.cpu().numpy(), oracle.assemble(mesh.conn, r, mesh.n_nodes, ncomp, g0))


def test_assembly_fp32_compensated(ctx):
    mesh = meshgen.structured_hex(6, 5, 4, 2, 0.1, 53)
    rng = np.random.default_rng(54)
    # large cancelling contributions make plain float32 sums lose digits
    r = rng.standard_normal((mesh.n_elems, 81)) * 1e4
    r[:, ::2] += 1e7
    r[:, 1::2] -= 1e7
    want = oracle.assemble(mesh.conn, r.astype(np.float32).astype(np.float64), mesh.n_nodes, 3)
    m = fe.Mesh(_t(mesh.coords, torch.float64), _t(mesh.conn, torch.int32))
    asm = fe.assembly_create(ctx, m)
    r32 = _t(r, torch.float32)
    comp = fe.assemble_vector(ctx, asm, 3, r32, "f32", flags=fe.ASSEMBLE_COMPENSATED).cpu().numpy()
    plain = fe.assemble_vector(ctx, asm, 3, r32, "f32").cpu().numpy()
    # Neumaier: |s - S| <= u |S| + O(n u^2) sum |x|, u = 2^-24, after the final
    # rounding of s + c to float32; the plain sum has no such bound
    sumabs = oracle.assemble(mesh.conn, np.abs(r.astype(np.float32)).astype(np.float64), mesh.n_nodes, 3)
    bound = 2.0 ** -24 * np.abs(want) + 64 * 2.0 ** -48 * sumabs
    assert np.all(np.abs(comp - want) <= bound)
    assert np.abs(plain - want).max() > np.abs(comp - want).max()
    again = fe.assemble_vector(ctx, asm, 3, r32, "f32", flags=fe.ASSEMBLE_COMPENSATED).cpu().numpy()
    np.testing.assert_array_equal(comp, again)  # deterministic


def test_assembly_rejects_out_of_range_nodes(ctx):
    mesh = meshgen.structured_hex(2, 2, 2, 1, 0.0, 0)
    conn = mesh.conn.copy()
    conn[3, 2] = mesh.n_nodes + 5
    m = fe.Mesh(_t(mesh.coords, torch.float64), _t(conn, torch.int32))
    with pytest.raises(fe.FEError) as ei:
        fe.assembly_create(ctx, m)
    assert ei.value.status == fe.FE_ERR_SHAPE


def test_results_are_deterministic(ctx):
    P, form, mat, u, Kref, rref, _ = _case(ctx, "elasticity", 2, (4, 3, 3), 61)
    args = [_t(mat, torch.float64), None, _t(u, torch.float32)]
    K1 = fe.eval_matrix(ctx, form, P.geom, args, "f32")
    K2 = fe.eval_matrix(ctx, form, P.geom, args, "f32")
    r1 = fe.eval_residual(ctx, form, P.geom, args, "f32")
    r2 = fe.eval_residual(ctx, form, P.geom, args, "f32")
    assert torch.equal(K1, K2) and torch.equal(r1, r2)


def test_geometry_views_evaluate_element_ranges(ctx):
    """A view over an element range aliases the parent's geometry: its matrices
    and residuals equal the parent's on that range bit for bit, and updating a
    view recomputes its range only."""
    mesh = meshgen.structured_hex(5, 4, 3, 2, 0.15, 7)
    lam, mu = meshgen.lame_materials(mesh)
    P = Problem(ctx, mesh, 2, 3)
    form = fe.elasticity_form(fe.MAT_LAME)
    mat = _t(np.stack([lam, mu], 1), torch.float64)
    u = _t(meshgen.normal_dofs(mesh, 3), torch.float32)
    K = fe.eval_matrix(ctx, form, P.geom, [mat, None, None], "f32")
    r = fe.eval_residual(ctx, form, P.geom, [mat, None, u], "f32")
    for e0, n in ((0, 7), (7, 30), (37, mesh.n_elems - 37)):
        v = P.geom.view(e0, n)
        v.update()
        Kv = fe.eval_matrix(ctx, form, v, [mat[e0:e0 + n], None, None], "f32")
        rv = fe.eval_residual(ctx, form, v, [mat[e0:e0 + n], None, u], "f32")
        ctx.check()
        assert torch.equal(Kv, K[e0:e0 + n])
        assert torch.equal(rv, r[e0:e0 + n])
        v.free()
    with pytest.raises(fe.FEError):
        P.geom.view(mesh.n_elems - 2, 3)
