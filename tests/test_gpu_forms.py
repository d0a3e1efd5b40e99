"""GPU parity of the remaining Tab. ewfd forms (weighted dot product, Stokes
coupling and its transpose, divergence) and of 'eval' mode for every form
(including the Cauchy stress), against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2107_04121_gb300 import fe, meshgen
from tests.parity import TOL, Problem, rel_vector_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

V, S, PA, M = fe.VIRTUAL, fe.STATE, fe.PARAMETER, fe.MATERIAL
NONE = fe.MAT_NONE


@pytest.fixture(scope="module")
def ctx(libfe):
    c = fe.Context(0)
    yield c
    c.close()


def _t(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)


def _case(ctx, elem, seed):
    if elem == "tet2":
        mesh = meshgen.tet_mesh(97, 2, np.random.default_rng(seed))
        ref = oracle.RefTet(2, 2)
        m = fe.Mesh(_t(mesh.coords, torch.float64), _t(mesh.conn, torch.int32))
        geom = fe.tet_geometry(ctx, m, 2)
        wdetJ, G, _ = oracle.geometry(mesh.coords, mesh.conn, ref)
        return mesh, ref, geom, wdetJ, G
    p = int(elem[1])
    mesh = meshgen.structured_hex(5, 3, 3, p, 0.15, seed) if p == 1 else meshgen.structured_hex(3, 3, 2, p, 0.15, seed)
    P = Problem(ctx, mesh, p, p + 1)
    wdetJ, G, _ = P.oracle_geometry()
    return mesh, P.ref, P.geom, wdetJ, G


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("elem", ["q1", "q2", "tet2"])
def test_weak_forms_match_oracle(ctx, elem, prec):
    mesh, ref, geom, wdetJ, G = _case(ctx, elem, 120)
    dt = torch.float64 if prec == "f64" else torch.float32
    rng = np.random.default_rng(121)
    E, nn = mesh.n_elems, mesh.n_nodes
    u3, p1 = rng.standard_normal(3 * nn), rng.standard_normal(nn)
    Mm = rng.standard_normal((E, 3, 3))
    tol = TOL[prec] * (20 if elem == "tet2" else 1)  # alternating GM weights (see test_gpu_tets)
    # weighted dot product
    f = fe.form_compile("ij,i,j", [(M, 1, fe.MAT_M33), (V, 3, NONE), (S, 3, NONE)])
    args = [_t(Mm, torch.float64), None, _t(u3, dt)]
    K = fe.eval_matrix(ctx, f, geom, args, prec)
    r = fe.eval_residual(ctx, f, geom, args, prec)
    assert _rel(K.cpu().numpy(), oracle.matrix_wdot(wdetJ, ref.phi, Mm)) <= tol
    assert _rel(r.cpu().numpy(), oracle.residual_wdot(mesh.conn, wdetJ, ref.phi, Mm, u3)) <= tol
    # Stokes coupling (v, p) and its transpose (u, q)
    B = oracle.matrix_stokes(wdetJ, G, ref.phi)
    f = fe.form_compile("i.i,0", [(V, 3, NONE), (S, 1, NONE)])
    K = fe.eval_matrix(ctx, f, geom, [None, _t(p1, dt)], prec)
    r = fe.eval_residual(ctx, f, geom, [None, _t(p1, dt)], prec)
    assert tuple(K.shape) == (E, 3 * ref.N, ref.N)
    assert _rel(K.cpu().numpy(), B) <= tol
    assert _rel(r.cpu().numpy(), oracle.residual_stokes(mesh.conn, wdetJ, G, ref.phi, p1)) <= tol
    f = fe.form_compile("i.i,0", [(S, 3, NONE), (V, 1, NONE)])
    K = fe.eval_matrix(ctx, f, geom, [_t(u3, dt), None], prec)
    r = fe.eval_residual(ctx, f, geom, [_t(u3, dt), None], prec)
    assert _rel(K.cpu().numpy(), B.transpose(0, 2, 1)) <= tol
    assert _rel(r.cpu().numpy(), oracle.residual_stokes_t(mesh.conn, wdetJ, G, ref.phi, u3)) <= tol
    # divergence (a linear form: residual only)
    f = fe.form_compile("i.i", [(V, 3, NONE)])
    r = fe.eval_residual(ctx, f, geom, [None], prec)
    assert _rel(r.cpu().numpy(), oracle.residual_stokes(mesh.conn, wdetJ, G, ref.phi)) <= tol
    with pytest.raises(fe.FEError):
        fe.eval_matrix(ctx, f, geom, [None], prec, diff_op=0)
    ctx.check()


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("elem", ["q1", "q2", "tet2"])
def test_eval_mode_matches_oracle(ctx, elem, prec):
    mesh, ref, geom, wdetJ, G = _case(ctx, elem, 130)
    dt = torch.float64 if prec == "f64" else torch.float32
    rng = np.random.default_rng(131)
    E, nn = mesh.n_elems, mesh.n_nodes
    s1, s2 = rng.standard_normal(nn), rng.standard_normal(nn)
    u, w, z = (rng.standard_normal(3 * nn) for _ in range(3))
    coef = rng.uniform(0.5, 2.0, E)
    lam, mu = rng.uniform(0.5, 2.0, E), rng.uniform(0.2, 1.0, E)
    D = oracle.lame_to_D(lam, mu)
    Mm = rng.standard_normal((E, 3, 3))
    tol = TOL[prec] * (20 if elem == "tet2" else 1)
    T = lambda a: _t(a, dt)
    F64 = lambda a: _t(a, torch.float64)
    cases = [
        ("0,0.i,0.i", [(M, 1, fe.MAT_SCALAR), (PA, 1, NONE), (PA, 1, NONE)], [F64(coef), T(s1), T(s2)],
         dict(kind="laplace", u=s1, w=s2, coef=coef)),
        ("0,0,0", [(M, 1, fe.MAT_SCALAR), (PA, 1, NONE), (S, 1, NONE)], [F64(coef), T(s1), T(s2)],
         dict(kind="mass", u=s1, w=s2, coef=coef, ncomp=1)),
        ("i,i", [(PA, 3, NONE), (PA, 3, NONE)], [T(u), T(w)], dict(kind="mass", u=u, w=w)),
        ("IK,s(i:j)->I,s(k:l)->K", [(M, 1, fe.MAT_LAME), (PA, 3, NONE), (PA, 3, NONE)],
         [F64(np.stack([lam, mu], 1)), T(u), T(w)], dict(kind="elasticity", u=u, w=w, mat=D)),
        ("ij,i,j", [(M, 1, fe.MAT_M33), (PA, 3, NONE), (PA, 3, NONE)], [F64(Mm), T(u), T(w)],
         dict(kind="wdot", u=u, w=w, mat=Mm)),
        ("i.i,0", [(PA, 3, NONE), (PA, 1, NONE)], [T(u), T(s1)], dict(kind="stokes", u=u, w=s1)),
        ("i.i", [(PA, 3, NONE)], [T(u)], dict(kind="div", u=u)),
        ("IK,s(k:l)->K", [(M, 1, fe.MAT_D66), (PA, 3, NONE)], [F64(D), T(u)], dict(kind="cauchy", u=u, mat=D)),
        ("i,i.j,j", [(PA, 3, NONE), (PA, 3, NONE), (PA, 3, NONE)], [T(u), T(w), T(z)],
         dict(kind="convect", u=u, w=w, z=z)),
    ]
    for expr, ops, args, ref_kw in cases:
        f = fe.form_compile(expr, ops)
        got = fe.eval_integral(ctx, f, geom, args, prec).cpu().numpy()
        kind = ref_kw.pop("kind")
        want = oracle.eval_form(kind, mesh.conn, wdetJ, G, ref.phi, **ref_kw)
        e = rel_vector_error(got, want)
        assert e <= tol, (expr, e)
    ctx.check()


def test_eval_and_weak_mode_misuse_is_rejected(ctx):
    mesh, ref, geom, wdetJ, G = _case(ctx, "q1", 140)
    u = _t(np.zeros(mesh.n_nodes), torch.float32)
    fev = fe.form_compile("0.i,0.i", [(PA, 1, NONE), (PA, 1, NONE)])
    with pytest.raises(fe.FEError):
        fe.eval_residual(ctx, fev, geom, [u, u], "f32")
    fw = fe.laplace_form()
    with pytest.raises(fe.FEError):
        fe.eval_integral(ctx, fw, geom, [None, u], "f32")


# ---- the Stokes coupling between fields of different orders (Taylor-Hood pairs) ----------

def _mixed_case(ctx, kind, seed):
    if kind == "Q2/Q1":
        mesh = meshgen.structured_hex(5, 4, 3, 2, 0.15, seed)
        m = fe.Mesh(_t(mesh.coords, torch.float64), _t(mesh.conn, torch.int32))
        geom = fe.hex_geometry(ctx, m, 2, 3)
        ref_u, ref_p = oracle.RefElement(2, 3), oracle.RefElement(1, 3)
        psi = fe.refbasis_hex(1, 3)[2]  # the library's Q1 basis at the 3 x 3 x 3 points
    else:
        mesh = meshgen.tet_mesh(97, 2, np.random.default_rng(seed))
        m = fe.Mesh(_t(mesh.coords, torch.float64), _t(mesh.conn, torch.int32))
        geom = fe.tet_geometry(ctx, m, 2)
        ref_u, ref_p = oracle.RefTet(2, 2), oracle.RefTet(1, 2)
        psi = fe.refbasis_tet(1, 2)[2]  # the library's P1 basis at the rule of P2
    conn_p, n_p = meshgen.vertex_connectivity(mesh)
    field = fe.Field(ctx, geom, psi, _t(conn_p, torch.int32), n_p)
    wdetJ, G, _ = oracle.geometry(mesh.coords, mesh.conn, ref_u)
    return mesh, geom, field, conn_p, n_p, ref_p, wdetJ, G


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("kind", ["Q2/Q1", "P2/P1"])
def test_mixed_order_stokes_matches_oracle(ctx, kind, prec):
    """The coupling div(v) p with a Q1 (P1) pressure beside a Q2 (P2) velocity and
    its transpose q div(u): element matrices (3N x Np and Np x 3N) and residuals
    against the oracle on distorted hexahedra and Delaunay tetrahedra."""
    mesh, geom, field, conn_p, n_p, ref_p, wdetJ, G = _mixed_case(ctx, kind, 130)
    dt = torch.float64 if prec == "f64" else torch.float32
    tol = TOL[prec] * (20 if kind == "P2/P1" else 1)  # alternating GM weights (see test_gpu_tets)
    rng = np.random.default_rng(131)
    p, u = rng.standard_normal(n_p), rng.standard_normal(3 * mesh.n_nodes)
    Bref = oracle.matrix_stokes_mixed(wdetJ, G, ref_p.phi)
    fs = fe.form_compile("i.i,0", [(V, 3, NONE), (S, 1, NONE)])
    ft = fe.form_compile("i.i,0", [(S, 3, NONE), (V, 1, NONE)])
    B = fe.eval_matrix_mixed(ctx, fs, geom, field, [None, None], prec)
    Bt = fe.eval_matrix_mixed(ctx, ft, geom, field, [None, None], prec)
    r = fe.eval_residual_mixed(ctx, fs, geom, field, [None, _t(p, dt)], prec)
    rt = fe.eval_residual_mixed(ctx, ft, geom, field, [_t(u, dt), None], prec)
    ctx.check()
    E, N, Np = mesh.n_elems, geom.N, field.n_basis
    assert B.shape == (E, 3 * N, Np) and Bt.shape == (E, Np, 3 * N)
    assert _rel(B.cpu().numpy(), Bref) <= tol
    assert _rel(Bt.cpu().numpy(), Bref.transpose(0, 2, 1)) <= tol
    assert rel_vector_error(r.cpu().numpy(), oracle.residual_stokes_mixed(conn_p, wdetJ, G, ref_p.phi, p)) <= tol
    assert rel_vector_error(rt.cpu().numpy(),
                            oracle.residual_stokes_t_mixed(mesh.conn, wdetJ, G, ref_p.phi, u)) <= tol
    field.free()


def test_mixed_order_stokes_reports_out_of_range_pressure_nodes(ctx):
    mesh, geom, field, conn_p, n_p, ref_p, wdetJ, G = _mixed_case(ctx, "Q2/Q1", 132)
    bad = conn_p.copy()
    bad[4, 3] = n_p + 7
    fb = fe.Field(ctx, geom, fe.refbasis_hex(1, 3)[2], _t(bad, torch.int32), n_p)
    fs = fe.form_compile("i.i,0", [(V, 3, NONE), (S, 1, NONE)])
    ctx.status()
    fe.eval_residual_mixed(ctx, fs, geom, fb, [None, _t(np.ones(n_p), torch.float64)], "f64")
    assert ctx.status() == (fe.FE_ERR_SHAPE, 4)
    fb.free()
    field.free()
