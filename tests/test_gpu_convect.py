"""GPU parity of the Navier-Stokes convective term 'i,i.j,j' (Eq. fe2) and its
derivative (Eq. fe4): libfe through the C ABI against the FP64 oracle."""
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


# (p, nq, cells): every (n1d, nq1d) pair with a kernel; cell counts leave a
# ragged last CTA for the element counts per CTA of both precisions
CASES = [(1, 2, (5, 4, 3)), (1, 3, (3, 3, 3)), (2, 3, (5, 3, 3)), (2, 4, (3, 2, 2)), (3, 4, (2, 2, 3))]
ROLES = {"nonlinear": (fe.STATE, fe.STATE), "wrt_u": (fe.STATE, fe.PARAMETER), "wrt_w": (fe.PARAMETER, fe.STATE)}


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("roles", list(ROLES))
@pytest.mark.parametrize("p,nq,n", CASES)
def test_convect_matches_oracle(ctx, p, nq, n, roles, prec):
    mesh = meshgen.structured_hex(*n, p, 0.15, 40 + p)
    P = Problem(ctx, mesh, p, nq)
    wdetJ, G, _ = P.oracle_geometry()
    rng = np.random.default_rng(50 + p)
    u = rng.standard_normal(3 * mesh.n_nodes)
    gr, ad = ROLES[roles]
    w = u if roles == "nonlinear" else rng.standard_normal(3 * mesh.n_nodes)
    form = fe.convect_form(advection=ad, gradient=gr)
    dt = torch.float64 if prec == "f64" else torch.float32
    ud = _t(u, dt)
    wd = ud if roles == "nonlinear" else _t(w, dt)
    args = [None, ud, wd]
    K = fe.eval_matrix(ctx, form, P.geom, args, prec)
    r = fe.eval_residual(ctx, form, P.geom, args, prec)
    ctx.check()
    Kref = oracle.matrix_convect(mesh.conn, wdetJ, P.ref.phi, G, u, w, wrt_u=gr == fe.STATE,
                                 wrt_w=ad == fe.STATE)
    rref = oracle.residual_convect(mesh.conn, wdetJ, P.ref.phi, G, u, w)
    ek = rel_matrix_error(K.cpu().numpy(), Kref)
    er = rel_vector_error(r.cpu().numpy(), rref)
    assert ek <= TOL[prec], ek
    assert er <= TOL[prec], er


@pytest.mark.parametrize("roles", ["nonlinear", "wrt_u"])
@pytest.mark.parametrize("p,n", [(1, (5, 4, 3)), (2, (5, 3, 3)), (3, (2, 2, 3)), (2, (20, 19, 18))])
def test_convect_residual_computes_stale_geometry(ctx, p, n, roles):
    """fe_eval_residual of the convective form on a stale float32-only deferred
    handle computes the FP64 geometry in the residual kernel: r, the stored copy and
    the matrix that follows equal the eager path's bit for bit (the largest case puts
    several element groups on every CTA)."""
    mesh = meshgen.structured_hex(*n, p, 0.15, 60 + p)
    P = Problem(ctx, mesh, p, p + 1)
    rng = np.random.default_rng(61 + p)
    u = _t(rng.standard_normal(3 * mesh.n_nodes), torch.float32)
    w = u if roles == "nonlinear" else _t(rng.standard_normal(3 * mesh.n_nodes), torch.float32)
    gr, ad = ROLES[roles]
    form = fe.convect_form(advection=ad, gradient=gr)
    eager = fe.hex_geometry(ctx, P.m, p, p + 1, flags=fe.GEOM_STORE_F32)
    lazy = fe.hex_geometry(ctx, P.m, p, p + 1, flags=fe.GEOM_STORE_F32 | fe.GEOM_DEFERRED)
    r_e = fe.eval_residual(ctx, form, eager, [None, u, w], "f32")
    for _ in range(2):
        lazy.update()
        r_l = fe.eval_residual(ctx, form, lazy, [None, u, w], "f32")
    ctx.check()
    assert torch.equal(r_l, r_e)
    assert torch.equal(lazy.get(fe.GEOM_JINV, "f32"), eager.get(fe.GEOM_JINV, "f32"))
    assert torch.equal(lazy.get(fe.GEOM_WDETJ, "f32"), eager.get(fe.GEOM_WDETJ, "f32"))
    assert torch.equal(fe.eval_matrix(ctx, form, lazy, [None, u, w], "f32"),
                       fe.eval_matrix(ctx, form, eager, [None, u, w], "f32"))
    if mesh.n_elems <= 100:
        wdetJ, G, _ = P.oracle_geometry()
        uh, wh = u.double().cpu().numpy(), w.double().cpu().numpy()
        rref = oracle.residual_convect(mesh.conn, wdetJ, P.ref.phi, G, uh, wh)
        assert rel_vector_error(r_l.cpu().numpy(), rref) <= TOL["f32"]


@pytest.mark.parametrize("roles", ["nonlinear", "wrt_u", "wrt_w"])
@pytest.mark.parametrize("p,n", [(1, (5, 4, 3)), (2, (5, 3, 3)), (3, (2, 2, 3)), (2, (20, 19, 18))])
def test_convect_matrix_computes_stale_geometry(ctx, p, n, roles):
    """fe_eval_matrix of the convective form on a stale float32-only deferred handle
    computes the FP64 geometry in the matrix kernel: K, the stored copy and the
    residual that follows equal the eager path's bit for bit (the largest case puts
    several element groups on every CTA), and K matches the oracle on small meshes."""
    mesh = meshgen.structured_hex(*n, p, 0.15, 80 + p)
    P = Problem(ctx, mesh, p, p + 1)
    rng = np.random.default_rng(81 + p)
    u = _t(rng.standard_normal(3 * mesh.n_nodes), torch.float32)
    w = u if roles == "nonlinear" else _t(rng.standard_normal(3 * mesh.n_nodes), torch.float32)
    gr, ad = ROLES[roles]
    form = fe.convect_form(advection=ad, gradient=gr)
    eager = fe.hex_geometry(ctx, P.m, p, p + 1, flags=fe.GEOM_STORE_F32)
    lazy = fe.hex_geometry(ctx, P.m, p, p + 1, flags=fe.GEOM_STORE_F32 | fe.GEOM_DEFERRED)
    K_e = fe.eval_matrix(ctx, form, eager, [None, u, w], "f32")
    for _ in range(2):
        lazy.update()
        K_l = fe.eval_matrix(ctx, form, lazy, [None, u, w], "f32")
    ctx.check()
    assert torch.equal(K_l, K_e)
    assert torch.equal(lazy.get(fe.GEOM_JINV, "f32"), eager.get(fe.GEOM_JINV, "f32"))
    assert torch.equal(lazy.get(fe.GEOM_WDETJ, "f32"), eager.get(fe.GEOM_WDETJ, "f32"))
    assert torch.equal(fe.eval_residual(ctx, form, lazy, [None, u, w], "f32"),
                       fe.eval_residual(ctx, form, eager, [None, u, w], "f32"))
    if mesh.n_elems <= 100:
        wdetJ, G, _ = P.oracle_geometry()
        uh, wh = u.double().cpu().numpy(), w.double().cpu().numpy()
        Kref = oracle.matrix_convect(mesh.conn, wdetJ, P.ref.phi, G, uh, wh, wrt_u=gr == fe.STATE,
                                     wrt_w=ad == fe.STATE)
        assert rel_matrix_error(K_l.cpu().numpy(), Kref) <= TOL["f32"]


def test_convect_smooth_field_config_small(ctx):
    """The smooth field sin(pi x) cos(pi y) a of the convection workload on a
    small cube; the assembled residual (compensated FP32) against the oracle's."""
    mesh, u = meshgen.convect_q2_cube(6, seed=3)
    P = Problem(ctx, mesh, 2, 3)
    wdetJ, G, _ = P.oracle_geometry()
    form = fe.convect_form()
    for prec, dt in (("f64", torch.float64), ("f32", torch.float32)):
        ud = _t(u, dt)
        K = fe.eval_matrix(ctx, form, P.geom, [None, ud, ud], prec)
        r = fe.eval_residual(ctx, form, P.geom, [None, ud, ud], prec)
        asm = fe.assembly_create(ctx, P.m)
        flags = fe.ASSEMBLE_COMPENSATED if prec == "f32" else 0
        g = fe.assemble_vector(ctx, asm, 3, r, prec, flags=flags)
        ctx.check()
        Kref = oracle.matrix_convect(mesh.conn, wdetJ, P.ref.phi, G, u)
        rref = oracle.residual_convect(mesh.conn, wdetJ, P.ref.phi, G, u)
        gref = oracle.assemble(mesh.conn, rref, mesh.n_nodes, 3)
        assert rel_matrix_error(K.cpu().numpy(), Kref) <= TOL[prec]
        assert rel_vector_error(r.cpu().numpy(), rref) <= TOL[prec]
        assert rel_vector_error(g.cpu().numpy(), gref) <= TOL[prec]


def test_convect_full_size_sampled_and_homogeneity(ctx):
    """64^3 Q2 cube (262,144 elements), the launch configuration of the
    benchmark: 64 sampled elements against the oracle in both precisions, and
    over all elements the degree-2 identity K(u) u_e = 2 r(u) in FP64."""
    mesh, u = meshgen.convect_q2_cube(64, seed=3)
    P = Problem(ctx, mesh, 2, 3)
    E = mesh.n_elems
    rng = np.random.default_rng(9)
    idx = np.unique(np.concatenate([[0, E - 1], rng.choice(E, 62, replace=False)]))
    wdetJ, G, _ = P.oracle_geometry(idx)
    Kref = oracle.matrix_convect(mesh.conn[idx], wdetJ, P.ref.phi, G, u)
    rref = oracle.residual_convect(mesh.conn[idx], wdetJ, P.ref.phi, G, u)
    form = fe.convect_form()
    for prec, dt in (("f32", torch.float32), ("f64", torch.float64)):
        ud = _t(u, dt)
        K = fe.eval_matrix(ctx, form, P.geom, [None, ud, ud], prec)
        r = fe.eval_residual(ctx, form, P.geom, [None, ud, ud], prec)
        ctx.check()
        sel = torch.from_numpy(idx).cuda()
        assert rel_matrix_error(K[sel].cpu().numpy(), Kref) <= TOL[prec]
        assert rel_vector_error(r[sel].cpu().numpy(), rref) <= TOL[prec]
        if prec == "f64":
            conn = P.conn_d.long()
            ue = torch.cat([ud[3 * conn + i] for i in range(3)], dim=1)      # (E, 81)
            Ku = torch.bmm(K, ue.unsqueeze(2)).squeeze(2)
            err = ((Ku - 2 * r).norm() / (2 * r).norm()).item()
            assert err <= 1e-12, err
        del K


def test_convect_rejections(ctx):
    mesh = meshgen.structured_hex(2, 2, 2, 2, 0.1, 3)
    P = Problem(ctx, mesh, 2, 3)
    u = _t(np.zeros(3 * mesh.n_nodes), torch.float32)
    form = fe.convect_form()
    for prec in ("tf32x3", "bf16x3", "bf16"):
        with pytest.raises(fe.FEError) as ei:
            fe.eval_matrix(ctx, form, P.geom, [None, u, u], prec)
        assert ei.value.status == fe.FE_ERR_UNSUPPORTED_SPEC
    # derivative with respect to a known field
    lin = fe.convect_form(advection=fe.PARAMETER)
    with pytest.raises(fe.FEError) as ei:
        fe.eval_matrix(ctx, lin, P.geom, [None, u, u], "f32", diff_op=2)
    assert ei.value.status == fe.FE_ERR_INVALID_ARG
    # a basis without its 1-D factors has no sum-factorised kernel
    _, wq, phi, dphi = fe.refbasis_hex(2, 3)
    g2 = fe.geometry(ctx, P.m, phi, dphi, wq)
    with pytest.raises(fe.FEError) as ei:
        fe.eval_residual(ctx, form, g2, [None, u, u], "f32")
    assert ei.value.status == fe.FE_ERR_UNSUPPORTED_SPEC


def test_convect_empty_mesh(ctx):
    coords = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
    conn = torch.zeros((0, 27), dtype=torch.int32, device="cuda")
    m = fe.Mesh(coords, conn)
    g = fe.hex_geometry(ctx, m, 2, 3)
    u = torch.zeros(3, dtype=torch.float32, device="cuda")
    form = fe.convect_form()
    K = fe.eval_matrix(ctx, form, g, [None, u, u], "f32")
    r = fe.eval_residual(ctx, form, g, [None, u, u], "f32")
    ctx.check()
    assert K.shape == (0, 81, 81) and r.shape == (0, 81)
