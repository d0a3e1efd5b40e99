"""GPU parity on tetrahedral meshes (P1-P3, Grundmann-Moller rules of index p):
geometry, matrix and residual modes of the Tab. ewfd forms against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2107_04121_gb300 import fe, meshgen
from tests.parity import TOL, rel_vector_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(libfe):
    c = fe.Context(0)
    yield c
    c.close()


def _t(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)


# element counts leave a ragged last CTA for every tile configuration
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("kind", ["laplace", "mass", "elasticity"])
@pytest.mark.parametrize("p,E", [(1, 301), (2, 157), (3, 83)])
def test_tet_matrix_and_residual_match_oracle(ctx, p, E, kind, prec):
    mesh = meshgen.tet_mesh(E, p, np.random.default_rng(80 + p))
    ref = oracle.RefTet(p, p)
    wdetJ, G, _ = oracle.geometry(mesh.coords, mesh.conn, ref)
    rng = np.random.default_rng(81)
    m = fe.Mesh(_t(mesh.coords, torch.float64), _t(mesh.conn, torch.int32))
    geom = fe.tet_geometry(ctx, m, p)
    dt = torch.float64 if prec == "f64" else torch.float32
    aw, aG, aphi = np.abs(wdetJ), np.abs(G), np.abs(ref.phi)
    if kind == "laplace":
        coef = rng.uniform(0.5, 2.0, E)
        form = fe.laplace_form(weighted=True)
        mat, nc = coef, 1
        Kref = oracle.matrix_laplace(wdetJ, G, coef)
        Kabs = oracle.matrix_laplace(aw, aG, coef)
        u = rng.standard_normal(mesh.n_nodes)
        rref = oracle.residual_laplace(mesh.conn, wdetJ, G, u, coef)
        rabs = oracle.residual_laplace(mesh.conn, aw, aG, np.abs(u), coef)
    elif kind == "mass":
        coef = rng.uniform(0.5, 2.0, E)
        form = fe.mass_form(1, weighted=True)
        mat, nc = coef, 1
        Kref = oracle.matrix_mass(wdetJ, ref.phi, 1, coef)
        Kabs = oracle.matrix_mass(aw, aphi, 1, coef)
        u = rng.standard_normal(mesh.n_nodes)
        rref = oracle.residual_mass(mesh.conn, wdetJ, ref.phi, u, 1, coef)
        rabs = oracle.residual_mass(mesh.conn, aw, aphi, np.abs(u), 1, coef)
    else:
        lam, mu = meshgen.lame_materials(mesh)
        form = fe.elasticity_form(fe.MAT_LAME)
        mat, nc = np.stack([lam, mu], 1), 3
        D = oracle.lame_to_D(lam, mu)
        Kref = oracle.matrix_elasticity(wdetJ, G, D)
        Kabs = oracle.matrix_elasticity(aw, aG, np.abs(D))
        u = rng.standard_normal(3 * mesh.n_nodes)
        rref = oracle.residual_elasticity(mesh.conn, wdetJ, G, D, u)
        rabs = oracle.residual_elasticity(mesh.conn, aw, aG, np.abs(D), np.abs(u))
    # Grundmann-Moller weights alternate in sign and P3 basis products change
    # sign, so element entries can be much smaller than the terms summed into
    # them: errors are measured against the sums of absolute terms (the same
    # forms of |w det J|, |phi|, |G|, |D|, |u|), the scale two summation orders
    # of the same terms differ on
    tol = TOL[prec]
    args = [_t(mat, torch.float64), None, _t(u, dt)]
    K = fe.eval_matrix(ctx, form, geom, args, prec)
    r = fe.eval_residual(ctx, form, geom, args, prec)
    wd = geom.get(fe.GEOM_WDETJ, prec)
    ctx.check()
    assert rel_vector_error(wd.cpu().numpy(), wdetJ) <= TOL[prec]
    Kg = K.cpu().numpy().astype(np.float64)
    ek = float((np.sqrt(((Kg - Kref) ** 2).sum((1, 2))) / np.sqrt((Kabs ** 2).sum((1, 2)))).max())
    er = float(np.linalg.norm(r.cpu().numpy() - rref) / np.linalg.norm(rabs))
    assert ek <= tol, ek
    assert er <= tol, er


def test_tet_refbasis_matches_oracle(libfe):
    for p in (1, 2, 3):
        for s in (0, 1, 2, 3, 4):
            pts, w, phi, dphi = fe.refbasis_tet(p, s)
            opts, ow = oracle.gm_rule(s)
            ophi, odphi = oracle.tet_basis(p, opts)
            np.testing.assert_allclose(pts, opts, atol=1e-15)
            np.testing.assert_allclose(w, ow, rtol=1e-13, atol=1e-16)
            np.testing.assert_allclose(phi, ophi, atol=1e-13)
            np.testing.assert_allclose(dphi, odphi, atol=1e-12)


@pytest.mark.parametrize("p,E", [(1, 301), (2, 157), (3, 83)])
def test_float32_tet_geometry_straight_and_curved(ctx, p, E):
    """A float32-only handle of the library's tetrahedron basis: straight-sided
    elements take J from their vertices (once per element), elements whose edge
    nodes moved off the straight edges take the isoparametric sum at every point;
    both against the oracle's FP64 geometry (float32 copies: a few float32 ulps)."""
    mesh = meshgen.tet_mesh(E, p, np.random.default_rng(85 + p))
    coords = mesh.coords.copy()
    if p > 1:
        # bend the edges of the first elements: move their non-vertex nodes
        h = np.abs(coords[mesh.conn[:5, 1]] - coords[mesh.conn[:5, 0]]).max()
        rng = np.random.default_rng(86)
        moved = np.unique(mesh.conn[:5, 1:p])
        coords[moved] += 0.05 * h * rng.uniform(-1, 1, (len(moved), 3))
    ref = oracle.RefTet(p, p)
    wdetJ, _, Jinv = oracle.geometry(coords, mesh.conn, ref, want_Jinv=True)
    m = fe.Mesh(_t(coords, torch.float64), _t(mesh.conn, torch.int32))
    g32 = fe.tet_geometry(ctx, m, p, flags=fe.GEOM_STORE_F32)
    ctx.check()
    wd = g32.get(fe.GEOM_WDETJ, "f32").cpu().numpy().astype(np.float64)
    ji = g32.get(fe.GEOM_JINV, "f32").cpu().numpy().astype(np.float64)
    assert np.abs(wd - wdetJ).max() <= 4e-7 * np.abs(wdetJ).max()
    # per element and point, J^-1 against its own scale
    sc = np.abs(Jinv).reshape(E, -1).max(1)[:, None, None, None]
    assert (np.abs(ji - Jinv) / sc).max() <= 4e-7
    if p > 1:
        # the bent elements really differ from the straight-edged map
        wd_straight, _, _ = oracle.geometry(mesh.coords, mesh.conn, ref)
        assert np.abs(wdetJ[:5] - wd_straight[:5]).max() > 1e-4 * np.abs(wdetJ[:5]).max()


@pytest.mark.parametrize("kind", ["laplace", "elasticity"])
def test_tensor_core_p3_matches_oracle(ctx, kind):
    """P3 Lame elasticity and the weighted Laplacian on the tensor cores (TF32x3):
    the Grundmann-Moller points ordered by weight sign, the negative ones entering
    through a negated operand copy.  Every element of a 1,201-element mesh (several
    elements per persistent CTA, a ragged last round) against the oracle, on the
    scale of the sums of absolute terms (the rule's weights alternate in sign), and
    symmetry."""
    E = 1201
    mesh = meshgen.tet_mesh(E, 3, np.random.default_rng(93))
    ref = oracle.RefTet(3, 3)
    wdetJ, G, _ = oracle.geometry(mesh.coords, mesh.conn, ref)
    aw, aG = np.abs(wdetJ), np.abs(G)
    rng = np.random.default_rng(94)
    m = fe.Mesh(_t(mesh.coords, torch.float64), _t(mesh.conn, torch.int32))
    geom = fe.tet_geometry(ctx, m, 3, flags=fe.GEOM_STORE_F32)
    if kind == "laplace":
        coef = rng.uniform(0.5, 2.0, E)
        form, mat = fe.laplace_form(weighted=True), coef
        Kref, Kabs = oracle.matrix_laplace(wdetJ, G, coef), oracle.matrix_laplace(aw, aG, coef)
    else:
        lam, mu = meshgen.lame_materials(mesh)
        form, mat = fe.elasticity_form(fe.MAT_LAME), np.stack([lam, mu], 1)
        D = oracle.lame_to_D(lam, mu)
        Kref, Kabs = oracle.matrix_elasticity(wdetJ, G, D), oracle.matrix_elasticity(aw, aG, np.abs(D))
    K = fe.eval_matrix(ctx, form, geom, [_t(mat, torch.float64), None, None], "tf32x3")
    ctx.check()
    Kg = K.cpu().numpy().astype(np.float64)
    assert Kg.shape == Kref.shape
    ek = float((np.sqrt(((Kg - Kref) ** 2).sum((1, 2))) / np.sqrt((Kabs ** 2).sum((1, 2)))).max())
    assert ek <= TOL["tf32x3"], ek
    scale = np.abs(Kabs).max()
    assert np.abs(Kg - Kg.transpose(0, 2, 1)).max() <= 10 * TOL["tf32x3"] * scale
    with pytest.raises(fe.FEError) as ei:
        fe.eval_matrix(ctx, form, geom, [_t(mat, torch.float64), None, None], "bf16x3")
    assert ei.value.status == fe.FE_ERR_UNSUPPORTED_SPEC
