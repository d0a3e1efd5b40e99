"""The benchmark workloads at their full sizes, in the launch configurations the
benchmark times, against the oracle on sampled elements (first, last and seeded
ones, each computed by the oracle on its own) and through properties that hold at
any size: the Q2 elasticity metric workload (48^3), the convection workload (64^3)
and the mixed batch (458,000 elements)."""
import numpy as np
import pytest

import oracle
from paper_2107_04121_gb300 import fe, meshgen
from tests.parity import TOL, rel_matrix_error, rel_vector_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(libfe):
    c = fe.Context(0)
    yield c
    c.close()


def _t(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)


def _sample(E, seed, k=62):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([[0, E - 1], rng.choice(E, min(k, E), replace=False)]))


def test_metric_workload_full_size(ctx):
    """48^3 Q2 elasticity (110,592 elements), the benchmark's step: the BF16x3
    tensor-core kernel computing the deferred FP64 geometry, the FP32 residual on
    its stored copy, compensated assembly."""
    mesh, lam, mu, u = meshgen.elasticity_q2_cube(48, seed=1)
    E = mesh.n_elems
    m = fe.Mesh(_t(mesh.coords, torch.float64), _t(mesh.conn, torch.int32))
    geom = fe.hex_geometry(ctx, m, 2, 3, flags=fe.GEOM_STORE_F32 | fe.GEOM_DEFERRED)
    form = fe.elasticity_form()
    mat = _t(np.stack([lam, mu], 1), torch.float64)
    u32 = _t(u, torch.float32)
    geom.update()
    K = fe.eval_matrix(ctx, form, geom, [mat, None, None], "bf16x3")
    r = fe.eval_residual(ctx, form, geom, [mat, None, u32], "bf16x3")
    g = fe.assemble_vector(ctx, fe.assembly_create(ctx, m), 3, r, "f32", flags=fe.ASSEMBLE_COMPENSATED)
    ctx.check()
    idx = _sample(E, 7)
    conn = mesh.conn[idx]
    wdetJ, G, _ = oracle.geometry(mesh.coords, conn, oracle.RefElement(2, 3))
    D = oracle.lame_to_D(lam[idx], mu[idx])
    it = torch.from_numpy(idx).cuda()
    Ks = K.index_select(0, it).cpu().numpy()
    rs = r.index_select(0, it).cpu().numpy()
    assert rel_matrix_error(Ks, oracle.matrix_elasticity(wdetJ, G, D)) <= TOL["bf16x3"]
    assert rel_vector_error(rs, oracle.residual_elasticity(conn, wdetJ, G, D, u)) <= TOL["f32"]
    # properties at any size: K_e symmetric, r_e = K_e u_e (the BF16x3 K against
    # the float32 residual), the assembly of r_e (float64 on the host) within the
    # compensated sum's bound, and no non-finite value anywhere
    assert np.abs(Ks - Ks.transpose(0, 2, 1)).max() <= 1e-5 * np.abs(Ks).max()
    ue = u.reshape(-1, 3)[conn].transpose(0, 2, 1).reshape(len(idx), -1)  # component-major (3 N)
    assert rel_vector_error(np.einsum("eij,ej->ei", Ks.astype(np.float64), ue), rs) <= 1e-5
    rh = r.cpu().numpy().astype(np.float64)
    want = oracle.assemble(mesh.conn, rh, mesh.n_nodes, 3)
    sumabs = oracle.assemble(mesh.conn, np.abs(rh), mesh.n_nodes, 3)
    assert np.all(np.abs(g.cpu().numpy() - want) <= 2.0 ** -24 * np.abs(want) + 64 * 2.0 ** -48 * sumabs)
    assert bool(torch.isfinite(K).all()) and bool(torch.isfinite(r).all())


def _elementwise_rel_errors(Kg, Kref):
    """||K_e - K_e^ref||_F / ||K_e^ref||_F for every element of a chunk."""
    d = Kg - Kref
    return np.sqrt(np.einsum("eij,eij->e", d, d) / np.einsum("eij,eij->e", Kref, Kref))


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_metric_workload_every_element(ctx, prec):
    """48^3 Q2 elasticity, the benchmark's step (the split-precision tensor-core
    kernel computing the deferred FP64 geometry, the FP32 residual on its stored
    copy): all 110,592 element matrices against the oracle, each within the 1e-5 bar
    (max_e ||K_e - K_ref||_F / ||K_ref||_F), and the residual array within 1e-5
    (||r - r_ref||_2 / ||r_ref||_2), in chunks of 13,824 elements."""
    mesh, lam, mu, u = meshgen.elasticity_q2_cube(48, seed=1)
    E = mesh.n_elems
    m = fe.Mesh(_t(mesh.coords, torch.float64), _t(mesh.conn, torch.int32))
    geom = fe.hex_geometry(ctx, m, 2, 3, flags=fe.GEOM_STORE_F32 | fe.GEOM_DEFERRED)
    form = fe.elasticity_form()
    mat = _t(np.stack([lam, mu], 1), torch.float64)
    geom.update()
    K = fe.eval_matrix(ctx, form, geom, [mat, None, None], prec)
    r = fe.eval_residual(ctx, form, geom, [mat, None, _t(u, torch.float32)], prec)
    ctx.check()
    ref = oracle.RefElement(2, 3)
    worst, r_num, r_den = 0.0, 0.0, 0.0
    chunk = 13824
    for c0 in range(0, E, chunk):
        sl = slice(c0, min(E, c0 + chunk))
        conn = np.ascontiguousarray(mesh.conn[sl])
        wdetJ, G, _ = oracle.geometry(mesh.coords, conn, ref)
        D = oracle.lame_to_D(lam[sl], mu[sl])
        Kref = oracle.matrix_elasticity(wdetJ, G, D)
        errs = _elementwise_rel_errors(K[sl].double().cpu().numpy(), Kref)
        worst = max(worst, float(errs.max()))
        rref = oracle.residual_elasticity(conn, wdetJ, G, D, u)
        dr = r[sl].double().cpu().numpy() - rref
        r_num += float((dr * dr).sum())
        r_den += float((rref * rref).sum())
        del Kref, errs
    print("%s: max over %d elements of the K_e error %.3e; residual %.3e" % (prec, E, worst, np.sqrt(r_num / r_den)))
    assert worst <= TOL[prec], worst
    assert np.sqrt(r_num / r_den) <= TOL["f32"]


def test_convection_workload_full_size(ctx):
    """64^3 Q2 convection (262,144 elements): FP32 K_e(u) and r_e(u), the residual
    computing the deferred geometry."""
    mesh, u = meshgen.convect_q2_cube(64, seed=3)
    E = mesh.n_elems
    m = fe.Mesh(_t(mesh.coords, torch.float64), _t(mesh.conn, torch.int32))
    geom = fe.hex_geometry(ctx, m, 2, 3, flags=fe.GEOM_STORE_F32 | fe.GEOM_DEFERRED)
    form = fe.convect_form()
    u32 = _t(u, torch.float32)
    geom.update()
    r = fe.eval_residual(ctx, form, geom, [None, u32, u32], "f32")
    K = fe.eval_matrix(ctx, form, geom, [None, u32, u32], "f32")
    ctx.check()
    idx = _sample(E, 9)
    conn = mesh.conn[idx]
    ref = oracle.RefElement(2, 3)
    wdetJ, G, _ = oracle.geometry(mesh.coords, conn, ref)
    it = torch.from_numpy(idx).cuda()
    Kref = oracle.matrix_convect(conn, wdetJ, ref.phi, G, u)
    rref = oracle.residual_convect(conn, wdetJ, ref.phi, G, u)
    assert rel_matrix_error(K.index_select(0, it).cpu().numpy(), Kref) <= TOL["f32"]
    assert rel_vector_error(r.index_select(0, it).cpu().numpy(), rref) <= TOL["f32"]
    assert bool(torch.isfinite(K).all()) and bool(torch.isfinite(r).all())


def test_mixed_batch_full_size(ctx):
    """P1/P2/P3 tetrahedra 200k/120k/40k and Q1/Q2/Q3 hexahedra 60k/30k/8k, the three
    forms per group in one autotuned, graph-captured batch with its geometry: sampled
    elements of every item against the oracle (on tetrahedra the errors are scaled by
    the sums of absolute terms, as the Grundmann-Moeller weights alternate in sign;
    on hexahedra by ||K_ref||_F)."""
    groups, items, keys = [], [], []
    for name, mesh in meshgen.mixed_mesh_groups(1.0, seed=2):
        p = int(name[1])
        tet = name[0] == "P"
        ref = oracle.RefTet(p, p) if tet else oracle.RefElement(p, p + 1)
        m = fe.Mesh(_t(mesh.coords, torch.float64), _t(mesh.conn, torch.int32))
        geom = fe.tet_geometry(ctx, m, p, flags=fe.GEOM_STORE_F32) if tet else \
            fe.hex_geometry(ctx, m, p, p + 1, flags=fe.GEOM_STORE_F32)
        rng = np.random.default_rng(200 + p + (10 if tet else 0))
        E = mesh.n_elems
        coef, lam, mu = rng.uniform(0.5, 2.0, E), rng.uniform(0.5, 2.0, E), rng.uniform(0.2, 1.0, E)
        groups.append((name, mesh, m, geom, ref, coef, lam, mu))
        for f in ("laplace", "mass", "elasticity"):
            form = fe.laplace_form(weighted=True) if f == "laplace" else (
                fe.mass_form(1, weighted=True) if f == "mass" else fe.elasticity_form(fe.MAT_LAME))
            mat = _t(np.stack([lam, mu], 1), torch.float64) if f == "elasticity" else _t(coef, torch.float64)
            items.append((geom, form, mat, None))
            keys.append((len(groups) - 1, f))
    b = fe.Batch(ctx, items, fe.BATCH_AUTOTUNE | fe.BATCH_GRAPH | fe.BATCH_GEOMETRY)
    outs = b.run()
    ctx.check()
    for (gi, f), K in zip(keys, outs):
        name, mesh, m, geom, ref, coef, lam, mu = groups[gi]
        idx = _sample(mesh.n_elems, 11, 14)
        conn = mesh.conn[idx]
        wdetJ, G, _ = oracle.geometry(mesh.coords, conn, ref)
        aw, aG = np.abs(wdetJ), np.abs(G)
        if f == "laplace":
            Kref, Kabs = oracle.matrix_laplace(wdetJ, G, coef[idx]), oracle.matrix_laplace(aw, aG, coef[idx])
        elif f == "mass":
            Kref = oracle.matrix_mass(wdetJ, ref.phi, 1, coef[idx])
            Kabs = oracle.matrix_mass(aw, np.abs(ref.phi), 1, coef[idx])
        else:
            D = oracle.lame_to_D(lam[idx], mu[idx])
            Kref, Kabs = oracle.matrix_elasticity(wdetJ, G, D), oracle.matrix_elasticity(aw, aG, np.abs(D))
        Kg = K.index_select(0, torch.from_numpy(idx).cuda()).cpu().numpy().astype(np.float64)
        scale = Kabs if name[0] == "P" else Kref  # Gauss weights on hexahedra are positive
        err = float((np.sqrt(((Kg - Kref) ** 2).sum((1, 2))) / np.sqrt((scale ** 2).sum((1, 2)))).max())
        assert err <= TOL["f32"], (name, f, err)
    b.free()


def test_element_matrices_past_2_31_entries(ctx):
    """70^3 Q2 elasticity (343,000 elements): K holds 2.25e9 entries; element
    327,310 straddles entry 2^31 and the later ones start past it (byte 2^33 in
    float32, 2^34 in FP64);
    the benchmark's step (the BF16x3 tensor-core kernel computing the deferred
    geometry, the residual, compensated assembly), the float32 CUDA-core and the
    FP64 matrix kernels, sampled on both sides of that boundary against the oracle."""
    mesh, lam, mu, u = meshgen.elasticity_q2_cube(70, seed=5)
    E = mesh.n_elems
    first_past = -(-(2 ** 31) // (81 * 81))  # first element starting past entry 2^31
    assert E * 81 * 81 > 2 ** 31 and first_past < E
    rng = np.random.default_rng(13)
    idx = np.unique(np.concatenate([[0, first_past - 2, first_past - 1, first_past, E - 1],
                                    rng.integers(first_past, E, 24)]))
    m = fe.Mesh(_t(mesh.coords, torch.float64), _t(mesh.conn, torch.int32))
    form = fe.elasticity_form()
    mat = _t(np.stack([lam, mu], 1), torch.float64)
    u32 = _t(u, torch.float32)
    conn = mesh.conn[idx]
    wdetJ, G, _ = oracle.geometry(mesh.coords, conn, oracle.RefElement(2, 3))
    D = oracle.lame_to_D(lam[idx], mu[idx])
    Kref = oracle.matrix_elasticity(wdetJ, G, D)
    it = torch.from_numpy(idx).cuda()

    gd = fe.hex_geometry(ctx, m, 2, 3, flags=fe.GEOM_STORE_F32 | fe.GEOM_DEFERRED)
    gd.update()
    K = fe.eval_matrix(ctx, form, gd, [mat, None, None], "bf16x3")
    r = fe.eval_residual(ctx, form, gd, [mat, None, u32], "bf16x3")
    g = fe.assemble_vector(ctx, fe.assembly_create(ctx, m), 3, r, "f32", flags=fe.ASSEMBLE_COMPENSATED)
    ctx.check()
    assert rel_matrix_error(K.index_select(0, it).cpu().numpy(), Kref) <= TOL["bf16x3"]
    assert rel_vector_error(r.index_select(0, it).cpu().numpy(),
                            oracle.residual_elasticity(conn, wdetJ, G, D, u)) <= TOL["f32"]
    rh = r.cpu().numpy().astype(np.float64)
    want = oracle.assemble(mesh.conn, rh, mesh.n_nodes, 3)
    sumabs = oracle.assemble(mesh.conn, np.abs(rh), mesh.n_nodes, 3)
    assert np.all(np.abs(g.cpu().numpy() - want) <= 2.0 ** -24 * np.abs(want) + 64 * 2.0 ** -48 * sumabs)
    del r, g, gd

    gs = fe.hex_geometry(ctx, m, 2, 3, flags=fe.GEOM_STORE_F64 | fe.GEOM_STORE_F32)
    fe.eval_matrix(ctx, form, gs, [mat, None, None], "f32", out=K)
    ctx.check()
    assert rel_matrix_error(K.index_select(0, it).cpu().numpy(), Kref) <= TOL["f32"]
    del K
    K64 = fe.eval_matrix(ctx, form, gs, [mat, None, None], "f64")
    ctx.check()
    assert rel_matrix_error(K64.index_select(0, it).cpu().numpy(), Kref) <= TOL["f64"]
