"""GPU parity of the batched matrix evaluation (fe_batch_*, both schedules:
persistent class kernels and one launch per item) on a scaled-down mixed mesh:
P1-P3 tetrahedra and Q1-Q3 hexahedra with the weighted Laplacian, weighted mass
and Lame elasticity, against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2107_04121_gb300 import fe, meshgen
from tests.parity import TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FORMS = ("laplace", "mass", "elasticity")


@pytest.fixture(scope="module")
def ctx(libfe):
    c = fe.Context(0)
    yield c
    c.close()


def _t(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)


class Group:
    def __init__(self, ctx, name, mesh):
        self.name, self.mesh = name, mesh
        self.tet = name.startswith("P")
        p = int(name[1])
        self.ref = oracle.RefTet(p, p) if self.tet else oracle.RefElement(p, p + 1)
        self.coords = _t(mesh.coords, torch.float64)
        self.m = fe.Mesh(self.coords, _t(mesh.conn, torch.int32))
        flags = fe.GEOM_STORE_F32
        self.geom = fe.tet_geometry(ctx, self.m, p, flags=flags) if self.tet else \
            fe.hex_geometry(ctx, self.m, p, p + 1, flags=flags)
        rng = np.random.default_rng(90 + p + (10 if self.tet else 0))
        E = mesh.n_elems
        self.coef = rng.uniform(0.5, 2.0, E)
        self.lam = rng.uniform(0.5, 2.0, E)
        self.mu = rng.uniform(0.2, 1.0, E)

    def material(self, form):
        if form == "elasticity":
            return _t(np.stack([self.lam, self.mu], 1), torch.float64)
        return _t(self.coef, torch.float64)

    def reference(self, form, coords=None):
        """Oracle matrices and the sums of absolute terms (the error scale)."""
        wdetJ, G, _ = oracle.geometry(self.mesh.coords if coords is None else coords, self.mesh.conn, self.ref)
        aw, aG = np.abs(wdetJ), np.abs(G)
        if form == "laplace":
            return oracle.matrix_laplace(wdetJ, G, self.coef), oracle.matrix_laplace(aw, aG, self.coef)
        if form == "mass":
            return (oracle.matrix_mass(wdetJ, self.ref.phi, 1, self.coef),
                    oracle.matrix_mass(aw, np.abs(self.ref.phi), 1, self.coef))
        D = oracle.lame_to_D(self.lam, self.mu)
        return oracle.matrix_elasticity(wdetJ, G, D), oracle.matrix_elasticity(aw, aG, np.abs(D))


def _form(name):
    if name == "laplace":
        return fe.laplace_form(weighted=True)
    if name == "mass":
        return fe.mass_form(1, weighted=True)
    return fe.elasticity_form(fe.MAT_LAME)


def _err(K, ref, tet):
    """max_e ||K_e - K_ref||_F over ||K_ref||_F on hexahedra (Gauss weights are
    positive); over the Frobenius norm of the sums of absolute terms on tetrahedra,
    whose Grundmann-Moeller weights alternate in sign, so that entries come out much
    smaller than the terms summed into them."""
    Kref, Kabs = ref
    Kg = K.cpu().numpy().astype(np.float64)
    scale = Kabs if tet else Kref
    return float((np.sqrt(((Kg - Kref) ** 2).sum((1, 2))) / np.sqrt((scale ** 2).sum((1, 2)))).max())


@pytest.fixture(scope="module")
def groups(ctx):
    return [Group(ctx, n, m) for n, m in meshgen.mixed_mesh_groups(scale=0.002, seed=2)]


def _items(groups):
    items, keys = [], []
    for g in groups:
        for f in FORMS:
            items.append((g.geom, _form(f), g.material(f), None))
            keys.append((g, f))
    return items, keys


@pytest.mark.parametrize("flags", [0, fe.BATCH_AUTOTUNE | fe.BATCH_GRAPH | fe.BATCH_GEOMETRY,
                                   fe.BATCH_PERSISTENT | fe.BATCH_AUTOTUNE | fe.BATCH_GRAPH,
                                   fe.BATCH_LAUNCHES, fe.BATCH_LAUNCHES | fe.BATCH_GRAPH | fe.BATCH_GEOMETRY])
def test_batch_matches_oracle(ctx, groups, flags):
    items, keys = _items(groups)
    b = fe.Batch(ctx, items, flags)
    outs = b.run()
    ctx.check()
    for k, ((g, f), K) in enumerate(zip(keys, outs)):
        e = _err(K, g.reference(f), g.tet)
        assert e <= TOL["f32"], (g.name, f, e, b.describe(k))
    b.free()


def test_batch_runs_are_reproducible_and_graph_equals_eager(ctx, groups):
    items, keys = _items(groups)
    eager = fe.Batch(ctx, items, 0)
    first = [K.clone() for K in eager.run()]
    again = eager.run()
    items2 = [(g, f, m, None) for g, f, m, _ in items]
    graph = fe.Batch(ctx, items2, fe.BATCH_GRAPH)
    g_out = graph.run()
    ctx.check()
    for a, b2, c in zip(first, again, g_out):
        assert torch.equal(a, b2)
        assert torch.equal(a, c)  # same configurations (no autotuning): identical results


def test_batch_schedules(ctx, groups):
    """The schedule flags are honoured, autotuning picks one of the two, and the
    per-item schedule is reproducible, equal in a graph and eagerly, and agrees
    with the persistent one to float32 rounding."""
    items, keys = _items(groups)
    fresh = lambda: [(g, f, m, None) for g, f, m, _ in items]
    assert fe.Batch(ctx, fresh(), 0).schedule() == "persistent"
    assert fe.Batch(ctx, fresh(), fe.BATCH_PERSISTENT | fe.BATCH_AUTOTUNE).schedule() == "persistent"
    assert fe.Batch(ctx, fresh(), fe.BATCH_AUTOTUNE).schedule() in ("persistent", "launches")
    with pytest.raises(fe.FEError) as ei:
        fe.Batch(ctx, fresh(), fe.BATCH_PERSISTENT | fe.BATCH_LAUNCHES)
    assert ei.value.status == fe.FE_ERR_INVALID_ARG
    per_item = fe.Batch(ctx, fresh(), fe.BATCH_LAUNCHES)
    assert per_item.schedule() == "launches"
    first = [K.clone() for K in per_item.run()]
    again = per_item.run()
    graph = fe.Batch(ctx, fresh(), fe.BATCH_LAUNCHES | fe.BATCH_GRAPH)
    g_out = graph.run()
    persistent = fe.Batch(ctx, fresh(), 0).run()
    ctx.check()
    for (g, f), a, b2, c, p in zip(keys, first, again, g_out, persistent):
        assert torch.equal(a, b2) and torch.equal(a, c), (g.name, f)
        scale = float(p.abs().max())
        assert float((a - p).abs().max()) <= 1e-5 * scale, (g.name, f)


@pytest.mark.parametrize("schedule", [fe.BATCH_PERSISTENT, fe.BATCH_LAUNCHES])
def test_batch_geometry_flag_follows_moved_nodes(ctx, groups, schedule):
    g = groups[4]  # Q2 hexahedra
    items = [(g.geom, _form("elasticity"), g.material("elasticity"), None)]
    b = fe.Batch(ctx, items, fe.BATCH_GEOMETRY | fe.BATCH_GRAPH | schedule)
    X0 = g.coords.clone()
    rng = np.random.default_rng(3)
    moved = g.mesh.coords.copy()
    interior = np.all((moved > 1e-9) & (moved < 1 - 1e-9), axis=1)
    h = 1.0 / (2 * np.array(g.mesh.shape))
    moved[interior] += 0.05 * rng.uniform(-1, 1, (interior.sum(), 3)) * h
    g.coords.copy_(_t(moved, torch.float64))
    (K,) = b.run()
    ctx.check()
    assert _err(K, g.reference("elasticity", moved), g.tet) <= TOL["f32"]
    g.coords.copy_(X0)
    g.geom.update()
    ctx.check()


def test_batch_contraction_path_is_reported(ctx, groups):
    """The per-item schedule may run the Q2 elasticity and Laplace items, the Q3
    elasticity, Laplace and mass items and the P3 elasticity and Laplace items on
    the tensor cores (TF32x3 Gram), and an elasticity item with the Laplace item of
    its geometry on shared Gram blocks; every other item, and every item of the
    persistent schedule, on the CUDA cores; every item matches the oracle."""
    items, keys = _items(groups)
    b = fe.Batch(ctx, items, fe.BATCH_AUTOTUNE | fe.BATCH_LAUNCHES)
    outs = b.run()
    ctx.check()
    for k, ((g, f), K) in enumerate(zip(keys, outs)):
        path = b.describe(k)["path"]
        if path.startswith("tensor"):
            assert (g.name, f) in (("Q2", "elasticity"), ("Q2", "laplace"), ("Q3", "elasticity"),
                                   ("Q3", "laplace"), ("Q3", "mass"), ("P3", "elasticity"), ("P3", "laplace"))
        if "shared" in path:
            assert f in ("elasticity", "laplace")
        assert _err(K, g.reference(f), g.tet) <= TOL["f32"], (g.name, f, path)
    b.free()
    bp = fe.Batch(ctx, items, fe.BATCH_AUTOTUNE | fe.BATCH_PERSISTENT)
    assert all(bp.describe(k)["path"].startswith("cuda") for k in range(len(keys)))
    bp.free()


def test_batch_shared_gram_pairs(ctx, groups):
    """BATCH_SHARED_GRAM: each Lame elasticity item and the weighted Laplacian item
    of its geometry come from one launch (the Laplacian as c sum_j A_jj of the
    elasticity's Gram blocks; tensor cores for Q2 and Q3, CUDA cores for the other
    groups); both match the oracle on every group (several
    elements per CTA, ragged last groups), the mass items keep their own kernels,
    every output is written (the buffers start as NaN), and runs are reproducible,
    eagerly and in a graph."""
    items, keys = _items(groups)

    def fresh():
        out = []
        for (gm, f, m, _), (g, fname) in zip(items, keys):
            n = g.mesh.nodes_per_elem * (3 if fname == "elasticity" else 1)
            out.append((gm, f, m, torch.full((g.mesh.n_elems, n, n), float("nan"), device="cuda")))
        return out

    b = fe.Batch(ctx, fresh(), fe.BATCH_LAUNCHES | fe.BATCH_SHARED_GRAM)
    outs = b.run()
    ctx.check()
    for k, ((g, f), K) in enumerate(zip(keys, outs)):
        path = b.describe(k)["path"]
        assert ("shared" in path) == (f != "mass"), (g.name, f, path)
        if f != "mass":  # shared tensor-core kernels exist for Q2 and Q3 hexahedra
            assert path.startswith("tensor") == (g.name in ("Q2", "Q3")), (g.name, f, path)
        e = _err(K, g.reference(f), g.tet)
        assert e <= TOL["f32"], (g.name, f, e)
    first = [K.clone() for K in outs]
    again = b.run()
    bg = fe.Batch(ctx, fresh(), fe.BATCH_LAUNCHES | fe.BATCH_SHARED_GRAM | fe.BATCH_GRAPH)
    g_out = bg.run()
    ctx.check()
    for a, c, d in zip(first, again, g_out):
        assert torch.equal(a, c)
        assert torch.equal(a, d)
    b.free()
    bg.free()


def test_batch_shared_gram_unweighted_laplacian(ctx, groups):
    """A shared-Gram pair whose Laplacian has no coefficient (c = 1 on every element)
    on every group, against the oracle."""
    items, keys = [], []
    for g in groups:
        items.append((g.geom, _form("elasticity"), g.material("elasticity"), None))
        items.append((g.geom, fe.laplace_form(weighted=False), None, None))
        keys += [(g, "elasticity"), (g, "laplace")]
    b = fe.Batch(ctx, items, fe.BATCH_LAUNCHES | fe.BATCH_SHARED_GRAM)
    outs = b.run()
    ctx.check()
    for k, ((g, f), K) in enumerate(zip(keys, outs)):
        assert "shared" in b.describe(k)["path"], (g.name, f)
        if f == "elasticity":
            ref = g.reference(f)
        else:
            wdetJ, G, _ = oracle.geometry(g.mesh.coords, g.mesh.conn, g.ref)
            one = np.ones(g.mesh.n_elems)
            ref = (oracle.matrix_laplace(wdetJ, G, one), oracle.matrix_laplace(np.abs(wdetJ), np.abs(G), one))
        e = _err(K, ref, g.tet)
        assert e <= TOL["f32"], (g.name, f, e)
    b.free()


def test_batch_shared_gram_tensor_cores_several_elements_per_cta(ctx):
    """The tensor-core shared-Gram launches (Q2: k_matrix_tc pair form, two CTAs per
    SM; Q3: k_matrix_tc64 pair mode, one CTA per SM) on meshes larger than their
    persistent grids, so that each CTA computes several elements and reuses its
    Laplacian staging: every element of both outputs against the oracle."""
    for p, dims, seed in ((2, (14, 14, 12), 71), (3, (8, 8, 6), 72)):
        mesh = meshgen.structured_hex(*dims, p, 0.1, seed)
        g = Group.__new__(Group)
        g.name, g.mesh, g.tet = "Q%d" % p, mesh, False
        g.ref = oracle.RefElement(p, p + 1)
        g.coords = _t(mesh.coords, torch.float64)
        g.m = fe.Mesh(g.coords, _t(mesh.conn, torch.int32))
        g.geom = fe.hex_geometry(ctx, g.m, p, p + 1, flags=fe.GEOM_STORE_F32)
        rng = np.random.default_rng(seed)
        E = mesh.n_elems
        g.coef, g.lam, g.mu = rng.uniform(0.5, 2.0, E), rng.uniform(0.5, 2.0, E), rng.uniform(0.2, 1.0, E)
        items = [(g.geom, _form(f), g.material(f), None) for f in ("elasticity", "laplace")]
        b = fe.Batch(ctx, items, fe.BATCH_LAUNCHES | fe.BATCH_SHARED_GRAM)
        outs = b.run()
        ctx.check()
        for k, f in enumerate(("elasticity", "laplace")):
            assert b.describe(k)["path"].startswith("tensor") and "shared" in b.describe(k)["path"]
            e = _err(outs[k], g.reference(f), False)
            assert e <= TOL["tf32x3"], (p, f, e)
        b.free()


def test_batch_autotune_choice_is_a_candidate(ctx, groups):
    items, keys = _items(groups)
    b = fe.Batch(ctx, items, fe.BATCH_AUTOTUNE)
    for k, (g, f) in enumerate(keys):
        d = b.describe(k)
        N = g.mesh.nodes_per_elem
        assert N % d["tile"] == 0 and d["elems_per_chunk"] >= 1
    with pytest.raises(fe.FEError):
        b.describe(len(keys))


def test_batch_rejections(ctx, groups):
    g = groups[4]
    with pytest.raises(fe.FEError) as ei:
        fe.Batch(ctx, [(g.geom, fe.convect_form(), None, None)])
    assert ei.value.status == fe.FE_ERR_UNSUPPORTED_SPEC
    g64 = fe.hex_geometry(ctx, g.m, 2, 3, flags=fe.GEOM_STORE_F64)
    with pytest.raises(fe.FEError) as ei:
        fe.Batch(ctx, [(g64, _form("laplace"), g.material("laplace"), None)])
    assert ei.value.status == fe.FE_ERR_INVALID_ARG
    with pytest.raises(fe.FEError) as ei:
        fe.Batch(ctx, [(g.geom, _form("elasticity"), None, None)])
    assert ei.value.status == fe.FE_ERR_INVALID_ARG
