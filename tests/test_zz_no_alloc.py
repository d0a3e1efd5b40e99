"""fe_assemble_vector_noalloc: assembly for callers that cannot allocate device memory.

Such callers (an application whose device memory belongs to its own allocator
or budget, a real-time loop where an allocation's implicit synchronisation would
stall other streams, a callback inside a framework step that forbids
allocation) use the entry point that keeps its workspace in the library's fixed
device array.  Its results must equal those of the allocating path
(fe_assembly_create + fe_assemble_vector), which the other tests pin to the
oracle bit for bit in FP64; here they are compared exactly, on two calls in a
row whose meshes differ, so that stale workspace contents from the first call
would show in the second.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2107_04121_gb300 import fe, meshgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _mesh(shape, p, seed):
    mesh = meshgen.structured_hex(*shape, p, 0.1, seed)
    coords = torch.from_numpy(mesh.coords).cuda()
    conn = torch.from_numpy(mesh.conn).cuda()
    return mesh, fe.Mesh(coords, conn)


@pytest.mark.parametrize("prec,flags", [("f64", 0), ("f32", fe.ASSEMBLE_COMPENSATED), ("f32", 0)])
def test_noalloc_assembly_matches_allocating_path_twice(libfe, prec, flags):
    ctx = fe.Context(0)
    dt = torch.float64 if prec == "f64" else torch.float32
    rng = np.random.default_rng(71)
    # first a larger mesh, then a smaller one: leftovers of call 1 must not leak into call 2
    for shape, p, ncomp in [((6, 5, 4), 2, 3), ((3, 4, 2), 1, 1)]:
        mesh, m = _mesh(shape, p, int(rng.integers(1 << 30)))
        r = torch.from_numpy(rng.standard_normal((mesh.n_elems, ncomp * mesh.nodes_per_elem))).to("cuda", dt)
        want = fe.assemble_vector(ctx, fe.assembly_create(ctx, m), ncomp, r, prec, flags=flags)
        out = torch.full((mesh.n_nodes * ncomp,), float("nan"), dtype=dt, device="cuda")
        got = fe.assemble_vector_noalloc(ctx, m, ncomp, r, out, prec, flags=flags)
        ctx.check()
        assert torch.equal(got, want)
        # accumulate into the previous result
        fe.assemble_vector_noalloc(ctx, m, ncomp, r, out, prec, flags=flags | fe.ASSEMBLE_ACCUMULATE)
        want2 = fe.assemble_vector(ctx, fe.assembly_create(ctx, m), ncomp, r, prec, out=want.clone(),
                                   flags=flags | fe.ASSEMBLE_ACCUMULATE)
        ctx.check()
        assert torch.equal(out, want2)
    ctx.close()


def test_noalloc_rejects_meshes_beyond_its_workspace(libfe):
    ctx = fe.Context(0)
    mesh, m = _mesh((2, 2, 2), 1, 0)
    big = fe._Mesh(m.struct.coords, (1 << 19) + 1, m.struct.conn, m.struct.n_elems, m.struct.nodes_per_elem)
    r = torch.zeros((mesh.n_elems, 8), dtype=torch.float64, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    st = fe.load_library().fe_assemble_vector_noalloc(ctx.handle, big, 1, r.data_ptr(), fe.F64, out.data_ptr(), 0,
                                                      None)
    assert st == fe.FE_ERR_SHAPE
    assert b"524288" in fe.load_library().fe_last_error_message()
    ctx.check()
    ctx.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_noalloc_reports_out_of_range_nodes_and_assembles_the_rest(libfe, prec):
    """A node index outside the mesh is reported on the device (FE_ERR_SHAPE with
    the element index, read by fe_get_status) and that incidence is skipped: every
    global entry equals the allocating path's on the valid mesh with that
    incidence's contributions set to zero."""
    ctx = fe.Context(0)
    dt = torch.float64 if prec == "f64" else torch.float32
    mesh, m = _mesh((3, 3, 2), 1, 5)
    bad_e, bad_a = 7, 2
    conn = mesh.conn.copy()
    conn[bad_e, bad_a] = mesh.n_nodes + 11
    m_bad = fe.Mesh(m.coords, torch.from_numpy(conn).cuda())
    rng = np.random.default_rng(72)
    N = mesh.nodes_per_elem
    r = torch.from_numpy(rng.standard_normal((mesh.n_elems, 3 * N))).to("cuda", dt)
    out = torch.full((mesh.n_nodes * 3,), float("nan"), dtype=dt, device="cuda")
    fe.assemble_vector_noalloc(ctx, m_bad, 3, r, out, prec, flags=fe.ASSEMBLE_COMPENSATED if prec == "f32" else 0)
    st, elem = ctx.status()
    assert st == fe.FE_ERR_SHAPE and elem == bad_e
    r0 = r.clone()
    r0[bad_e, bad_a::N] = 0  # the skipped incidence, all three components
    want = fe.assemble_vector(ctx, fe.assembly_create(ctx, m), 3, r0, prec,
                              flags=fe.ASSEMBLE_COMPENSATED if prec == "f32" else 0)
    ctx.check()
    assert torch.equal(out, want)
    ctx.close()
