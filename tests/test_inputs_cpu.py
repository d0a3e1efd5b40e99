"""The seeded synthetic inputs (meshgen) follow their stated recipe: grid layout and
numbering, the interior perturbation and its bound, the order of the draws from one
PCG64 stream per mesh, the material ranges, the smooth convection field, and the
mixed-mesh groups (sizes, orientation, shared nodes).  Valid geometry (det J > 0,
volumes) is checked with the oracle."""
import numpy as np
import pytest

import oracle
from paper_2107_04121_gb300 import meshgen


def test_structured_hex_numbering_x_fastest():
    nx, ny, nz, p = 3, 2, 2, 2
    m = meshgen.structured_hex(nx, ny, nz, p)
    NX, NY, NZ = nx * p + 1, ny * p + 1, nz * p + 1
    assert m.n_nodes == NX * NY * NZ == meshgen.grid_node_count(nx, ny, nz, p)
    assert m.conn.shape == (nx * ny * nz, (p + 1) ** 3) and m.conn.dtype == np.int32
    h = np.array([1.0 / (nx * p), 1.0 / (ny * p), 1.0 / (nz * p)])
    # node i + NX j + NX NY k sits at (i, j, k) h
    for (i, j, k) in [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (NX - 1, NY - 1, NZ - 1), (3, 2, 1)]:
        np.testing.assert_array_equal(m.coords[i + NX * j + NX * NY * k], np.array([i, j, k]) * h)
    # element ex + nx ey + nx ny ez, local node (a, b, c) -> grid node (ex p + a, ey p + b, ez p + c)
    for ex, ey, ez in [(0, 0, 0), (1, 0, 0), (2, 1, 1), (0, 1, 0)]:
        e = ex + nx * ey + nx * ny * ez
        for a, b, c in [(0, 0, 0), (2, 0, 0), (0, 2, 0), (1, 1, 2), (2, 2, 2)]:
            g = (ex * p + a) + NX * (ey * p + b) + NX * NY * (ez * p + c)
            assert m.conn[e, a + (p + 1) * b + (p + 1) ** 2 * c] == g


def test_perturbation_moves_interior_nodes_within_the_bound_only():
    n, p, a = 4, 2, 0.15
    flat = meshgen.structured_hex(n, n, n, p)
    moved = meshgen.structured_hex(n, n, n, p, a, seed=7)
    h = 1.0 / (n * p)
    d = moved.coords - flat.coords
    on_boundary = np.any((flat.coords < 1e-12) | (flat.coords > 1 - 1e-12), axis=1)
    assert np.all(d[on_boundary] == 0.0)
    assert np.all(np.abs(d[~on_boundary]) <= a * h * (1 + 1e-12))
    assert np.all(np.abs(d[~on_boundary]) > 0.0)
    # the offsets are the first draws of the mesh's stream, scaled by a h
    offs = np.random.default_rng(7).uniform(-1.0, 1.0, size=(flat.n_nodes, 3))
    np.testing.assert_allclose(d[~on_boundary], a * h * offs[~on_boundary], rtol=0, atol=1e-15)
    np.testing.assert_array_equal(meshgen.structured_hex(n, n, n, p, a, seed=7).coords, moved.coords)
    assert not np.array_equal(meshgen.structured_hex(n, n, n, p, a, seed=8).coords, moved.coords)


def test_draw_order_coordinates_then_materials_then_dofs():
    mesh, lam, mu, u = meshgen.elasticity_q2_cube(3, seed=11)
    rng = np.random.default_rng(11)
    rng.uniform(-1.0, 1.0, size=(mesh.n_nodes, 3))
    np.testing.assert_array_equal(lam, rng.uniform(0.5, 2.0, size=mesh.n_elems))
    np.testing.assert_array_equal(mu, rng.uniform(0.2, 1.0, size=mesh.n_elems))
    np.testing.assert_array_equal(u, rng.standard_normal(3 * mesh.n_nodes))
    assert lam.min() >= 0.5 and lam.max() <= 2.0 and mu.min() >= 0.2 and mu.max() <= 1.0


def test_benchmark_perturbation_gives_valid_elements_that_tile_the_cube():
    """At the metric workload's +-0.15 h every Q2 element keeps det J > 0 at its
    Gauss points, and the elements tile the unit cube (sum of w det J = 1)."""
    mesh, _, _, _ = meshgen.elasticity_q2_cube(6, seed=1)
    wdetJ, _, _ = oracle.geometry(mesh.coords, mesh.conn, oracle.RefElement(2, 3))
    assert wdetJ.min() > 0.0
    assert abs(wdetJ.sum() - 1.0) <= 1e-12


def test_convection_field_is_the_stated_smooth_field():
    mesh, u = meshgen.convect_q2_cube(4, seed=3)
    rng = np.random.default_rng(3)
    rng.uniform(-1.0, 1.0, size=(mesh.n_nodes, 3))
    amp = rng.standard_normal(3)
    x, y = mesh.coords[:, 0], mesh.coords[:, 1]
    np.testing.assert_allclose(u.reshape(-1, 3), np.sin(np.pi * x)[:, None] * np.cos(np.pi * y)[:, None] * amp,
                               rtol=0, atol=1e-15)


def test_bar_mesh_is_the_papers_n_by_1_by_1_bar():
    m = meshgen.bar_mesh(5, 2)
    assert m.n_elems == 5 and m.n_nodes == 11 * 3 * 3
    assert m.coords[:, 0].max() == 5.0 and m.coords[:, 1].max() == 1.0 and m.coords[:, 2].max() == 1.0


def test_mixed_mesh_groups_sizes_orientation_and_shared_nodes():
    groups = meshgen.mixed_mesh_groups(scale=0.002, seed=2)
    assert [g[0] for g in groups] == ["P1", "P2", "P3", "Q1", "Q2", "Q3"]
    for (name, mesh), target, n_per in zip(groups[:3], (200_000, 120_000, 40_000), (4, 10, 20)):
        p = int(name[1])
        assert mesh.n_elems == max(8, round(target * 0.002)) and mesh.nodes_per_elem == n_per
        assert mesh.conn.min() >= 0 and mesh.conn.max() < mesh.n_nodes
        # straight-sided, positively oriented tetrahedra inside the unit cube
        wdetJ, _, _ = oracle.geometry(mesh.coords, mesh.conn, oracle.RefTet(p, p))
        assert np.all(wdetJ.sum(1) > 0.0)
        assert mesh.coords.min() >= 0.0 and mesh.coords.max() <= 1.0
        # edge and face nodes are shared between neighbours: fewer nodes than slots
        if p > 1:
            assert len(np.unique(mesh.conn)) == mesh.n_nodes < mesh.n_elems * n_per
    f = 0.002 ** (1.0 / 3.0)
    for (name, mesh), shape in zip(groups[3:], ((50, 40, 30), (40, 30, 25), (20, 20, 20))):
        p = int(name[1])
        sh = tuple(max(1, int(round(n * f))) for n in shape)
        assert mesh.shape == sh and mesh.n_elems == int(np.prod(sh)) and mesh.nodes_per_elem == (p + 1) ** 3
    # the same seed gives the same meshes
    again = meshgen.mixed_mesh_groups(scale=0.002, seed=2)
    for (_, a), (_, b) in zip(groups, again):
        np.testing.assert_array_equal(a.coords, b.coords)
        np.testing.assert_array_equal(a.conn, b.conn)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_tet_lattice_nodes_x_fastest(p):
    L = meshgen._lattice(p)
    assert len(L) == (p + 1) * (p + 2) * (p + 3) // 6
    assert np.all(L.sum(1) == p) and np.all(L >= 0)
    # x fastest: the first p + 1 nodes run along the x edge (i = 0 .. p, j = k = 0)
    np.testing.assert_array_equal(L[:p + 1, 1], np.arange(p + 1))
    assert np.all(L[:p + 1, 2:] == 0)
