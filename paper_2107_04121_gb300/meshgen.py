"""Seeded synthetic inputs: structured hexahedral meshes, materials and DOF vectors.

This module only draws random numbers and lays out mesh topology; it holds none
of the finite element arithmetic (no basis, quadrature, geometry mapping or
form).  The same generators feed both the CUDA library and the FP64 oracle.

Conventions (the paper, Sec. 6, uses a 1D bar of n x 1 x 1 hexahedra whose
element-level work equals that of any other hex mesh of the same size):
  * domain [0, Lx] x [0, Ly] x [0, Lz], nx * ny * nz hexahedra of order p;
  * global nodes on the (nx p + 1) x (ny p + 1) x (nz p + 1) equispaced grid,
    numbered x fastest;
  * element (ex, ey, ez) has index ex + nx ey + nx ny ez, local node (i, j, k)
    (x fastest, i + (p+1) j + (p+1)^2 k) maps to grid node (ex p + i, ey p + j, ez p + k);
  * interior nodes (not on the boundary of the box) are moved by a uniform
    random offset in [-a h, a h] per coordinate, h = node spacing on that axis;
  * one numpy PCG64 stream per mesh, drawn in this order: the coordinate
    offsets (n_nodes, 3) for all nodes (boundary draws discarded), then the
    materials, then the DOF vector.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class HexMesh:
    coords: np.ndarray  # (n_nodes, 3) float64
    conn: np.ndarray  # (n_elems, (p+1)^3) int32
    order: int
    shape: tuple  # (nx, ny, nz)
    rng: np.random.Generator  # positioned after the coordinate draws

    @property
    def n_nodes(self) -> int:
        return self.coords.shape[0]

    @property
    def n_elems(self) -> int:
        return self.conn.shape[0]

    @property
    def nodes_per_elem(self) -> int:
        return self.conn.shape[1]


def grid_node_count(nx: int, ny: int, nz: int, p: int) -> int:
    return (nx * p + 1) * (ny * p + 1) * (nz * p + 1)


def structured_hex(nx: int, ny: int, nz: int, p: int = 1, perturb: float = 0.0, seed: int = 0,
                   lengths=(1.0, 1.0, 1.0)) -> HexMesh:
    """Structured order-p hexahedral mesh with interior nodes perturbed."""
    NX, NY, NZ = nx * p + 1, ny * p + 1, nz * p + 1
    ix, iy, iz = np.meshgrid(np.arange(NX), np.arange(NY), np.arange(NZ), indexing="ij")
    # x fastest: flatten in (z, y, x) order
    ix = ix.transpose(2, 1, 0).ravel()
    iy = iy.transpose(2, 1, 0).ravel()
    iz = iz.transpose(2, 1, 0).ravel()
    h = np.array([lengths[0] / (nx * p), lengths[1] / (ny * p), lengths[2] / (nz * p)])
    coords = np.stack([ix * h[0], iy * h[1], iz * h[2]], axis=1).astype(np.float64)
    rng = np.random.default_rng(seed)
    offs = rng.uniform(-1.0, 1.0, size=(coords.shape[0], 3))
    if perturb != 0.0:
        interior = (ix > 0) & (ix < NX - 1) & (iy > 0) & (iy < NY - 1) & (iz > 0) & (iz < NZ - 1)
        coords[interior] += perturb * offs[interior] * h[None, :]
    n1 = p + 1
    ex, ey, ez = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ex = ex.transpose(2, 1, 0).ravel()
    ey = ey.transpose(2, 1, 0).ravel()
    ez = ez.transpose(2, 1, 0).ravel()
    li, lj, lk = np.meshgrid(np.arange(n1), np.arange(n1), np.arange(n1), indexing="ij")
    li = li.transpose(2, 1, 0).ravel()
    lj = lj.transpose(2, 1, 0).ravel()
    lk = lk.transpose(2, 1, 0).ravel()
    gx = ex[:, None] * p + li[None, :]
    gy = ey[:, None] * p + lj[None, :]
    gz = ez[:, None] * p + lk[None, :]
    conn = (gx + NX * gy + NX * NY * gz).astype(np.int32)
    return HexMesh(coords=coords, conn=np.ascontiguousarray(conn), order=p, shape=(nx, ny, nz), rng=rng)


def lame_materials(mesh: HexMesh, lam_range=(0.5, 2.0), mu_range=(0.2, 1.0)):
    """Per-element Lame parameters lambda ~ U[lam_range], mu ~ U[mu_range]."""
    lam = mesh.rng.uniform(lam_range[0], lam_range[1], size=mesh.n_elems)
    mu = mesh.rng.uniform(mu_range[0], mu_range[1], size=mesh.n_elems)
    return lam, mu


def normal_dofs(mesh: HexMesh, ncomp: int) -> np.ndarray:
    """Global DOF vector u ~ N(0, 1), index ncomp * node + comp."""
    return mesh.rng.standard_normal(mesh.n_nodes * ncomp)


def bar_mesh(n_cells: int, p: int, seed: int = 0) -> HexMesh:
    """The paper's benchmark mesh: a 1D bar of n x 1 x 1 hexahedra (Sec. 6)."""
    return structured_hex(n_cells, 1, 1, p, 0.0, seed, lengths=(float(n_cells), 1.0, 1.0))


# Named workloads --------------------------------------------------------------

def laplace_q1_cube(n: int = 8, seed: int = 0):
    """Weak Laplacian on an n^3 Q1 cube, interior nodes +-0.1h, u ~ N(0,1) per node."""
    mesh = structured_hex(n, n, n, 1, 0.1, seed)
    u = normal_dofs(mesh, 1)
    return mesh, u


def elasticity_q2_cube(n: int = 48, seed: int = 1, perturb: float = 0.15):
    """Q2 linear elasticity on an n^3 cube, interior nodes +-0.15h,
    lambda ~ U[0.5, 2], mu ~ U[0.2, 1] per element, u ~ N(0,1) per DOF."""
    mesh = structured_hex(n, n, n, 2, perturb, seed)
    lam, mu = lame_materials(mesh)
    u = normal_dofs(mesh, 3)
    return mesh, lam, mu, u


def smooth_vector_field(mesh: HexMesh) -> np.ndarray:
    """u_i(node) = a_i sin(pi x) cos(pi y) with amplitudes a ~ N(0, 1) in R^3 drawn
    from the mesh's generator; global index 3 * node + i."""
    a = mesh.rng.standard_normal(3)
    x, y = mesh.coords[:, 0], mesh.coords[:, 1]
    s = np.sin(np.pi * x) * np.cos(np.pi * y)
    return (s[:, None] * a[None, :]).reshape(-1)


def convect_q2_cube(n: int = 64, seed: int = 3, perturb: float = 0.1):
    """Q2 Navier-Stokes convection on an n^3 cube, interior nodes +-0.1h,
    with the smooth velocity field of smooth_vector_field."""
    mesh = structured_hex(n, n, n, 2, perturb, seed)
    u = smooth_vector_field(mesh)
    return mesh, u


# ---- tetrahedral meshes ---------------------------------------------------------------

@dataclasses.dataclass
class TetMesh:
    coords: np.ndarray  # (n_nodes, 3) float64
    conn: np.ndarray  # (n_elems, N) int32, N = (p+1)(p+2)(p+3)/6
    order: int
    rng: np.random.Generator

    n_nodes = HexMesh.n_nodes
    n_elems = HexMesh.n_elems
    nodes_per_elem = HexMesh.nodes_per_elem


def _lattice(p: int):
    """Barycentric multi-indices (a0, a1, a2, a3) of the order-p lattice nodes,
    x fastest: node (i, j, k)/p has a = (p - i - j - k, i, j, k)."""
    return np.array([(p - i - j - k, i, j, k) for k in range(p + 1) for j in range(p + 1 - k)
                     for i in range(p + 1 - k - j)], dtype=np.int64)


def delaunay_tets(target: int, rng: np.random.Generator, points_per_tet: float = 1 / 6.55):
    """`target` positively oriented tetrahedra of the Delaunay triangulation of
    ceil(target * points_per_tet) uniform points in the unit cube (more points,
    drawn from the same stream, are appended while the triangulation has fewer
    than `target` tetrahedra): tets sorted lexicographically by their sorted
    vertex ids, the first `target` kept (independent of the triangulator's
    output order)."""
    from scipy.spatial import Delaunay
    n_pts = int(np.ceil(target * points_per_tet)) + 4
    pts = rng.uniform(0.0, 1.0, size=(n_pts, 3))
    while True:
        simp = Delaunay(pts).simplices.astype(np.int64)
        v = pts[simp]
        vol6 = np.einsum("ij,ij->i", np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]), v[:, 3] - v[:, 0])
        neg = vol6 < 0
        simp[neg] = simp[neg][:, [0, 1, 3, 2]]
        simp = simp[np.abs(vol6) > 1e-15]
        if len(simp) >= target:
            break
        pts = np.concatenate([pts, rng.uniform(0.0, 1.0, size=(len(pts) // 10 + 8, 3))], 0)
    key = np.sort(simp, axis=1)
    simp = simp[np.lexsort(key.T[::-1])]
    return pts, simp[:target]


def tet_mesh(target: int, p: int, rng: np.random.Generator) -> TetMesh:
    """Order-p straight-sided tetrahedra of a Delaunay mesh (delaunay_tets).
    Global nodes: the triangulation's vertices (only those used, renumbered in
    order of first use by the sorted tets), then p - 1 nodes per edge, then one
    node per face for p = 3; edge and face nodes are shared by neighbouring
    elements.  An edge node is keyed by (smaller vertex id, larger vertex id,
    its barycentric index at the larger one)."""
    pts, simp = delaunay_tets(target, rng)
    used, inv = np.unique(simp.ravel(), return_inverse=True)
    simp = inv.reshape(simp.shape)
    vx = pts[used]
    L = _lattice(p)                              # (N, 4)
    E, N = len(simp), len(L)
    nz = (L > 0)
    kind = nz.sum(1)                             # 1 vertex, 2 edge, 3 face
    conn = np.empty((E, N), dtype=np.int64)
    coords_parts = [vx]
    base = len(vx)
    # vertex nodes
    for a in np.where(kind == 1)[0]:
        conn[:, a] = simp[:, int(np.argmax(L[a]))]
    # edge nodes
    ea = np.where(kind == 2)[0]
    if len(ea):
        ends = np.array([np.where(nz[a])[0] for a in ea])           # local vertex pair per edge node
        g0, g1 = simp[:, ends[:, 0]], simp[:, ends[:, 1]]             # (E, n_edge_nodes)
        k0, k1 = L[ea, ends[:, 0]], L[ea, ends[:, 1]]
        lo, hi = np.minimum(g0, g1), np.maximum(g0, g1)
        k_hi = np.where(g1 > g0, k1[None, :], k0[None, :])            # index at the larger vertex
        keys = np.stack([lo.ravel(), hi.ravel(), k_hi.ravel()], 1)
        uk, einv = np.unique(keys, axis=0, return_inverse=True)
        conn[:, ea] = base + einv.reshape(E, len(ea))
        xe = (vx[uk[:, 0]] * (p - uk[:, 2:3]) + vx[uk[:, 1]] * uk[:, 2:3]) / p
        coords_parts.append(xe)
        base += len(uk)
    # face nodes (p = 3: barycentric (1, 1, 1, 0) patterns)
    fa = np.where(kind == 3)[0]
    if len(fa):
        tri = np.array([np.where(nz[a])[0] for a in fa])
        keys = np.sort(np.stack([simp[:, tri[:, 0]], simp[:, tri[:, 1]], simp[:, tri[:, 2]]], 2), axis=2)
        uk, finv = np.unique(keys.reshape(-1, 3), axis=0, return_inverse=True)
        conn[:, fa] = base + finv.reshape(E, len(fa))
        coords_parts.append(vx[uk].mean(1))
        base += len(uk)
    coords = np.concatenate(coords_parts, 0)
    return TetMesh(coords=np.ascontiguousarray(coords), conn=np.ascontiguousarray(conn.astype(np.int32)), order=p,
                   rng=rng)


def vertex_connectivity(mesh):
    """Connectivity of the order-1 field on the vertices of an order-p mesh (the
    scalar field of a mixed-order pair, e.g. a Q1 or P1 pressure beside a Q2 or P2
    velocity): (E, 8) for hexahedra in the reference order of Q1 nodes (x fastest),
    numbered on the (nx+1)(ny+1)(nz+1) vertex grid; (E, 4) for tetrahedra in the P1
    lattice order, numbered like the mesh's vertex nodes (which come first).
    Returns (conn, n_vertices).  Topology only."""
    if isinstance(mesh, TetMesh):
        L = _lattice(mesh.order)
        loc = [int(np.where(L[:, b] == mesh.order)[0][0]) for b in range(4)]
        conn = np.ascontiguousarray(mesh.conn[:, loc])
        return conn, int(conn.max()) + 1 if conn.size else 0
    nx, ny, nz = mesh.shape
    q1 = structured_hex(nx, ny, nz, 1)
    return q1.conn, q1.n_nodes


def mixed_mesh_groups(scale: float = 1.0, seed: int = 2):
    """The mixed-element workload: P1, P2, P3 tetrahedra (200k, 120k, 40k,
    Delaunay meshes drawn from one stream of seed `seed` in that order) and Q1,
    Q2, Q3 hexahedra (60k = 50x40x30, 30k = 40x30x25, 8k = 20x20x20, +-0.1h,
    seeds seed + 10 + p); `scale` < 1 shrinks every group (tests).  Returns a
    list of (name, mesh) in that order; each mesh carries its generator for the
    materials."""
    rng = np.random.default_rng(seed)
    groups = []
    for p, target in ((1, 200_000), (2, 120_000), (3, 40_000)):
        groups.append(("P%d" % p, tet_mesh(max(8, int(round(target * scale))), p, rng)))
    for p, shape in ((1, (50, 40, 30)), (2, (40, 30, 25)), (3, (20, 20, 20))):
        f = scale ** (1.0 / 3.0)
        sh = tuple(max(1, int(round(n * f))) for n in shape)
        groups.append(("Q%d" % p, structured_hex(*sh, p, 0.1, seed + 10 + p)))
    return groups
