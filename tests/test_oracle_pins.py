"""Pins of the FP64 oracle against what the mathematics and the paper fix.

None of these re-types the oracle's formulas: each check uses a closed form,
exact rational integration (tests/exact_fe.py), a library routine
(numpy.polynomial.legendre.leggauss), an invariant of the forms, or values
printed in the paper (tests/golden/).  Cimrman, arXiv 2107.04121.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2107_04121_gb300 import meshgen
from tests import exact_fe

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# -- quadrature ----------------------------------------------------------------

@pytest.mark.parametrize("n", list(range(1, 9)))
def test_gauss_matches_leggauss(n):
    x, w = oracle.gauss_1d(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(x, 0.5 * (xr + 1.0), rtol=0, atol=2e-15)
    np.testing.assert_allclose(w, 0.5 * wr, rtol=0, atol=2e-15)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_gauss_integrates_monomials_exactly(n):
    x, w = oracle.gauss_1d(n)
    for k in range(2 * n):
        assert abs(np.dot(w, x ** k) - 1.0 / (k + 1)) < 1e-15
    # degree 2n is not integrated exactly
    assert abs(np.dot(w, x ** (2 * n)) - 1.0 / (2 * n + 1)) > 1e-8


def test_hex_quadrature_lexicographic_x_fastest():
    pts, w = oracle.hex_quadrature(3)
    g, gw = np.polynomial.legendre.leggauss(3)
    g, gw = 0.5 * (g + 1), 0.5 * gw
    assert abs(w.sum() - 1.0) < 4e-15
    np.testing.assert_allclose(pts[1], [g[1], g[0], g[0]], atol=1e-15)
    np.testing.assert_allclose(pts[3], [g[0], g[1], g[0]], atol=1e-15)
    np.testing.assert_allclose(pts[9], [g[0], g[0], g[1]], atol=1e-15)
    np.testing.assert_allclose(w[13], gw[1] ** 3, atol=1e-15)


# -- reference basis ------------------------------------------------------------

def _ref_nodes(p):
    n1 = p + 1
    t = np.arange(n1) / p
    return np.array([[t[i], t[j], t[k]] for k in range(n1) for j in range(n1) for i in range(n1)])


@pytest.mark.parametrize("p", [1, 2, 3])
def test_basis_is_nodal_and_partition_of_unity(p):
    nodes = _ref_nodes(p)
    phi, dphi = oracle.hex_basis(p, nodes)
    np.testing.assert_allclose(phi, np.eye(nodes.shape[0]), atol=1e-13)
    rng = np.random.default_rng(5)
    x = rng.uniform(0, 1, (20, 3))
    phi, dphi = oracle.hex_basis(p, x)
    np.testing.assert_allclose(phi.sum(1), 1.0, atol=1e-13)
    np.testing.assert_allclose(dphi.sum(2), 0.0, atol=1e-11)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_basis_gradient_matches_finite_differences(p):
    rng = np.random.default_rng(6)
    x = rng.uniform(0.1, 0.9, (6, 3))
    phi, dphi = oracle.hex_basis(p, x)
    h = 1e-6
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        fp, _ = oracle.hex_basis(p, x + e)
        fm, _ = oracle.hex_basis(p, x - e)
        np.testing.assert_allclose(dphi[:, k, :], (fp - fm) / (2 * h), atol=5e-8)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_basis_reproduces_tensor_polynomials(p):
    # f = x^p y^(p-1) z + 2 lies in Q_p, so its interpolant is exact
    f = lambda X: X[:, 0] ** p * X[:, 1] ** (p - 1) * X[:, 2] + 2.0
    df = lambda X: np.stack([p * X[:, 0] ** (p - 1) * X[:, 1] ** (p - 1) * X[:, 2],
                             (p - 1) * X[:, 0] ** p * X[:, 1] ** max(p - 2, 0) * X[:, 2] if p > 1 else 0 * X[:, 0],
                             X[:, 0] ** p * X[:, 1] ** (p - 1)], 1)
    nodes = _ref_nodes(p)
    x = np.random.default_rng(7).uniform(0, 1, (15, 3))
    phi, dphi = oracle.hex_basis(p, x)
    np.testing.assert_allclose(phi @ f(nodes), f(x), atol=1e-12)
    np.testing.assert_allclose(np.einsum("qkn,n->qk", dphi, f(nodes)), df(x), atol=1e-11)


# -- closed forms on undistorted elements -----------------------------------------

def test_q1_unit_cube_laplacian_closed_form():
    """K^ab of the unit-cube Q1 Laplacian: 1/3 (same node), 0 (edge neighbour),
    -1/12 (face diagonal), -1/12 (body diagonal); a cube of side h gives h K^."""
    n = 8
    mesh = meshgen.structured_hex(n, n, n, 1, 0.0, 0)
    ref = oracle.RefElement(1, 2)
    wdetJ, G, _ = oracle.geometry(mesh.coords, mesh.conn, ref)
    K = oracle.matrix_laplace(wdetJ, G)
    nodes = _ref_nodes(1)
    diff = (np.abs(nodes[:, None, :] - nodes[None, :, :]) > 0.5).sum(-1)
    Khat = np.select([diff == 0, diff == 1, diff == 2, diff == 3], [1 / 3, 0.0, -1 / 12, -1 / 12])
    np.testing.assert_allclose(K, np.broadcast_to(Khat / n, K.shape), rtol=0, atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_box_element_matches_exact_kronecker_integrals(p):
    h = (0.5, 0.7, 1.3)
    mesh = meshgen.structured_hex(1, 1, 1, p, 0.0, 0, lengths=h)
    mesh.coords[:] += np.array([0.25, -1.0, 3.0])  # translation does not change the forms
    ref = oracle.RefElement(p, p + 1)
    wdetJ, G, _ = oracle.geometry(mesh.coords, mesh.conn, ref)
    lam, mu = np.array([1.7]), np.array([0.6])
    KL = oracle.matrix_laplace(wdetJ, G)[0]
    KM = oracle.matrix_mass(wdetJ, ref.phi)[0]
    KE = oracle.matrix_elasticity(wdetJ, G, oracle.lame_to_D(lam, mu))[0]
    for got, want in [(KL, exact_fe.box_laplace(p, h)), (KM, exact_fe.box_mass(p, h)),
                      (KE, exact_fe.box_elasticity(p, h, lam[0], mu[0]))]:
        assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()


def test_affine_element_geometry():
    """An affine map x = A xi + t is reproduced exactly: J = A, det J = det A."""
    rng = np.random.default_rng(8)
    A = np.eye(3) + 0.3 * rng.standard_normal((3, 3))
    if np.linalg.det(A) < 0:
        A[:, 0] *= -1
    t = rng.standard_normal(3)
    for p in (1, 2, 3):
        X = _ref_nodes(p) @ A.T + t
        conn = np.arange(X.shape[0], dtype=np.int32)[None, :]
        ref = oracle.RefElement(p, p + 1)
        wdetJ, G, Jinv = oracle.geometry(X, conn, ref, want_Jinv=True)
        np.testing.assert_allclose(wdetJ[0], ref.w * np.linalg.det(A), rtol=1e-13)
        np.testing.assert_allclose(Jinv[0], np.broadcast_to(np.linalg.inv(A), Jinv[0].shape), atol=1e-13)
        want_G = np.einsum("kj,qka->qja", np.linalg.inv(A), ref.dphi)
        np.testing.assert_allclose(G[0], want_G, atol=1e-12)


def test_inverted_element_is_reported():
    mesh = meshgen.structured_hex(2, 2, 2, 1, 0.0, 0)
    conn = mesh.conn.copy()
    conn[3, [0, 1]] = conn[3, [1, 0]]  # mirror element 3
    with pytest.raises(ValueError, match="element 3"):
        oracle.geometry(mesh.coords, conn, oracle.RefElement(1, 2))


# -- invariants on distorted meshes --------------------------------------------------

@pytest.fixture(scope="module", params=[1, 2, 3])
def distorted(request):
    p = request.param
    mesh = meshgen.structured_hex(3, 3, 3, p, 0.15, 11)
    lam, mu = meshgen.lame_materials(mesh)
    # det J of an order-p map has degree 3p - 1 per axis: a Gauss rule with
    # 2 nq - 1 >= 3p - 1 integrates the element volumes exactly
    nq = max(p + 1, (3 * p + 1) // 2)
    ref = oracle.RefElement(p, nq)
    wdetJ, G, _ = oracle.geometry(mesh.coords, mesh.conn, ref)
    return mesh, ref, wdetJ, G, lam, mu


def test_volumes_sum_to_one(distorted):
    mesh, ref, wdetJ, G, lam, mu = distorted
    assert abs(wdetJ.sum() - 1.0) < 1e-13
    M = oracle.matrix_mass(wdetJ, ref.phi)
    np.testing.assert_allclose(M.sum((1, 2)), wdetJ.sum(1), rtol=1e-13)


def test_laplace_rows_sum_to_zero_and_symmetry(distorted):
    mesh, ref, wdetJ, G, lam, mu = distorted
    K = oracle.matrix_laplace(wdetJ, G)
    scale = np.abs(K).max()
    assert np.abs(K.sum(2)).max() < 1e-13 * scale
    assert np.abs(K - K.transpose(0, 2, 1)).max() < 1e-14 * scale
    # positive semi-definite with exactly one zero eigenvalue (constants)
    ev = np.linalg.eigvalsh(K[0])
    assert ev[0] > -1e-13 * scale and ev[1] > 1e-6 * scale


def test_patch_test_linear_field(distorted):
    mesh, ref, wdetJ, G, lam, mu = distorted
    b = np.array([0.3, -1.2, 0.7])
    u = mesh.coords @ b + 0.5
    grad = np.einsum("eqja,ea->eqj", G, u[mesh.conn])
    np.testing.assert_allclose(grad, np.broadcast_to(b, grad.shape), atol=1e-12)


def test_elasticity_rigid_body_modes_and_symmetry(distorted):
    mesh, ref, wdetJ, G, lam, mu = distorted
    K = oracle.matrix_elasticity(wdetJ, G, oracle.lame_to_D(lam, mu))
    X = mesh.coords[mesh.conn]  # (E, N, 3)
    E, N = mesh.conn.shape
    modes = []
    for i in range(3):
        m = np.zeros((E, 3, N))
        m[:, i, :] = 1.0
        modes.append(m)
    for axis in range(3):  # rotations u = w x x
        w = np.zeros(3)
        w[axis] = 1.0
        modes.append(np.cross(w, X).transpose(0, 2, 1))
    scale = np.abs(K).max()
    for m in modes:
        Ku = np.einsum("eij,ej->ei", K, m.reshape(E, 3 * N))
        assert np.abs(Ku).max() < 1e-12 * scale * max(1.0, np.abs(m).max())
    assert np.abs(K - K.transpose(0, 2, 1)).max() < 1e-14 * scale
    # exactly six zero eigenvalues
    ev = np.linalg.eigvalsh(K[0])
    assert np.all(np.abs(ev[:6]) < 1e-10 * scale) and ev[6] > 1e-6 * scale


def test_residual_equals_matrix_times_dofs(distorted):
    mesh, ref, wdetJ, G, lam, mu = distorted
    rng = np.random.default_rng(9)
    E, N = mesh.conn.shape
    u1 = rng.standard_normal(mesh.n_nodes)
    u3 = rng.standard_normal(3 * mesh.n_nodes)
    ue3 = u3.reshape(-1, 3)[mesh.conn].transpose(0, 2, 1).reshape(E, 3 * N)  # component-major
    coef = rng.uniform(0.5, 2.0, E)
    D = oracle.lame_to_D(lam, mu)
    cases = [
        (oracle.matrix_laplace(wdetJ, G, coef), oracle.residual_laplace(mesh.conn, wdetJ, G, u1, coef), u1[mesh.conn]),
        (oracle.matrix_mass(wdetJ, ref.phi, 1, coef), oracle.residual_mass(mesh.conn, wdetJ, ref.phi, u1, 1, coef),
         u1[mesh.conn]),
        (oracle.matrix_mass(wdetJ, ref.phi, 3), oracle.residual_mass(mesh.conn, wdetJ, ref.phi, u3, 3), ue3),
        (oracle.matrix_elasticity(wdetJ, G, D), oracle.residual_elasticity(mesh.conn, wdetJ, G, D, u3), ue3),
    ]
    for K, r, ue in cases:
        want = np.einsum("eij,ej->ei", K, ue)
        assert np.abs(r - want).max() < 1e-12 * np.abs(want).max()


def test_vector_mass_is_block_diagonal_scalar_mass(distorted):
    mesh, ref, wdetJ, G, lam, mu = distorted
    M1 = oracle.matrix_mass(wdetJ, ref.phi, 1)
    M3 = oracle.matrix_mass(wdetJ, ref.phi, 3)
    N = M1.shape[1]
    for i in range(3):
        for k in range(3):
            blk = M3[:, i * N:(i + 1) * N, k * N:(k + 1) * N]
            np.testing.assert_array_equal(blk, M1 if i == k else 0.0)


@pytest.mark.parametrize("p", [1, 2])
def test_assembled_laplace_residual_of_linear_field_vanishes_inside(p):
    mesh = meshgen.structured_hex(3, 3, 3, p, 0.1, 12)
    ref = oracle.RefElement(p, p + 1)
    wdetJ, G, _ = oracle.geometry(mesh.coords, mesh.conn, ref)
    u = mesh.coords @ np.array([1.0, -2.0, 0.5]) + 3.0
    g = oracle.assemble(mesh.conn, oracle.residual_laplace(mesh.conn, wdetJ, G, u), mesh.n_nodes, 1)
    X = mesh.coords
    inside = np.all((X > 1e-9) & (X < 1 - 1e-9), axis=1)
    assert inside.sum() > 0
    assert np.abs(g[inside]).max() < 1e-12
    assert np.abs(g[~inside]).max() > 1e-3


def test_assemble_matches_brute_force_and_volume():
    mesh = meshgen.structured_hex(4, 3, 2, 2, 0.1, 13)
    ref = oracle.RefElement(2, 3)
    wdetJ, G, _ = oracle.geometry(mesh.coords, mesh.conn, ref)
    r = oracle.residual_mass(mesh.conn, wdetJ, ref.phi, np.ones(3 * mesh.n_nodes), 3)
    g = oracle.assemble(mesh.conn, r, mesh.n_nodes, 3)
    want = np.zeros(3 * mesh.n_nodes)
    E, N = mesh.conn.shape
    for e in range(E):
        for a in range(N):
            for i in range(3):
                want[3 * mesh.conn[e, a] + i] += r[e, i * N + a]
    np.testing.assert_array_equal(g, want)
    # sum of the assembled mass action on a constant field is the volume per component
    np.testing.assert_allclose(g.reshape(-1, 3).sum(0), 1.0, rtol=1e-13)
    g2 = oracle.assemble(mesh.conn, r, mesh.n_nodes, 3, g)
    np.testing.assert_allclose(g2, 2 * g, rtol=1e-15)


# -- the paper's printed sizes --------------------------------------------------------

def _tab_cdc():
    rows = []
    with open(os.path.join(GOLDEN, "tab_cdc.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([float(x) for x in line.split()])
    return rows


def test_tab_cdc_sizes():
    """Tab. cdc: bar-mesh DOF counts and FP64 output sizes of (n_c, n_dr[, n_dc]) arrays."""
    for cells, p, nqp, ndofs, _, rs, Ms, rv, Mv in _tab_cdc():
        cells, p = int(cells), int(p)
        N = (p + 1) ** 3
        assert (p + 1) ** 3 == nqp  # (p+1)^3 Gauss points
        assert meshgen.grid_node_count(cells, 1, 1, p) == ndofs
        mb = lambda n: round(n * 8 / 1e6, 1)
        assert mb(cells * N) == rs
        assert mb(cells * N * N) == Ms
        assert mb(cells * 3 * N) == rv
        assert mb(cells * 9 * N * N) == Mv
    mesh = meshgen.bar_mesh(1024, 2)
    assert mesh.n_nodes == 18441 and mesh.n_elems == 1024


def test_printed_einsum_shapes():
    """Operand and output shapes printed in Sec. 5.3 for 1024-cell meshes."""
    ref2 = oracle.RefElement(2, 3)
    mesh = meshgen.bar_mesh(4, 2)
    wdetJ, G, _ = oracle.geometry(mesh.coords, mesh.conn, ref2)
    assert G.shape[1:] == (27, 3, 27)  # cqjd (1024, 27, 3, 27)
    assert oracle.matrix_laplace(wdetJ, G).shape[1:] == (27, 27)  # cde (1024, 27, 27)
    ref1 = oracle.RefElement(1, 2)
    mesh1 = meshgen.bar_mesh(4, 1)
    w1, G1, _ = oracle.geometry(mesh1.coords, mesh1.conn, ref1)
    M = oracle.matrix_mass(w1, ref1.phi, 3)
    assert M.reshape(4, 3, 8, 3, 8).shape[1:] == (3, 8, 3, 8)  # crdse (1024, 3, 8, 3, 8)
    D = oracle.lame_to_D(np.ones(4), np.ones(4))
    assert D.shape[1:] == (6, 6)
    assert oracle.matrix_elasticity(w1, G1, D).reshape(4, 3, 8, 3, 8).shape[1:] == (3, 8, 3, 8)  # cresf


# -- Navier-Stokes convective term 'i,i.j,j' (Eq. fe2, fe4) ------------------------

def _box_linear_field(p, seed):
    rng = np.random.default_rng(seed)
    h = (0.5, 0.7, 1.3)
    x0 = np.array([0.25, -1.0, 3.0])
    mesh = meshgen.structured_hex(1, 1, 1, p, 0.0, 0, lengths=h)
    mesh.coords[:] += x0
    A = rng.standard_normal((3, 3))
    c = rng.standard_normal(3)
    u = (mesh.coords @ A.T + c).reshape(-1)  # u[3 node + i] = (A x + c)_i
    return mesh, h, x0, A, c, u


@pytest.mark.parametrize("p", [1, 2, 3])
def test_convect_box_linear_field_closed_form(p):
    """On a box with the linear field u = A x + c (w = u): the residual is
    int phi_a (A (A x + c))_i = M (nodal values of A(Ax + c)), the derivative with
    respect to the advection operand is A_ik M, and with respect to the gradient
    operand delta_ik int phi_a (u . grad phi_b), all from exact 1-D integrals."""
    mesh, h, x0, A, c, u = _box_linear_field(p, 21 + p)
    ref = oracle.RefElement(p, p + 1)
    wdetJ, G, _ = oracle.geometry(mesh.coords, mesh.conn, ref)
    N = ref.N
    M = exact_fe.box_mass(p, h)
    nodal = mesh.coords[mesh.conn[0]] @ A.T + c        # (N, 3): u at the element's nodes
    accel = nodal @ A.T                                # (A u)(x_node) = A (A x + c)
    r_want = np.concatenate([M @ accel[:, i] for i in range(3)])
    r = oracle.residual_convect(mesh.conn, wdetJ, ref.phi, G, u)[0]
    assert np.abs(r - r_want).max() <= 1e-13 * np.abs(r_want).max()
    Kw = oracle.matrix_convect(mesh.conn, wdetJ, ref.phi, G, u, wrt_u=False, wrt_w=True)[0]
    Ku = oracle.matrix_convect(mesh.conn, wdetJ, ref.phi, G, u, wrt_u=True, wrt_w=False)[0]
    Kw_want = np.kron(A, M)
    Cb = exact_fe.box_convection(p, h, x0, A, c)
    Ku_want = np.kron(np.eye(3), Cb)
    assert np.abs(Kw - Kw_want).max() <= 1e-13 * np.abs(Kw_want).max()
    assert np.abs(Ku - Ku_want).max() <= 1e-13 * np.abs(Ku_want).max()


@pytest.fixture(scope="module", params=[1, 2])
def convect_case(request):
    p = request.param
    mesh = meshgen.structured_hex(2, 2, 2, p, 0.15, 31)
    rng = np.random.default_rng(32)
    u = rng.standard_normal(3 * mesh.n_nodes)
    w = rng.standard_normal(3 * mesh.n_nodes)
    ref = oracle.RefElement(p, p + 1)
    wdetJ, G, _ = oracle.geometry(mesh.coords, mesh.conn, ref)
    return mesh, ref, wdetJ, G, u, w


def _element_dofs(conn, v):
    """v_e[e, i*N + a] = v[3 conn[e, a] + i]."""
    return np.concatenate([v[3 * conn + i] for i in range(3)], axis=1)


def test_convect_jacobian_is_exact_central_difference(convect_case):
    """r(u) is quadratic in u, so a central difference of any step is exact up to
    rounding: (r(u + s d) - r(u - s d)) / 2s = K(u) d_e."""
    mesh, ref, wdetJ, G, u, w = convect_case
    d = np.random.default_rng(33).standard_normal(u.shape)
    s = 0.5
    rp = oracle.residual_convect(mesh.conn, wdetJ, ref.phi, G, u + s * d)
    rm = oracle.residual_convect(mesh.conn, wdetJ, ref.phi, G, u - s * d)
    K = oracle.matrix_convect(mesh.conn, wdetJ, ref.phi, G, u)
    got = np.einsum("erc,ec->er", K, _element_dofs(mesh.conn, d))
    fd = (rp - rm) / (2 * s)
    assert np.abs(got - fd).max() <= 1e-12 * np.abs(fd).max()


def test_convect_degree_two_homogeneity(convect_case):
    """Euler's relation for a form quadratic in u: K(u) u_e = 2 r(u)."""
    mesh, ref, wdetJ, G, u, w = convect_case
    K = oracle.matrix_convect(mesh.conn, wdetJ, ref.phi, G, u)
    r = oracle.residual_convect(mesh.conn, wdetJ, ref.phi, G, u)
    got = np.einsum("erc,ec->er", K, _element_dofs(mesh.conn, u))
    assert np.abs(got - 2 * r).max() <= 1e-12 * np.abs(r).max()


def test_convect_partial_derivatives_are_the_linear_actions(convect_case):
    """With distinct operands the form is linear in each: the derivative with
    respect to the gradient operand applied to u_e, and the one with respect to
    the advection operand applied to w_e, both give r(u, w); the two terms add
    up to the full derivative."""
    mesh, ref, wdetJ, G, u, w = convect_case
    r = oracle.residual_convect(mesh.conn, wdetJ, ref.phi, G, u, w)
    Ku = oracle.matrix_convect(mesh.conn, wdetJ, ref.phi, G, u, w, wrt_u=True, wrt_w=False)
    Kw = oracle.matrix_convect(mesh.conn, wdetJ, ref.phi, G, u, w, wrt_u=False, wrt_w=True)
    Kb = oracle.matrix_convect(mesh.conn, wdetJ, ref.phi, G, u, w)
    sc = np.abs(r).max()
    assert np.abs(np.einsum("erc,ec->er", Ku, _element_dofs(mesh.conn, u)) - r).max() <= 1e-12 * sc
    assert np.abs(np.einsum("erc,ec->er", Kw, _element_dofs(mesh.conn, w)) - r).max() <= 1e-12 * sc
    assert np.abs(Ku + Kw - Kb).max() <= 1e-13 * np.abs(Kb).max()


def test_convect_rows_of_advection_block_sum_to_zero(convect_case):
    """sum_b grad phi_b = 0 (partition of unity): every row of the derivative with
    respect to the gradient operand sums to zero within its diagonal block, and
    its off-diagonal blocks vanish."""
    mesh, ref, wdetJ, G, u, w = convect_case
    N = ref.N
    Ku = oracle.matrix_convect(mesh.conn, wdetJ, ref.phi, G, u, w, wrt_u=True, wrt_w=False)
    sc = np.abs(Ku).max()
    for i in range(3):
        for k in range(3):
            blk = Ku[:, i * N:(i + 1) * N, k * N:(k + 1) * N]
            if i == k:
                assert np.abs(blk.sum(2)).max() <= 1e-13 * sc
            else:
                assert np.abs(blk).max() == 0.0


def test_convect_constant_advection_of_constant_field_vanishes(convect_case):
    """A constant field has no gradient: r(u = const) = 0 on distorted elements."""
    mesh, ref, wdetJ, G, u, w = convect_case
    uc = np.tile(np.array([0.3, -1.2, 2.0]), mesh.n_nodes)
    r = oracle.residual_convect(mesh.conn, wdetJ, ref.phi, G, uc, w)
    assert np.abs(r).max() <= 1e-13


# -- adjoint of the assembled elasticity residual, J = |R|^2 / 2 ----------------------

@pytest.fixture(scope="module")
def adjoint_case():
    mesh = meshgen.structured_hex(2, 2, 3, 2, 0.1, 4)
    lam, mu = meshgen.lame_materials(mesh)
    u = meshgen.normal_dofs(mesh, 3)
    ref = oracle.RefElement(2, 3)
    J, dlam, dmu, dX = oracle.elasticity_objective_gradient(mesh.coords, mesh.conn, ref, lam, mu, u)
    return mesh, ref, lam, mu, u, J, dlam, dmu, dX


def test_adjoint_material_gradient_is_exact_central_difference(adjoint_case):
    """R is linear in (lambda, mu), so J is quadratic and a central difference of
    any step equals the directional derivative up to rounding."""
    mesh, ref, lam, mu, u, J, dlam, dmu, dX = adjoint_case
    rng = np.random.default_rng(41)
    for _ in range(3):
        dl, dm = rng.standard_normal(lam.shape), rng.standard_normal(mu.shape)
        s = 0.1
        Jp, _ = oracle.elasticity_objective(mesh.coords, mesh.conn, ref, lam + s * dl, mu + s * dm, u)
        Jm, _ = oracle.elasticity_objective(mesh.coords, mesh.conn, ref, lam - s * dl, mu - s * dm, u)
        fd = (Jp - Jm) / (2 * s)
        an = dlam @ dl + dmu @ dm
        assert abs(fd - an) <= 1e-12 * abs(J), (fd, an)


def test_adjoint_coordinate_gradient_matches_central_difference(adjoint_case):
    """The shape derivative against central differences of the objective in
    seeded unit directions over all node coordinates (step 1e-6, O(h^2))."""
    mesh, ref, lam, mu, u, J, dlam, dmu, dX = adjoint_case
    rng = np.random.default_rng(42)
    for _ in range(5):
        d = rng.standard_normal(mesh.coords.shape)
        d /= np.linalg.norm(d)
        h = 1e-6
        Jp, _ = oracle.elasticity_objective(mesh.coords + h * d, mesh.conn, ref, lam, mu, u)
        Jm, _ = oracle.elasticity_objective(mesh.coords - h * d, mesh.conn, ref, lam, mu, u)
        fd = (Jp - Jm) / (2 * h)
        an = float((dX * d).sum())
        assert abs(fd - an) <= 1e-7 * np.linalg.norm(dX), (fd, an)


def test_adjoint_coordinate_gradient_is_translation_invariant(adjoint_case):
    """J does not change when every node moves by the same vector: the node
    gradients sum to zero in each direction."""
    mesh, ref, lam, mu, u, J, dlam, dmu, dX = adjoint_case
    assert np.abs(dX.sum(0)).max() <= 1e-12 * np.abs(dX).sum()


def test_adjoint_material_gradient_closed_form_on_homogeneous_stretch():
    """One box element, u = uniform stretch e (u = diag(e) x): grad u = diag(e) at
    every point, and with rbar = R the per-element terms are wdetJ-weighted
    products; check d/dlambda = sum_q wdetJ div(u) div(rbar_h) against a direct
    evaluation of rbar's divergence through the exact box integrals."""
    h = (0.5, 0.7, 1.3)
    mesh = meshgen.structured_hex(1, 1, 1, 2, 0.0, 0, lengths=h)
    e = np.array([0.3, -0.2, 0.5])
    u = (mesh.coords * e).reshape(-1)
    ref = oracle.RefElement(2, 3)
    lam, mu = np.array([1.3]), np.array([0.7])
    wdetJ, G, _ = oracle.geometry(mesh.coords, mesh.conn, ref)
    # a given adjoint field rbar: a second linear field, so div(rbar_h) = trace(Bm)
    Bm = np.array([[0.2, 0.1, 0.0], [0.0, -0.4, 0.3], [0.5, 0.0, 0.1]])
    rbar = (mesh.coords @ Bm.T).reshape(-1)
    dlam, dmu, _ = oracle.adjoint_elasticity_terms(mesh.conn, wdetJ, G, lam, mu, u, rbar)
    vol = h[0] * h[1] * h[2]
    epsb = 0.5 * (Bm + Bm.T)
    assert abs(dlam[0] - vol * e.sum() * np.trace(Bm)) <= 1e-13
    assert abs(dmu[0] - vol * 2 * (np.diag(e) * epsb).sum()) <= 1e-13


# -- tetrahedra: Grundmann-Moller rules and Lagrange bases ----------------------------

from math import factorial as _fact


@pytest.mark.parametrize("s", [0, 1, 2, 3, 4])
def test_gm_rule_integrates_monomials_exactly(s):
    """int_T x^a y^b z^c = a! b! c! / (a + b + c + 3)! for a + b + c <= 2s + 1."""
    pts, w = oracle.gm_rule(s)
    assert len(w) == {0: 1, 1: 5, 2: 15, 3: 35, 4: 70}[s]
    deg = 2 * s + 1
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            for c in range(deg + 1 - a - b):
                exact = _fact(a) * _fact(b) * _fact(c) / _fact(a + b + c + 3)
                got = float((w * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c).sum())
                assert abs(got - exact) <= 1e-15 + 1e-13 * exact, (s, a, b, c)


def _tet_nodes(p):
    return np.array([(i / p, j / p, k / p) for k in range(p + 1) for j in range(p + 1 - k)
                     for i in range(p + 1 - k - j)])


@pytest.mark.parametrize("p", [1, 2, 3])
def test_tet_basis_nodal_partition_and_reproduction(p):
    X = _tet_nodes(p)
    N = len(X)
    assert N == (p + 1) * (p + 2) * (p + 3) // 6
    phi, dphi = oracle.tet_basis(p, X)
    np.testing.assert_allclose(phi, np.eye(N), atol=1e-14)
    pts, _ = oracle.gm_rule(3)
    phi, dphi = oracle.tet_basis(p, pts)
    np.testing.assert_allclose(phi.sum(1), 1.0, atol=1e-14)
    np.testing.assert_allclose(dphi.sum(2), 0.0, atol=1e-12)
    # every polynomial of degree <= p is reproduced by its nodal interpolant
    for a in range(p + 1):
        for b in range(p + 1 - a):
            for c in range(p + 1 - a - b):
                f = lambda x: x[..., 0] ** a * x[..., 1] ** b * x[..., 2] ** c
                np.testing.assert_allclose(phi @ f(X), f(pts), atol=1e-13)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_tet_basis_gradient_matches_finite_differences(p):
    pts = np.array([[0.2, 0.3, 0.1], [0.05, 0.6, 0.25], [0.4, 0.1, 0.35]])
    phi, dphi = oracle.tet_basis(p, pts)
    h = 1e-6
    for c in range(3):
        e = np.zeros(3)
        e[c] = h
        fp, _ = oracle.tet_basis(p, pts + e)
        fm, _ = oracle.tet_basis(p, pts - e)
        np.testing.assert_allclose(dphi[:, c, :], (fp - fm) / (2 * h), atol=1e-8)


def _random_tet(seed):
    rng = np.random.default_rng(seed)
    V = rng.standard_normal((4, 3))
    if np.linalg.det(V[1:] - V[0]) < 0:
        V[[2, 3]] = V[[3, 2]]
    return V


def _tet_element(p, V):
    """Node coordinates of the straight-sided order-p tet on vertices V."""
    X = _tet_nodes(p)
    L = np.stack([1 - X.sum(1), X[:, 0], X[:, 1], X[:, 2]], 1)
    return L @ V


def test_p1_tet_closed_forms():
    """P1: K_ab = V grad(l_a) . grad(l_b), M_ab = V (1 + delta_ab) / 20."""
    Vx = _random_tet(71)
    ref = oracle.RefTet(1, 1)
    conn = np.arange(4, dtype=np.int32)[None, :]
    wdetJ, G, _ = oracle.geometry(Vx, conn, ref)
    vol = abs(np.linalg.det(Vx[1:] - Vx[0])) / 6
    A = np.vstack([np.ones(4), Vx.T])            # l = A^-1 [1, x]
    gl = np.linalg.inv(A)[:, 1:]                 # grad l_a (4, 3)
    K = oracle.matrix_laplace(wdetJ, G)[0]
    M = oracle.matrix_mass(wdetJ, ref.phi)[0]
    np.testing.assert_allclose(K, vol * gl @ gl.T, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(M, vol * (1 + np.eye(4)) / 20, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("p", [2, 3])
def test_higher_order_tet_invariants(p):
    Vx = _random_tet(72 + p)
    X = _tet_element(p, Vx)
    conn = np.arange(len(X), dtype=np.int32)[None, :]
    ref = oracle.RefTet(p, p)
    wdetJ, G, _ = oracle.geometry(X, conn, ref)
    vol = abs(np.linalg.det(Vx[1:] - Vx[0])) / 6
    K = oracle.matrix_laplace(wdetJ, G)[0]
    M = oracle.matrix_mass(wdetJ, ref.phi)[0]
    assert abs(wdetJ.sum() - vol) <= 1e-13 * vol
    assert np.abs(K.sum(1)).max() <= 1e-12 * np.abs(K).max()
    np.testing.assert_allclose(K, K.T, atol=1e-13 * np.abs(K).max())
    assert abs(M.sum() - vol) <= 1e-13 * vol
    # the mass integrand phi_a phi_b (degree 2p) is integrated exactly by the
    # index-p rule: a rule of higher index gives the same matrix
    ref_hi = oracle.RefTet(p, p + 2)
    wd_hi, _, _ = oracle.geometry(X, conn, ref_hi)
    M_hi = oracle.matrix_mass(wd_hi, ref_hi.phi)[0]
    np.testing.assert_allclose(M, M_hi, atol=1e-14 * np.abs(M).max())
    # elasticity annihilates the six rigid-body modes
    lam, mu = np.array([1.4]), np.array([0.6])
    KE = oracle.matrix_elasticity(wdetJ, G, oracle.lame_to_D(lam, mu))[0]
    N = len(X)
    for mode in range(6):
        v = np.zeros((3, N))
        if mode < 3:
            v[mode] = 1.0
        else:
            a, b = [(0, 1), (1, 2), (0, 2)][mode - 3]
            v[a], v[b] = -X[:, b], X[:, a]
        assert np.abs(KE @ v.reshape(-1)).max() <= 1e-12 * np.abs(KE).max()


@pytest.mark.parametrize("p", [1, 2, 3])
def test_tet_mesh_patch_test(p):
    """On the conforming Delaunay mesh the assembled Laplace residual of a linear
    field vanishes at every node off the mesh boundary (the P_p space holds
    linear fields and the rule of index p integrates the products exactly)."""
    mesh = meshgen.tet_mesh(600, p, np.random.default_rng(5))
    ref = oracle.RefTet(p, p)
    wdetJ, G, _ = oracle.geometry(mesh.coords, mesh.conn, ref)
    u = mesh.coords @ np.array([0.7, -1.3, 0.4]) + 0.2
    r = oracle.residual_laplace(mesh.conn, wdetJ, G, u)
    R = oracle.assemble(mesh.conn, r, mesh.n_nodes, 1)
    X = mesh.coords
    # boundary of the triangulated domain (the points' convex hull): faces of one
    # tet only; every node on such a face (its barycentric index at the opposite
    # vertex is 0) is a boundary node
    L = np.array([(p - i - j - k, i, j, k) for k in range(p + 1) for j in range(p + 1 - k)
                  for i in range(p + 1 - k - j)])
    vert = [int(np.argmax(L[:, m])) for m in range(4)]        # local vertex nodes
    faces = {}
    for e, c in enumerate(mesh.conn):
        for m in range(4):
            key = tuple(sorted(c[vert[o]] for o in range(4) if o != m))
            faces.setdefault(key, []).append((e, m))
    inside = np.ones(mesh.n_nodes, dtype=bool)
    for lst in faces.values():
        if len(lst) == 1:
            e, m = lst[0]
            inside[mesh.conn[e][L[:, m] == 0]] = False
    assert inside.sum() > 10
    # zero up to the rounding of the summed terms K_ab u_b (slivers of a Delaunay
    # mesh give large entries that cancel)
    K = oracle.matrix_laplace(wdetJ, G)
    scale = (np.abs(K) * np.abs(u[mesh.conn])[:, None, :]).sum(2).max()
    assert np.abs(R[inside]).max() <= 1e-13 * scale
    vol = sum(abs(np.linalg.det(X[c[vert[1:]]] - X[c[vert[0]]])) / 6 for c in mesh.conn)
    assert abs(wdetJ.sum() - vol) <= 1e-12


# -- remaining Tab. ewfd forms and eval mode --------------------------------------------

@pytest.mark.parametrize("p", [1, 2])
def test_stokes_wdot_divergence_on_box_match_exact_integrals(p):
    h = (0.5, 0.7, 1.3)
    mesh = meshgen.structured_hex(1, 1, 1, p, 0.0, 0, lengths=h)
    mesh.coords[:] += np.array([0.25, -1.0, 3.0])
    ref = oracle.RefElement(p, p + 1)
    wdetJ, G, _ = oracle.geometry(mesh.coords, mesh.conn, ref)
    N = ref.N
    Bs = exact_fe.box_stokes_blocks(p, h)
    B = oracle.matrix_stokes(wdetJ, G, ref.phi)[0]
    want = np.concatenate(Bs, 0)
    assert np.abs(B - want).max() <= 1e-13 * np.abs(want).max()
    # divergence: int d phi_a / d x_i = sum_b B_i[a][b] (partition of unity)
    rd = oracle.residual_stokes(mesh.conn, wdetJ, G, ref.phi)[0]
    np.testing.assert_allclose(rd, want.sum(1), atol=1e-13)
    # Stokes with a linear pressure: B applied to its nodal values
    rng = np.random.default_rng(3)
    pl = mesh.coords @ rng.standard_normal(3) + 0.5
    rs = oracle.residual_stokes(mesh.conn, wdetJ, G, ref.phi, pl)[0]
    np.testing.assert_allclose(rs, want @ pl[mesh.conn[0]], atol=1e-12)
    # transposed coupling: r_T = sum_i B_i^T u_i
    u = rng.standard_normal(3 * mesh.n_nodes)
    rt = oracle.residual_stokes_t(mesh.conn, wdetJ, G, ref.phi, u)[0]
    ue = u.reshape(-1, 3)[mesh.conn[0]]
    np.testing.assert_allclose(rt, sum(Bs[i].T @ ue[:, i] for i in range(3)), atol=1e-12)
    # weighted dot: M kron the exact mass matrix, and its residual K u
    M = rng.standard_normal((1, 3, 3))
    K = oracle.matrix_wdot(wdetJ, ref.phi, M)[0]
    Kw = np.kron(M[0], exact_fe.box_mass(p, h))
    assert np.abs(K - Kw).max() <= 1e-13 * np.abs(Kw).max()
    rw = oracle.residual_wdot(mesh.conn, wdetJ, ref.phi, M, u)[0]
    np.testing.assert_allclose(rw, Kw @ np.concatenate([ue[:, i] for i in range(3)]), atol=1e-12)


def test_eval_mode_linear_fields_on_distorted_mesh(distorted):
    """Integrals over the unit cube (total volume 1) of products of linear
    fields, whose integrands are constants: the element values sum to them."""
    mesh, ref, wdetJ, G, lam, mu = distorted
    rng = np.random.default_rng(8)
    A, Bm = rng.standard_normal((3, 3)), rng.standard_normal((3, 3))
    a, b, c, d = (rng.standard_normal(3) for _ in range(4))
    X = mesh.coords
    ev = lambda kind, u, **kw: oracle.eval_form(kind, mesh.conn, wdetJ, G, ref.phi, u, **kw).sum(0)
    # scalar Laplace: grad(a.x) . grad(b.x) = a . b
    assert abs(ev("laplace", X @ a, w=X @ b)[0] - a @ b) <= 1e-12
    # dot products of constants
    assert abs(ev("mass", np.full(mesh.n_nodes, 2.0), w=np.full(mesh.n_nodes, 3.0), ncomp=1)[0] - 6.0) <= 1e-12
    uc, wc = np.tile(c, mesh.n_nodes), np.tile(d, mesh.n_nodes)
    assert abs(ev("mass", uc, w=wc)[0] - c @ d) <= 1e-12
    Mw = np.broadcast_to(A, (mesh.n_elems, 3, 3)).copy()
    assert abs(ev("wdot", uc, w=wc, mat=Mw)[0] - c @ A @ d) <= 1e-12
    # linear vector fields u = A x, w = B x: eps(u) = sym(A) (engineering shear in Voigt)
    uA, wB = (X @ A.T).reshape(-1), (X @ Bm.T).reshape(-1)
    voigt = lambda F: np.array([F[0, 0], F[1, 1], F[2, 2], F[0, 1] + F[1, 0], F[0, 2] + F[2, 0], F[1, 2] + F[2, 1]])
    D = oracle.lame_to_D(lam, mu)
    got = oracle.eval_form("elasticity", mesh.conn, wdetJ, G, ref.phi, uA, w=wB, mat=D)[:, 0]
    want = np.einsum("i,eij,j->e", voigt(A), D, voigt(Bm)) * wdetJ.sum(1)
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-14)
    cau = oracle.eval_form("cauchy", mesh.conn, wdetJ, G, ref.phi, uA, mat=D)
    np.testing.assert_allclose(cau, np.einsum("eij,j->ei", D, voigt(A)) * wdetJ.sum(1)[:, None], rtol=1e-11,
                               atol=1e-14)
    assert abs(ev("div", uA)[0] - np.trace(A)) <= 1e-12
    assert abs(ev("stokes", uA, w=np.full(mesh.n_nodes, 2.0))[0] - 2 * np.trace(A)) <= 1e-12
    # convection u_i (d w_i / d x_j) z_j with constant u, z and w = B x: c^T B d
    assert abs(ev("convect", uc, w=wB, z=wc)[0] - c @ Bm @ d) <= 1e-12


def test_eval_mode_equals_bilinear_form_of_the_matrices(distorted):
    """eval(u, w) = w_e . K_e u_e for the Laplacian and elasticity, element by element."""
    mesh, ref, wdetJ, G, lam, mu = distorted
    rng = np.random.default_rng(9)
    u, w = rng.standard_normal(mesh.n_nodes), rng.standard_normal(mesh.n_nodes)
    K = oracle.matrix_laplace(wdetJ, G)
    e1 = oracle.eval_form("laplace", mesh.conn, wdetJ, G, ref.phi, u, w=w)[:, 0]
    np.testing.assert_allclose(e1, np.einsum("ea,eab,eb->e", w[mesh.conn], K, u[mesh.conn]), rtol=1e-11,
                               atol=1e-13)
    u3, w3 = rng.standard_normal(3 * mesh.n_nodes), rng.standard_normal(3 * mesh.n_nodes)
    D = oracle.lame_to_D(lam, mu)
    KE = oracle.matrix_elasticity(wdetJ, G, D)
    e2 = oracle.eval_form("elasticity", mesh.conn, wdetJ, G, ref.phi, u3, w=w3, mat=D)[:, 0]
    ue = np.concatenate([u3[3 * mesh.conn + i] for i in range(3)], 1)
    we = np.concatenate([w3[3 * mesh.conn + i] for i in range(3)], 1)
    np.testing.assert_allclose(e2, np.einsum("ea,eab,eb->e", we, KE, ue), rtol=1e-11, atol=1e-13)


# -- mixed-order Stokes pair (Q2/Q1, P2/P1) ------------------------------------------------

def test_mixed_order_stokes_on_box_matches_exact_integrals():
    """Q2 velocity, Q1 pressure on a box: B_i[a][b] = int d_i phi_a psi_b from exact
    rational 1-D integrals of the two Lagrange bases; the residual of the coupling
    is B p_e and that of the transposed coupling sum_i B_i^T u_i."""
    h = (0.5, 0.7, 1.3)
    mesh = meshgen.structured_hex(1, 1, 1, 2, 0.0, 0, lengths=h)
    mesh.coords[:] += np.array([0.25, -1.0, 3.0])
    ref_u, ref_p = oracle.RefElement(2, 3), oracle.RefElement(1, 3)
    wdetJ, G, _ = oracle.geometry(mesh.coords, mesh.conn, ref_u)
    Bs = exact_fe.box_stokes_mixed_blocks(2, 1, h)
    want = np.concatenate(Bs, 0)
    B = oracle.matrix_stokes_mixed(wdetJ, G, ref_p.phi)[0]
    assert B.shape == (81, 8)
    assert np.abs(B - want).max() <= 1e-13 * np.abs(want).max()
    conn_p, n_p = meshgen.vertex_connectivity(mesh)
    assert conn_p.shape == (1, 8) and n_p == 8
    rng = np.random.default_rng(5)
    p = rng.standard_normal(n_p)
    rs = oracle.residual_stokes_mixed(conn_p, wdetJ, G, ref_p.phi, p)[0]
    np.testing.assert_allclose(rs, want @ p[conn_p[0]], atol=1e-12)
    u = rng.standard_normal(3 * mesh.n_nodes)
    rt = oracle.residual_stokes_t_mixed(mesh.conn, wdetJ, G, ref_p.phi, u)[0]
    ue = u.reshape(-1, 3)[mesh.conn[0]]
    np.testing.assert_allclose(rt, sum(Bs[i].T @ ue[:, i] for i in range(3)), atol=1e-12)


def test_mixed_order_stokes_with_equal_bases_is_the_stokes_coupling():
    """With the velocity's own basis as the second basis the mixed functions are the
    equal-order coupling, bit for bit (the same sums in the same order)."""
    mesh = meshgen.structured_hex(2, 2, 1, 2, 0.15, 9)
    ref = oracle.RefElement(2, 3)
    wdetJ, G, _ = oracle.geometry(mesh.coords, mesh.conn, ref)
    np.testing.assert_array_equal(oracle.matrix_stokes_mixed(wdetJ, G, ref.phi),
                                  oracle.matrix_stokes(wdetJ, G, ref.phi))
    rng = np.random.default_rng(6)
    p, u = rng.standard_normal(mesh.n_nodes), rng.standard_normal(3 * mesh.n_nodes)
    np.testing.assert_array_equal(oracle.residual_stokes_mixed(mesh.conn, wdetJ, G, ref.phi, p),
                                  oracle.residual_stokes(mesh.conn, wdetJ, G, ref.phi, p))
    np.testing.assert_array_equal(oracle.residual_stokes_t_mixed(mesh.conn, wdetJ, G, ref.phi, u),
                                  oracle.residual_stokes_t(mesh.conn, wdetJ, G, ref.phi, u))


@pytest.mark.parametrize("kind", ["Q2/Q1", "P2/P1"])
def test_mixed_order_stokes_invariants_on_distorted_meshes(kind):
    """Distorted Q2 hexahedra and Delaunay P2 tetrahedra with the order-1 pressure on
    their vertices: sum_a B[(i,a), b] = 0 (sum_a d_i phi_a = 0); for a linear
    velocity u = A x + c, div u = tr A, so the transposed residual sums to tr A times
    the element volume (the basis psi sums to one, the rules integrate w det J
    exactly), and on straight-sided tetrahedra each entry is tr A V_e / 4; r = B p_e
    and r_T = B^T u_e."""
    if kind == "Q2/Q1":
        mesh = meshgen.structured_hex(3, 2, 2, 2, 0.15, 10)
        ref_u, ref_p = oracle.RefElement(2, 3), oracle.RefElement(1, 3)
    else:
        mesh = meshgen.tet_mesh(40, 2, np.random.default_rng(11))
        ref_u, ref_p = oracle.RefTet(2, 2), oracle.RefTet(1, 2)
    conn_p, n_p = meshgen.vertex_connectivity(mesh)
    wdetJ, G, _ = oracle.geometry(mesh.coords, mesh.conn, ref_u)
    B = oracle.matrix_stokes_mixed(wdetJ, G, ref_p.phi)
    E, N = mesh.n_elems, ref_u.N
    scale = np.abs(B).max()
    assert np.abs(B.reshape(E, 3, N, -1).sum(2)).max() <= 1e-13 * scale * N
    rng = np.random.default_rng(12)
    A, c = rng.standard_normal((3, 3)), rng.standard_normal(3)
    u = (mesh.coords @ A.T + c).ravel()
    rt = oracle.residual_stokes_t_mixed(mesh.conn, wdetJ, G, ref_p.phi, u)
    vol = wdetJ.sum(1)
    np.testing.assert_allclose(rt.sum(1), np.trace(A) * vol, rtol=1e-12, atol=1e-14)
    if kind == "P2/P1":
        np.testing.assert_allclose(rt, np.repeat(np.trace(A) * vol[:, None] / 4, 4, 1), rtol=1e-11, atol=1e-14)
    ue = u.reshape(-1, 3)[mesh.conn].transpose(0, 2, 1).reshape(E, 3 * N)
    np.testing.assert_allclose(rt, np.einsum("erb,er->eb", B, ue), rtol=1e-12, atol=1e-13 * np.abs(rt).max())
    p = rng.standard_normal(n_p)
    rs = oracle.residual_stokes_mixed(conn_p, wdetJ, G, ref_p.phi, p)
    np.testing.assert_allclose(rs, np.einsum("erb,eb->er", B, p[conn_p]), rtol=1e-12, atol=1e-13 * np.abs(rs).max())
