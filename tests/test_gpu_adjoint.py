"""GPU parity of the adjoint of the assembled elasticity residual: the
fe_eval_residual_adjoint kernel against the oracle's per-element terms, and the
torch.autograd path (J = |R|^2 / 2) against the oracle gradient and central
differences."""
import numpy as np
import pytest

import oracle
from paper_2107_04121_gb300 import fe, meshgen
from tests.parity import TOL, Problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(libfe):
    c = fe.Context(0)
    yield c
    c.close()


def _t(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("p,nq,n", [(1, 2, (5, 4, 3)), (2, 3, (3, 3, 4)), (2, 4, (2, 3, 2)), (3, 4, (2, 2, 3))])
def test_adjoint_kernel_matches_oracle(ctx, p, nq, n, prec):
    mesh = meshgen.structured_hex(*n, p, 0.15, 60 + p)
    lam, mu = meshgen.lame_materials(mesh)
    u = meshgen.normal_dofs(mesh, 3)
    rbar = np.random.default_rng(61).standard_normal(3 * mesh.n_nodes)
    P = Problem(ctx, mesh, p, nq)
    wdetJ, G, _ = P.oracle_geometry()
    dl, dm, dx = oracle.adjoint_elasticity_terms(mesh.conn, wdetJ, G, lam, mu, u, rbar)
    dt = torch.float64 if prec == "f64" else torch.float32
    form = fe.elasticity_form(fe.MAT_LAME)
    mat = _t(np.stack([lam, mu], 1), torch.float64)
    d_mat, d_xe = fe.eval_residual_adjoint(ctx, form, P.geom, [mat, None, _t(u, dt)], _t(rbar, dt), prec)
    ctx.check()
    d_mat = d_mat.cpu().numpy()
    assert _rel(d_mat[:, 0], dl) <= TOL[prec]
    assert _rel(d_mat[:, 1], dm) <= TOL[prec]
    assert _rel(d_xe.cpu().numpy(), dx) <= TOL[prec]


def _objective_setup(ctx, n, precision):
    from paper_2107_04121_gb300 import autograd as fad
    mesh, lam, mu, u = meshgen.elasticity_q2_cube(n, seed=4, perturb=0.1)
    X = _t(mesh.coords, torch.float64)
    conn = _t(mesh.conn, torch.int32)
    prob = fad.ElasticityProblem(ctx, X, conn, 2, 3, precision)
    dt = prob.dtype
    lam_t = _t(lam, dt).requires_grad_()
    mu_t = _t(mu, dt).requires_grad_()
    u_t = _t(u, dt).requires_grad_()
    X.requires_grad_()

    def J():
        R = fad.assembled_elasticity_residual(prob, lam_t, mu_t, X, u_t)
        return 0.5 * (R.double() * R.double()).sum()

    return mesh, lam, mu, u, prob, lam_t, mu_t, X, u_t, J


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_autograd_gradient_matches_oracle_gradient(ctx, precision):
    """32^3 Q2 cube (32,768 hexes, +-0.1h, seed 4): the gradients of
    J = |R|^2 / 2 from loss.backward() against the oracle's."""
    mesh, lam, mu, u, prob, lam_t, mu_t, X, u_t, J = _objective_setup(ctx, 32, precision)
    loss = J()
    loss.backward()
    ctx.check()
    ref = oracle.RefElement(2, 3)
    Jref, dl, dm, dX = oracle.elasticity_objective_gradient(mesh.coords, mesh.conn, ref, lam, mu, u)
    tol = TOL[precision]
    assert abs(loss.item() - Jref) <= tol * Jref
    assert _rel(lam_t.grad.cpu().numpy(), dl) <= tol
    assert _rel(mu_t.grad.cpu().numpy(), dm) <= tol
    assert _rel(X.grad.cpu().numpy(), dX) <= tol


def test_autograd_gradient_matches_central_differences(ctx):
    """FP64 path, 32^3: central differences with h = 1e-6 in 50 seeded unit
    directions per parameter group (lambda, mu, X, u).  J is quadratic in
    lambda, mu and u (R is linear in each), so there the difference is exact up
    to rounding; in X it is second-order accurate."""
    mesh, lam, mu, u, prob, lam_t, mu_t, X, u_t, J = _objective_setup(ctx, 32, "f64")
    loss = J()
    loss.backward()
    grads = {"lam": lam_t.grad.clone(), "mu": mu_t.grad.clone(), "X": X.grad.clone(), "u": u_t.grad.clone()}
    params = {"lam": lam_t, "mu": mu_t, "X": X, "u": u_t}
    rng = np.random.default_rng(4)
    h = 1e-6
    for name, t in params.items():
        g = grads[name]
        worst = 0.0
        for _ in range(50):
            d = _t(rng.standard_normal(tuple(t.shape)), torch.float64)
            d /= d.norm()
            with torch.no_grad():
                t += h * d
                Jp = J().item()
                t -= 2 * h * d
                Jm = J().item()
                t += h * d
            fd = (Jp - Jm) / (2 * h)
            an = float((g * d).sum())
            worst = max(worst, abs(fd - an) / g.norm().item())
        assert worst <= 1e-6, (name, worst)
    ctx.check()


def test_adjoint_rejections(ctx):
    mesh = meshgen.structured_hex(2, 2, 2, 2, 0.1, 3)
    P = Problem(ctx, mesh, 2, 3)
    u = _t(np.zeros(3 * mesh.n_nodes), torch.float32)
    mat = _t(np.ones((mesh.n_elems, 2)), torch.float64)
    form = fe.elasticity_form(fe.MAT_LAME)
    for prec in ("tf32x3", "bf16x3"):
        with pytest.raises(fe.FEError) as ei:
            fe.eval_residual_adjoint(ctx, form, P.geom, [mat, None, u], u, prec)
        assert ei.value.status in (fe.FE_ERR_UNSUPPORTED_SPEC, fe.FE_ERR_INVALID_ARG)
    lap = fe.laplace_form()
    us = _t(np.zeros(mesh.n_nodes), torch.float32)
    with pytest.raises(fe.FEError) as ei:
        fe.eval_residual_adjoint(ctx, lap, P.geom, [None, us], u, "f32")
    assert ei.value.status == fe.FE_ERR_UNSUPPORTED_SPEC
