"""Differentiable evaluation through torch.autograd: the assembled elasticity
residual R(u; lambda, mu, X) as a torch.autograd.Function whose backward runs
the library's adjoint kernel (fe_eval_residual_adjoint) and assembly.

The forward evaluates the FP64 geometry of the current node coordinates X, the
element residuals (Algorithm 1 of Cimrman, arXiv 2107.04121, form
'IK,s(i:j)->I,s(k:l)->K') and their assembly.  The backward recomputes the
geometry from X instead of keeping it from the forward, then maps the incoming
gradient Rbar = dL/dR to
  dL/dlambda_e, dL/dmu_e  (per element)      adjoint kernel, material terms
  dL/dX (n_nodes, 3)                         adjoint kernel + assembly (shape derivative)
  dL/du                                      K^T Rbar = assembled residual of Rbar (K is symmetric)
PyTorch supplies memory and the autograd graph; every step runs in libfe."""
from __future__ import annotations

import torch

from . import fe


class ElasticityProblem:
    """A hex mesh whose node coordinates X (a float64 CUDA tensor, (n_nodes, 3))
    are read by the geometry handle in place: changing X and evaluating again
    (or differentiating) uses the new coordinates."""

    def __init__(self, ctx: fe.Context, X: torch.Tensor, conn: torch.Tensor, p: int = 2, nq: int = 3,
                 precision: str = "f64"):
        if X.dtype != torch.float64 or not X.is_cuda or not X.is_contiguous():
            raise ValueError("X must be a contiguous float64 CUDA tensor")
        if precision not in ("f64", "f32"):
            raise ValueError("precision must be f64 or f32")
        self.ctx, self.X, self.precision = ctx, X, precision
        self.conn = conn
        self.mesh = fe.Mesh(X, conn)
        # float32: a deferred handle, whose geometry the first residual of each
        # evaluation computes in the same kernel (fe_eval_residual)
        flags = fe.GEOM_STORE_F64 if precision == "f64" else fe.GEOM_STORE_F32 | fe.GEOM_DEFERRED
        self.geom = fe.hex_geometry(ctx, self.mesh, p, nq, flags=flags)
        self.form = fe.elasticity_form(fe.MAT_LAME)
        self.asm = fe.assembly_create(ctx, self.mesh)
        self.dtype = torch.float64 if precision == "f64" else torch.float32

    def _assemble(self, r_e):
        flags = 0 if self.precision == "f64" else fe.ASSEMBLE_COMPENSATED
        return fe.assemble_vector(self.ctx, self.asm, 3, r_e, self.precision, flags=flags)

    def residual(self, lam, mu, u):
        """R (n_nodes * 3) for the current X, without autograd."""
        self.geom.update()
        mat = torch.stack([lam.detach(), mu.detach()], 1).to(torch.float64).contiguous()
        r = fe.eval_residual(self.ctx, self.form, self.geom, [mat, None, u.detach().to(self.dtype).contiguous()],
                             self.precision)
        return self._assemble(r)


class AssembledElasticityResidual(torch.autograd.Function):
    @staticmethod
    def forward(fctx, lam, mu, X, u, prob: ElasticityProblem):
        if X.data_ptr() != prob.X.data_ptr():
            raise ValueError("X must be the coordinate tensor the problem was built on")
        R = prob.residual(lam, mu, u)
        fctx.prob = prob
        fctx.save_for_backward(lam, mu, u)
        return R

    @staticmethod
    def backward(fctx, Rbar):
        prob = fctx.prob
        lam, mu, u = fctx.saved_tensors
        need_mat = fctx.needs_input_grad[0] or fctx.needs_input_grad[1]
        need_x = fctx.needs_input_grad[2]
        need_u = fctx.needs_input_grad[3]
        rbar = Rbar.detach().to(prob.dtype).contiguous()
        mat = torch.stack([lam.detach(), mu.detach()], 1).to(torch.float64).contiguous()
        ud = u.detach().to(prob.dtype).contiguous()
        prob.geom.update()  # the geometry is recomputed, not kept from the forward
        dlam = dmu = dX = du = None
        if need_u:
            # first, so that (float32) this residual computes the geometry that the
            # adjoint kernel then reads
            r = fe.eval_residual(prob.ctx, prob.form, prob.geom, [mat, None, rbar], prob.precision)
            du = prob._assemble(r).to(u.dtype)
        if need_mat or need_x:
            d_mat, d_xe = fe.eval_residual_adjoint(prob.ctx, prob.form, prob.geom, [mat, None, ud], rbar,
                                                   prob.precision, want_mat=need_mat, want_x=need_x)
            if need_mat:
                dlam = d_mat[:, 0].to(lam.dtype)
                dmu = d_mat[:, 1].to(mu.dtype)
            if need_x:
                dX = prob._assemble(d_xe).view(-1, 3).to(prob.X.dtype)
        return dlam, dmu, dX, du, None


def assembled_elasticity_residual(prob: ElasticityProblem, lam, mu, X, u):
    """R(u; lambda, mu, X), differentiable in lambda, mu, X and u."""
    return AssembledElasticityResidual.apply(lam, mu, X, u, prob)
