"""Differentiable slab functional: torch.autograd.Function around the libstm forward and adjoint solves.

One Newton step from a fixed linearisation point w solves J(w; nu) X = b(U, nu) + c(w, w) (Problem 3.1,
Eq. linNewEq); the drag-like functional is J(X) = j . X (velocity integrated over the wake region and
the slab). The backward pass solves the adjoint system J^T lambda = j with the same hierarchy
(transposed SpMV, transposed cell inverses, P / P^T, transposed coarse inverse) and returns
  dJ/dU = lambda . db/dU,   dJ/dnu = lambda . (db/dnu - (dJ/dnu) X),
both formed inside libstm (stm_adjoint_gradient). Every vector operation runs in libstm; this module
only sequences the calls.
"""
from __future__ import annotations

import torch

from .solver import Hierarchy


class SlabFunctional:
    """Hierarchy + fixed linearisation point + functional weights; re-factors when nu changes."""

    def __init__(self, hier: Hierarchy, X_lin: torch.Tensor, wake_lo, wake_hi, rtol=1e-12, restart=30,
                 max_iter=1000):
        self.h = hier
        self.X_lin = X_lin
        self.rtol, self.restart, self.max_iter = rtol, restart, max_iter
        self.j = torch.empty_like(X_lin)
        self._nu = None
        self.last_info = {}
        hier.assemble_jacobian(X_lin)
        hier.functional_weights(wake_lo, wake_hi, self.j)

    def prepare(self, nu: float):
        if self._nu != nu:
            self.h.assemble_jacobian(self.X_lin, nu=nu)
            self.h.factor_cells()
            self._nu = nu

    def solve(self, b, transpose=False):
        x = torch.zeros_like(b)
        info = self.h.gmres_solve(b, x, rtol=self.rtol, restart=self.restart, max_iter=self.max_iter,
                                  transpose=transpose)
        self.last_info["adjoint" if transpose else "forward"] = info
        return x

    def value_and_state(self, U: float, nu: float):
        self.prepare(nu)
        b = torch.empty_like(self.X_lin)
        self.h.assemble_load(U, nu, b, w=self.X_lin)
        X = self.solve(b)
        return self.h.dot(self.j, X), X

    def gradient(self, U: float, nu: float, X: torch.Tensor):
        self.prepare(nu)
        gU, gnu, info = self.h.adjoint_gradient(U, nu, self.j, X, rtol=self.rtol, restart=self.restart,
                                                max_iter=self.max_iter)
        self.last_info["adjoint"] = info
        return gU, gnu


class GMGSolveFunctional(torch.autograd.Function):
    """J = GMGSolveFunctional.apply(U, nu, slab_functional) with U, nu scalar tensors."""

    @staticmethod
    def forward(ctx, U, nu, sf: SlabFunctional):
        Uv, nuv = float(U), float(nu)
        value, X = sf.value_and_state(Uv, nuv)
        ctx.sf, ctx.U, ctx.nu = sf, Uv, nuv
        ctx.X = X
        return torch.tensor(value, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_out):
        gU, gnu = ctx.sf.gradient(ctx.U, ctx.nu, ctx.X)
        g = float(grad_out)
        return (torch.tensor(g * gU, dtype=torch.float64), torch.tensor(g * gnu, dtype=torch.float64), None)
