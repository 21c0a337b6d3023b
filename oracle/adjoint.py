"""Oracle, part 3: one Newton step from a fixed linearisation point and its adjoint gradients
(TEST INFRASTRUCTURE ONLY).

With w fixed, the slab state after one Newton step solves J(w; nu) X = b(U, nu) + c(w, w):
  * b(U, nu) is the right-hand side of Problem 3.1 with f = 0 (Eqs. Def:Lh and Def:B_GamD): the Nitsche
    terms of the inflow data g = U g_1 on x = 0 (zero on walls and obstacle) plus the previous-slab
    term <v(t_{n-1}^-), psi(t_{n-1}^+)> with v(t_{n-1}^-) = U g_1 e_x (Poiseuille field);
  * c(w, w) is the convection term at w, so that J(w) X = b + c is exactly one Newton step
    (Eq. linNewEq with X^{m+1} = X^m + D).
The functional is J(X) = int_{I_n} int_wake v_1 dx dt = j . X. Gradients by the adjoint:
  J^T lambda = j,  dJ/dU = lambda . db/dU,  dJ/dnu = lambda . (db/dnu - (dJ/dnu) X).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import fem


def inflow_profile(x, length):
    """Poiseuille profile g_1: 4y(H-y)/H^2 in 2D, 16 y(H-y) z(L-z)/(H^2 L^2) in 3D."""
    H = length[1]
    g = 4.0 * x[:, 1] * (H - x[:, 1]) / H**2
    if x.shape[1] == 3:
        L2 = length[2]
        g = g * 4.0 * x[:, 2] * (L2 - x[:, 2]) / L2**2
    return g


def newton_rhs(level: fem.Level, X_lin, U, nu, tau, gamma1=35.0, gamma2=35.0, with_convection=True):
    """b(U, nu) (+ c(w, w)) on `level`."""
    d = level.dim
    L = level.length

    def g(pts, t):
        out = np.zeros((pts.shape[0], d))
        on_inflow = np.abs(pts[:, 0]) < 1e-12
        out[:, 0] = np.where(on_inflow, U * inflow_profile(pts, L), 0.0)
        return out

    def v_prev(pts):
        out = np.zeros((pts.shape[0], d))
        out[:, 0] = U * inflow_profile(pts, L)
        return out

    b = fem.assemble_load(level, tau, nu, gamma1, gamma2, g=g, v_prev=v_prev)
    if with_convection:
        b = b + fem.convection_residual(level, X_lin, tau)
    return b


def db_dU(level, X_lin, nu, tau, gamma1=35.0, gamma2=35.0):
    return newton_rhs(level, X_lin, 1.0, nu, tau, gamma1, gamma2, with_convection=False)


def db_dnu(level, X_lin, U, tau, gamma1=35.0, gamma2=35.0):
    """b is affine in nu: db/dnu = b(U, 1) - b(U, 0) (convection part independent of nu)."""
    return (newton_rhs(level, X_lin, U, 1.0, tau, gamma1, gamma2, with_convection=False)
            - newton_rhs(level, X_lin, U, 0.0, tau, gamma1, gamma2, with_convection=False))


def functional_weights(level: fem.Level, wake_lo, wake_hi, tau):
    """j with j . X = int_{I_n} int_wake v_1 dx dt; wake = cells with lo <= index < hi (this level's units)."""
    rt = fem.ref_tables(level.dim)
    vol = float(np.prod(level.h))
    Mt, _, _ = fem.time_matrices(level.k, tau)
    tint = Mt.sum(axis=1)
    inside = np.ones(level.C, dtype=bool)
    for m in range(level.dim):
        inside &= (level.cell_xyz[:, m] >= wake_lo[m]) & (level.cell_xyz[:, m] < wake_hi[m])
    cell_int = vol * rt.Wq @ rt.phi  # int_T phi_i
    j = np.zeros(level.N)
    for a in range(level.k + 1):
        rows = a * level.block + level.cell_nodes[inside]
        np.add.at(j, rows.ravel(), np.broadcast_to(tint[a] * cell_int, rows.shape).ravel())
    return j


def dJ_dnu_apply(level, X_lin, tau, x, gamma1=35.0, gamma2=35.0):
    """(dJ/dnu) x; J is affine in nu, so dJ/dnu = J(nu = 1) - J(nu = 0)."""
    J1 = fem.assemble_jacobian(level, X_lin, tau, 1.0, gamma1, gamma2)
    J0 = fem.assemble_jacobian(level, X_lin, tau, 0.0, gamma1, gamma2)
    return J1 @ x - J0 @ x


def functional_direct(level, X_lin, U, nu, tau, j, gamma1=35.0, gamma2=35.0):
    """J(U, nu) = j . X with X from a direct sparse solve (used for finite differences)."""
    Jm = fem.assemble_jacobian(level, X_lin, tau, nu, gamma1, gamma2)
    X = spla.spsolve(Jm.tocsc(), newton_rhs(level, X_lin, U, nu, tau, gamma1, gamma2))
    return float(j @ X), X


def adjoint_gradient(level, X_lin, U, nu, tau, j, gamma1=35.0, gamma2=35.0, solve=None, solve_t=None):
    """(J, dJ/dU, dJ/dnu) by one forward and one adjoint solve (direct solves unless given)."""
    Jm = fem.assemble_jacobian(level, X_lin, tau, nu, gamma1, gamma2)
    b = newton_rhs(level, X_lin, U, nu, tau, gamma1, gamma2)
    X = spla.spsolve(Jm.tocsc(), b) if solve is None else solve(b)
    lam = spla.spsolve(Jm.T.tocsc(), j) if solve_t is None else solve_t(j)
    gU = lam @ db_dU(level, X_lin, nu, tau, gamma1, gamma2)
    gnu = lam @ (db_dnu(level, X_lin, U, tau, gamma1, gamma2) - dJ_dnu_apply(level, X_lin, tau, X, gamma1, gamma2))
    return float(j @ X), float(gU), float(gnu), X, lam
