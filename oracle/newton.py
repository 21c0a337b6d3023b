"""Oracle, part 4: the nonlinear slab problem, damped Newton and time marching (TEST INFRASTRUCTURE ONLY).

Sec. 3 writes the fully discrete slab problem as F_n(X) = 0 (Eq. nonlineq) and solves it by
Newton's method with the Jacobian J = dF/dX (Eqs. linNewEq, definition_jacobian_global, linNewEqU),
damped by a line search. With the data of the adjoint workload (f = 0, inflow g = U g_1, previous
slab value U g_1 e_x):
    F(X) = A X + c(X, X) - b(U, nu),
  A       the linear part of the slab operator: the Jacobian at w = 0 (time derivative, viscous and
          Nitsche terms, pressure coupling),
  c(X, X) the convection term int_{I_n} <(v . grad) v, psi> dt, quadratic in X,
  b       the load of Problem 3.1 (inflow Nitsche data and the previous-slab term).
Its Jacobian at X is J(X) = A + N(X) with N the Newton linearisation of c.

Newton step m: solve J(X^m) D = -F(X^m), then X^{m+1} = X^m + lambda D with the first lambda in
1, 1/2, 1/4, ... (at most `max_halvings` halvings) that decreases ||F||_2 (the paper does not print
its line search; this is the plain backtracking reading). Stop when ||F|| <= abs_tol or
||F|| <= ||F(X^0)|| / reduction, the criterion of Sec. 5.1 (1e-10 or a reduction by 1e4).
The linear systems go to the oracle's GMG-preconditioned FGMRES on a hierarchy built at X^m
(coarse levels take X^m at their own nodes), or to a sparse LU.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import adjoint, fem, solvers


def lattice_from_dofs(level: fem.Level, X):
    """Inverse of Level.dofs_from_lattice: the lattice state [k+1, d*P + n_p*Cf] of a DoF vector
    (removed lattice points and cells are zero)."""
    d, K = level.dim, level.k + 1
    out = np.zeros((K, d * level.P + level.np_ * int(np.prod(level.cells))))
    for l in range(K):
        for i in range(d):
            out[l, i * level.P + level.lat_of_node] = X[l * level.block + i * level.R:
                                                        l * level.block + (i + 1) * level.R]
        pcol = d * level.P + (level.active_full[:, None] * level.np_ + np.arange(level.np_)).ravel()
        out[l, pcol] = X[l * level.block + d * level.R:(l + 1) * level.block]
    return out


def inflow_load(level: fem.Level, U, nu, tau, gamma1=35.0, gamma2=35.0):
    """The inflow part of the load: int_{I_n} B_GamD(g, (psi, xi)) dt with g = U g_1 e_x on x = 0 and
    g = 0 on the walls and the obstacle (Eqs. Def:Lh, Def:B_GamD)."""
    d = level.dim

    def g(pts, t):
        out = np.zeros((pts.shape[0], d))
        on_inflow = np.abs(pts[:, 0]) < 1e-12
        out[:, 0] = np.where(on_inflow, U * adjoint.inflow_profile(pts, level.length), 0.0)
        return out

    return fem.assemble_load(level, tau, nu, gamma1, gamma2, g=g)


def prev_slab_load(level: fem.Level, X_prev):
    """<v_h(t_{n-1}^-), psi(t_{n-1}^+)> for a discrete previous slab (Problem 3.1): the right Radau
    nodes end at the slab end, so v_h(t_{n-1}^-) is the velocity of the previous slab's last time node;
    entry (a, l, i) = chi_a(0) (M v_l)_i with the Q2 mass matrix M."""
    d, k = level.dim, level.k
    rt = fem.ref_tables(d)
    Mloc = float(np.prod(level.h)) * np.einsum("q,qi,qj->ij", rt.Wq, rt.phi, rt.phi)
    chi0 = fem.lagrange_time(k, np.array([0.0]))[0][:, 0]
    vend = level.velocity_nodal(X_prev)[k]  # [d, R]
    out = np.zeros(level.N)
    for l in range(d):
        mv = np.zeros(level.R)
        np.add.at(mv, level.cell_nodes.ravel(), (vend[l][level.cell_nodes] @ Mloc.T).ravel())
        for a in range(k + 1):
            out[a * level.block + l * level.R:a * level.block + (l + 1) * level.R] += chi0[a] * mv
    return out


class SlabProblem:
    """F and its pieces on one level for fixed (U, nu). X_prev: the previous slab's DoF vector (its
    last time node is the initial value); None: the Poiseuille field U g_1 e_x."""

    def __init__(self, level: fem.Level, U, nu, tau, gamma1=35.0, gamma2=35.0, X_prev=None):
        self.level, self.U, self.nu, self.tau = level, U, nu, tau
        self.gamma1, self.gamma2 = gamma1, gamma2
        self.A = fem.assemble_jacobian(level, np.zeros(level.N), tau, nu, gamma1, gamma2)
        if X_prev is None:
            self.b = adjoint.newton_rhs(level, None, U, nu, tau, gamma1, gamma2, with_convection=False)
        else:
            self.b = inflow_load(level, U, nu, tau, gamma1, gamma2) + prev_slab_load(level, X_prev)

    def residual(self, X):
        """F(X) = A X + c(X, X) - b."""
        return self.A @ X + fem.convection_residual(self.level, X, self.tau) - self.b

    def jacobian(self, X):
        return fem.assemble_jacobian(self.level, X, self.tau, self.nu, self.gamma1, self.gamma2)


def newton_solve(wl, X0, U, nu=None, linear="gmg", lin_rtol=1e-10, abs_tol=1e-10, reduction=1e4,
                 max_newton=20, max_halvings=8, X_prev=None):
    """Damped Newton for F(X) = 0 on the finest level of workload `wl`, from X0.

    Returns (X, info) with info = {"res": [||F(X^m)|| for m = 0..], "lam": [lambda_m],
    "gmres_iters": [per step], "converged": bool}.
    """
    nu = wl.nu if nu is None else nu
    f = 2 ** (wl.n_levels - 1)
    fine = fem.Level(wl.dim, wl.k, wl.fine_cells, wl.length, tuple(x * f for x in wl.obstacle_lo),
                     tuple(x * f for x in wl.obstacle_hi))
    prob = SlabProblem(fine, U, nu, wl.tau, wl.gamma1, wl.gamma2, X_prev=X_prev)
    X = np.array(X0, dtype=np.float64)
    F = prob.residual(X)
    res = [float(np.linalg.norm(F))]
    lams, its = [], []
    target = max(abs_tol, res[0] / reduction)
    converged = res[0] <= target
    for _ in range(max_newton):
        if converged:
            break
        if linear == "gmg":
            H = solvers.Hierarchy(wl, lattice_from_dofs(fine, X), nu=nu)
            D, inf = H.solve(-F, rtol=lin_rtol)
            its.append(int(inf["iters"]))
        else:
            D = spla.spsolve(prob.jacobian(X).tocsc(), -F)
            its.append(0)
        lam = 1.0
        for _h in range(max_halvings + 1):
            Xt = X + lam * D
            Ft = prob.residual(Xt)
            rt = float(np.linalg.norm(Ft))
            if rt < res[-1] or _h == max_halvings:
                break
            lam *= 0.5
        X, F = Xt, Ft
        res.append(rt)
        lams.append(lam)
        converged = rt <= target
    return X, {"res": res, "lam": lams, "gmres_iters": its, "converged": converged, "level": fine}


def time_march(wl, X_init, U, n_slabs, j=None, **newton_kw):
    """Slabs I_1 .. I_n in sequence (Problem 3.1): slab n starts from the last time node of slab n-1
    (X_init for n = 1), each solved by newton_solve from the previous slab's state. Returns the slab
    states and, with weights j, the functional history j . X_n."""
    states, values, infos = [], [], []
    X_prev = np.array(X_init, dtype=np.float64)
    for _ in range(n_slabs):
        X, info = newton_solve(wl, X_prev, U, X_prev=X_prev, **newton_kw)
        states.append(X)
        infos.append(info)
        if j is not None:
            values.append(float(j @ X))
        X_prev = X
    return states, values, infos
