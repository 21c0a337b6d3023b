"""Oracle, part 2: cell inverses, Vanka smoothers, V-cycle and flexible GMRES (TEST INFRASTRUCTURE).

All arithmetic is FP64 and follows the paper's statements step by step:
  * cell matrices J_T = J[idx_T, idx_T] are restrictions of the ASSEMBLED global Jacobian
    (Sec. 4.4: the entries of J on the cell's DoFs), inverted explicitly (Sec. 4.3, LAPACK LU);
  * the local Vanka update S_T(d, r) = d_T + omega J_T^{-1} (r - J d)_T (Eq. LocVanka with the
    damping of Sec. 5.3), taken over all k+1 time nodes of the cell;
  * the V-cycle of Algorithm 1 with a direct coarse solve on level 1 and transfer P / P^T (Sec. 4.1);
  * right-preconditioned flexible GMRES (Sec. 3) with modified Gram-Schmidt and Givens rotations.

Readings of points where the paper is silent or garbled (each also listed in the design notes):
  * Eq. LocVanka uses r_0 (r with pressure rows zeroed, Eq. defr0); the smoother here uses the full
    residual r - J d, whose fixed point is J^{-1} r (`literal_r0=True` gives the printed variant).
  * Shared velocity DoFs (Sec. 4.2 "last update wins") are combined three ways: multiplicity-
    weighted additive (default), 2^d-colour multiplicative, and the literal overwrite in which the
    cell with the highest index wins.
  * Algorithm 1 computes t = r_g - J_g d_g into a separate vector, prolongates the coarse-grid
    correction d_{g-1}, and post-smooths against the original r_g.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem

ADDITIVE, COLOURED, OVERWRITE = "additive", "coloured", "overwrite"


# ----------------------------------------------------------------------------------------------
# Cell matrices and inverses (Sec. 4.3, Sec. 4.4)
# ----------------------------------------------------------------------------------------------
def cell_matrices(J: sp.csr_matrix, idx, cells=None):
    """J_T = J[idx_T, idx_T] for the given cells: [nc, n, n]."""
    cells = np.arange(idx.shape[0]) if cells is None else np.asarray(cells)
    Jc = J.tocsr()
    out = np.zeros((cells.size, idx.shape[1], idx.shape[1]))
    for c_i, c in enumerate(cells):
        out[c_i] = Jc[idx[c]][:, idx[c]].toarray()
    return out


def cell_inverses(J, idx, cells=None):
    """Explicit inverses J_T^{-1} by LU with partial pivoting (LAPACK getrf/getri via numpy)."""
    return np.linalg.inv(cell_matrices(J, idx, cells))


def multiplicity(level: fem.Level):
    """m_i = number of cells whose local DoF set contains global DoF i."""
    m = np.zeros(level.N)
    np.add.at(m, level.idx.ravel(), 1.0)
    return m


# ----------------------------------------------------------------------------------------------
# Vanka smoothing step (Sec. 4.2, Eq. LocVanka; damping Sec. 5.3)
# ----------------------------------------------------------------------------------------------
def vanka_step(level, J, inv, d, r, omega, variant=ADDITIVE, transpose=False, literal_r0=False):
    """One sweep of the cell-based space-time Vanka smoother; returns the new d.

    additive : d + omega W sum_T R_T^T J_T^{-1} R_T (r - J d),  W = diag(1/m_i)
    coloured : for each colour c = 0..2^d-1:  t = r - J d;  d_T += omega J_T^{-1} t_T  for T in c
    overwrite: t = r - J d once; for T in increasing index order d_new[idx_T] = d[idx_T] +
               omega (J_T^{-1} t_T), each write replacing earlier ones (Sec. 4.2, last write wins)
    transpose=True smooths for J^T with (J_T)^{-T}.
    """
    A = J.T.tocsr() if transpose else J
    Ainv = np.transpose(inv, (0, 2, 1)) if transpose else inv
    idx = level.idx
    rr = _r0(level, r) if literal_r0 else r
    if variant == ADDITIVE:
        t = rr - A @ d
        y = np.einsum("cij,cj->ci", Ainv, t[idx])
        corr = np.zeros_like(d)
        np.add.at(corr, idx.ravel(), y.ravel())
        return d + omega * corr / multiplicity(level)
    if variant == COLOURED:
        d = d.copy()
        for col in range(2**level.dim):
            t = rr - A @ d
            for c in np.nonzero(level.colour == col)[0]:
                d[idx[c]] += omega * Ainv[c] @ t[idx[c]]
        return d
    if variant == OVERWRITE:
        t = rr - A @ d
        out = d.copy()
        for c in range(level.C):
            out[idx[c]] = d[idx[c]] + omega * Ainv[c] @ t[idx[c]]
        return out
    raise ValueError(variant)


def _r0(level, r):
    """Eq. defr0: r with every pressure component set to zero."""
    r0 = r.copy()
    for l in range(level.k + 1):
        r0[l * level.block + level.dim * level.R:(l + 1) * level.block] = 0.0
    return r0


# ----------------------------------------------------------------------------------------------
# Hierarchy, V-cycle (Algorithm 1) and FGMRES (Sec. 3)
# ----------------------------------------------------------------------------------------------
class Hierarchy:
    """Levels 0 (coarsest) .. G-1 (finest), Jacobians on every level, transfers, cell inverses."""

    def __init__(self, wl, state_fine, nu=None, variant=ADDITIVE, with_inverses=True):
        self.wl = wl
        self.nu = wl.nu if nu is None else nu
        self.variant = variant
        self.levels = []
        for g in range(1, wl.n_levels + 1):
            f = 2 ** (g - 1)
            cells = wl.cells_at(g)
            lo = tuple(x * f for x in wl.obstacle_lo)
            hi = tuple(x * f for x in wl.obstacle_hi)
            self.levels.append(fem.Level(wl.dim, wl.k, cells, wl.length, lo, hi))
        fine_cells = wl.fine_cells
        self.X_lin = []
        self.J = []
        for lev in self.levels:
            st = fem.fine_lattice_to_level(state_fine, fine_cells, lev)
            X = lev.dofs_from_lattice(st)
            self.X_lin.append(X)
            self.J.append(fem.assemble_jacobian(lev, X, wl.tau, self.nu, wl.gamma1, wl.gamma2))
        self.P = [None] + [fem.prolongation(self.levels[g - 1], self.levels[g])
                           for g in range(1, len(self.levels))]
        self.inv = [None] * len(self.levels)
        if with_inverses:
            for g in range(1, len(self.levels)):
                self.inv[g] = cell_inverses(self.J[g], self.levels[g].idx)
        self.coarse_lu = spla.splu(self.J[0].tocsc())

    @property
    def fine(self):
        return self.levels[-1]

    def coarse_solve(self, r, transpose=False):
        """d_1 = J_1^{-1} r_1 (Algorithm 1, direct coarse solver)."""
        return self.coarse_lu.solve(r, trans="T" if transpose else "N")

    def vcycle(self, r, g=None, transpose=False):
        """Algorithm 1, Multigrid(0, r_g, g), with V(nu1, nu2) smoothing; returns d_g."""
        g = len(self.levels) - 1 if g is None else g
        if g == 0:
            return self.coarse_solve(r, transpose)
        lev, J = self.levels[g], self.J[g]
        A = J.T.tocsr() if transpose else J
        d = np.zeros_like(r)
        for _ in range(self.wl.nu1):
            d = vanka_step(lev, J, self.inv[g], d, r, self.wl.omega, self.variant, transpose)
        t = r - A @ d
        rc = self.P[g].T @ t
        dc = self.vcycle(rc, g - 1, transpose)
        d = d + self.P[g] @ dc
        for _ in range(self.wl.nu2):
            d = vanka_step(lev, J, self.inv[g], d, r, self.wl.omega, self.variant, transpose)
        return d

    def solve(self, b, rtol=None, restart=None, maxit=1000, transpose=False, x0=None):
        A = self.J[-1].T.tocsr() if transpose else self.J[-1]
        return fgmres(lambda v: A @ v, lambda v: self.vcycle(v, transpose=transpose), b,
                      x0=x0, restart=self.wl.restart if restart is None else restart,
                      rtol=self.wl.rtol if rtol is None else rtol, maxit=maxit)


def fgmres(matvec, precond, b, x0=None, restart=30, rtol=1e-10, maxit=1000):
    """Right-preconditioned flexible GMRES(restart) with modified Gram-Schmidt (Sec. 3).

    Stops when the recurrence residual |g_{j+1}| <= rtol ||b||_2 (then recomputes the true
    residual) or after maxit iterations. Restarts from the true residual.
    Returns (x, info) with info = dict(iters, restarts, rel_res_true, converged, history).
    """
    n = b.size
    x = np.zeros(n) if x0 is None else x0.copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros(n), dict(iters=0, restarts=0, rel_res_true=0.0, converged=True, history=[])
    tol = rtol * bnorm
    it, restarts, history = 0, 0, []
    while True:
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        history.append(beta / bnorm)
        if beta <= tol or it >= maxit:
            return x, dict(iters=it, restarts=restarts, rel_res_true=beta / bnorm,
                           converged=beta <= tol, history=history)
        V = np.zeros((restart + 1, n))
        Z = np.zeros((restart, n))
        H = np.zeros((restart + 1, restart))
        cs, sn = np.zeros(restart), np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        converged = False
        for j in range(restart):
            Z[j] = precond(V[j])
            w = matvec(Z[j])
            for i in range(j + 1):
                H[i, j] = V[i] @ w
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                hi, hi1 = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * hi + sn[i] * hi1
                H[i + 1, j] = -sn[i] * hi + cs[i] * hi1
            rho = math.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / rho, H[j + 1, j] / rho
            H[j, j] = rho
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            j_done = j + 1
            history.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= tol or it >= maxit:
                converged = abs(g[j + 1]) <= tol
                break
        y = sla.solve_triangular(H[:j_done, :j_done], g[:j_done])
        x = x + Z[:j_done].T @ y
        restarts += 1
        if converged or it >= maxit:
            r = b - matvec(x)
            rel = np.linalg.norm(r) / bnorm
            return x, dict(iters=it, restarts=restarts - 1, rel_res_true=rel,
                           converged=converged, history=history)
