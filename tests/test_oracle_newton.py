"""Pins of the oracle's nonlinear slab residual and damped Newton (Sec. 3, Eqs. nonlineq, linNewEq,
linNewEqU; stopping rule of Sec. 5.1)."""
import numpy as np
import pytest
from scipy import optimize

import synth
from helpers import poiseuille_state as _poiseuille_state
from oracle import adjoint, fem, newton


def _fine(wl):
    f = 2 ** (wl.n_levels - 1)
    return fem.Level(wl.dim, wl.k, wl.fine_cells, wl.length, tuple(x * f for x in wl.obstacle_lo),
                     tuple(x * f for x in wl.obstacle_hi))


def _start(wl, lev, amp=0.1):
    return lev.dofs_from_lattice(synth.linearisation_point(wl, amp=amp))


def test_residual_matches_jacobian_form():
    """F(X) = A X + c(X,X) - b equals J(X) X - c(X,X) - b, since J(X) = A + N(X) and N(X) X = 2 c(X,X)."""
    wl = synth.small_workload(2, 1, (4, 1), 2, obstacle=False)
    lev = _fine(wl)
    prob = newton.SlabProblem(lev, 0.3, wl.nu, wl.tau)
    rng = np.random.default_rng(3)
    X = rng.standard_normal(lev.N)
    F1 = prob.residual(X)
    F2 = prob.jacobian(X) @ X - fem.convection_residual(lev, X, wl.tau) - prob.b
    assert np.abs(F1 - F2).max() <= 1e-12 * np.abs(F1).max()


def test_residual_of_zero_state_is_minus_load():
    wl = synth.small_workload(2, 2, (4, 1), 2, obstacle=False)
    lev = _fine(wl)
    prob = newton.SlabProblem(lev, 0.3, wl.nu, wl.tau)
    assert np.array_equal(prob.residual(np.zeros(lev.N)), -prob.b)
    # b is linear in U (no source term): F(0; 2U) = 2 F(0; U)
    prob2 = newton.SlabProblem(lev, 0.6, wl.nu, wl.tau)
    assert np.abs(prob2.b - 2.0 * prob.b).max() <= 1e-14 * np.abs(prob.b).max()


def test_lattice_round_trip():
    wl = synth.small_workload(2, 1, (4, 1), 2, obstacle=True)
    lev = _fine(wl)
    X = np.random.default_rng(5).standard_normal(lev.N)
    assert np.array_equal(lev.dofs_from_lattice(newton.lattice_from_dofs(lev, X)), X)


def test_newton_root_matches_minpack():
    """The damped Newton iterate converges to the root that MINPACK's hybrid method finds from F alone."""
    wl = synth.small_workload(2, 1, (4, 1), 1, obstacle=False)
    lev = _fine(wl)
    X0 = _start(wl, lev)
    X, info = newton.newton_solve(wl, X0, 0.3, linear="lu", abs_tol=1e-13, reduction=1e30)
    assert info["converged"], info["res"]
    prob = newton.SlabProblem(lev, 0.3, wl.nu, wl.tau)
    sol = optimize.root(prob.residual, X0, method="hybr", options={"xtol": 1e-13})
    assert np.linalg.norm(prob.residual(sol.x)) < 1e-9
    assert np.abs(X - sol.x).max() <= 1e-8 * np.abs(X).max()


def test_newton_converges_quadratically():
    """From a far start (100x the synthetic perturbation) every step that starts below 0.1 satisfies
    ||F_{m+1}|| <= ||F_m||^2: a wrong Jacobian (a dropped or mis-signed term, Picard instead of
    Newton) converges only linearly and fails this once ||F_m|| is small."""
    wl = synth.small_workload(2, 1, (4, 1), 1, obstacle=False)
    lev = _fine(wl)
    X0 = _start(wl, lev, amp=10.0)
    _, info = newton.newton_solve(wl, X0, 0.3, linear="lu", abs_tol=1e-13, reduction=1e30)
    r = info["res"]
    assert info["converged"]
    checked = 0
    for m in range(len(r) - 1):
        if r[m] < 0.1 and r[m + 1] > 1e-14:
            assert r[m + 1] <= r[m] ** 2, r
            checked += 1
    assert checked >= 2, r
    assert all(lam == 1.0 for lam in info["lam"])


def test_stopping_rule():
    """Stop at the first iterate with ||F|| <= max(abs_tol, ||F_0|| / reduction) (Sec. 5.1)."""
    wl = synth.small_workload(2, 1, (4, 1), 1, obstacle=False)
    lev = _fine(wl)
    X0 = _start(wl, lev, amp=2.0)
    _, info = newton.newton_solve(wl, X0, 0.3, linear="lu", abs_tol=1e-10, reduction=1e4)
    r = info["res"]
    target = max(1e-10, r[0] / 1e4)
    assert r[-1] <= target and all(x > target for x in r[:-1])


@pytest.mark.slow
def test_gmg_newton_equals_direct_newton():
    wl = synth.small_workload(2, 2, (8, 2), 2, obstacle=True)
    lev = _fine(wl)
    X0 = _start(wl, lev)
    Xg, ig = newton.newton_solve(wl, X0, 0.3, linear="gmg", lin_rtol=1e-12, abs_tol=1e-12, reduction=1e30)
    Xd, idd = newton.newton_solve(wl, X0, 0.3, linear="lu", abs_tol=1e-12, reduction=1e30)
    assert len(ig["res"]) == len(idd["res"])
    assert np.abs(Xg - Xd).max() <= 1e-9 * np.abs(Xd).max()


# ---------------------------------------------------------------------------------------------
# previous-slab load and time marching (Problem 3.1)
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("dim,k", [(2, 1), (2, 2), (3, 1)])
def test_prev_slab_load_equals_analytic_poiseuille_term(dim, k):
    """The Poiseuille field is exactly Q2, so the discrete previous-slab term of its interpolant equals
    the analytic term <U g_1 e_x, psi(t_{n-1}^+)>."""
    cells = (4, 2) if dim == 2 else (4, 2, 2)
    wl = synth.small_workload(dim, k, cells, 1, obstacle=False)
    lev = _fine(wl)
    U = 0.3
    X = _poiseuille_state(lev, U, wl.nu)
    g_only = newton.inflow_load(lev, U, wl.nu, wl.tau)
    analytic = adjoint.newton_rhs(lev, None, U, wl.nu, wl.tau, with_convection=False) - g_only
    discrete = newton.prev_slab_load(lev, X)
    assert np.abs(discrete - analytic).max() <= 1e-13 * np.abs(analytic).max()


@pytest.mark.parametrize("k", [1, 2])
def test_poiseuille_is_a_discrete_steady_solution(k):
    """In a channel without obstacle, Poiseuille flow with its linear pressure and do-nothing outflow
    solves the Navier-Stokes slab problem exactly in Q2/P1disc x dG(k): F vanishes to rounding, which
    pins every term of A, c and b (time derivative and jump, viscous and Nitsche forms, pressure
    coupling, convection, inflow data, previous-slab term) at once."""
    wl = synth.small_workload(2, k, (8, 2), 1, obstacle=False)
    lev = _fine(wl)
    U = 0.3
    X = _poiseuille_state(lev, U, wl.nu)
    for prev in (None, X):
        prob = newton.SlabProblem(lev, U, wl.nu, wl.tau, X_prev=prev)
        F = prob.residual(X)
        assert np.linalg.norm(F) <= 1e-12 * np.linalg.norm(prob.b), np.linalg.norm(F)
    # a wrong pressure level is not a solution (the outflow condition fixes it)
    Xs = X.copy()
    for a in range(lev.k + 1):
        Xs[a * lev.block + lev.dim * lev.R::lev.np_][:lev.C] += 0.01
    assert np.linalg.norm(newton.SlabProblem(lev, U, wl.nu, wl.tau).residual(Xs)) > 1e-6


def test_time_march_from_poiseuille_stays():
    wl = synth.small_workload(2, 1, (8, 2), 2, obstacle=False)
    lev = _fine(wl)
    X = _poiseuille_state(lev, 0.3, wl.nu)
    states, _, infos = newton.time_march(wl, X, 0.3, 3, linear="lu", abs_tol=1e-12, reduction=1e30)
    for Xn, inf in zip(states, infos):
        assert inf["converged"]
        assert np.abs(Xn - X).max() <= 1e-10 * np.abs(X).max()
