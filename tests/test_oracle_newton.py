"""Pins of the oracle's nonlinear slab residual and damped Newton (Sec. 3, Eqs. nonlineq, linNewEq,
linNewEqU; stopping rule of Sec. 5.1)."""
import numpy as np
import pytest
from scipy import optimize

import synth
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
