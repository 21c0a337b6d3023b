"""Pins of the oracle's adjoint gradients against central finite differences (CPU only)."""
import numpy as np
import pytest

import synth
from oracle import adjoint, fem


def _setup(wl):
    f = 2 ** (wl.n_levels - 1)
    lev = fem.Level(wl.dim, wl.k, wl.fine_cells, wl.length, tuple(x * f for x in wl.obstacle_lo),
                    tuple(x * f for x in wl.obstacle_hi))
    X_lin = lev.dofs_from_lattice(synth.linearisation_point(wl))
    wake_lo = (wl.obstacle_hi[0] * f, wl.obstacle_lo[1] * f) + ((0,) if wl.dim == 3 else ())
    wake_hi = ((wl.obstacle_hi[0] + 2) * f, wl.obstacle_hi[1] * f) + ((wl.fine_cells[2],) if wl.dim == 3 else ())
    j = adjoint.functional_weights(lev, wake_lo, wake_hi, wl.tau)
    return lev, X_lin, j


@pytest.mark.parametrize("wl", [synth.small_workload(2, 1, (8, 3), 2, obstacle=True, seed=51),
                                synth.small_workload(2, 2, (6, 3), 2, obstacle=True, seed=52)])
def test_adjoint_gradient_matches_central_differences(wl):
    lev, X_lin, j = _setup(wl)
    U, nu = 0.3, wl.nu
    J0, gU, gnu, _, _ = adjoint.adjoint_gradient(lev, X_lin, U, nu, wl.tau, j)
    h = 1e-6
    fU = (adjoint.functional_direct(lev, X_lin, U + h, nu, wl.tau, j)[0]
          - adjoint.functional_direct(lev, X_lin, U - h, nu, wl.tau, j)[0]) / (2 * h)
    fnu = (adjoint.functional_direct(lev, X_lin, U, nu + h, wl.tau, j)[0]
           - adjoint.functional_direct(lev, X_lin, U, nu - h, wl.tau, j)[0]) / (2 * h)
    assert abs(gU - fU) <= 1e-5 * abs(fU), (gU, fU)
    assert abs(gnu - fnu) <= 1e-5 * abs(fnu), (gnu, fnu)


def test_convection_term_euler_identity():
    """c(w, w) is quadratic in w, so its Newton derivative satisfies (J(w) - J(0)) w = 2 c(w, w)."""
    wl = synth.small_workload(2, 2, (6, 3), 2, obstacle=True, seed=53)
    lev, X_lin, _ = _setup(wl)
    Jw = fem.assemble_jacobian(lev, X_lin, wl.tau, wl.nu)
    J0 = fem.assemble_jacobian(lev, np.zeros(lev.N), wl.tau, wl.nu)
    c = fem.convection_residual(lev, X_lin, wl.tau)
    np.testing.assert_allclose((Jw - J0) @ X_lin, 2 * c, atol=1e-12 * np.abs(c).max())


def test_rhs_linear_in_U_and_affine_in_nu():
    wl = synth.small_workload(2, 1, (6, 3), 2, obstacle=True, seed=54)
    lev, X_lin, _ = _setup(wl)
    b = lambda U, nu: adjoint.newton_rhs(lev, X_lin, U, nu, wl.tau, with_convection=False)
    np.testing.assert_allclose(b(0.6, 1e-3), 2 * b(0.3, 1e-3), atol=1e-14)
    np.testing.assert_allclose(b(0.3, 2e-3) - 2 * b(0.3, 1e-3) + b(0.3, 0.0), 0.0, atol=1e-14)
    np.testing.assert_allclose(adjoint.db_dU(lev, X_lin, 1e-3, wl.tau), b(1.0, 1e-3), atol=1e-14)


def test_functional_weights_integrate_constants():
    """j . X for X = 1 in every velocity-1 entry equals |wake| * tau (sum of basis functions is 1)."""
    wl = synth.small_workload(2, 1, (8, 3), 2, obstacle=True, seed=55)
    lev, _, j = _setup(wl)
    X = np.zeros(lev.N)
    for a in range(lev.k + 1):
        X[a * lev.block: a * lev.block + lev.R] = 1.0
    f = 2 ** (wl.n_levels - 1)
    area = (2 * f * lev.h[0]) * ((wl.obstacle_hi[1] - wl.obstacle_lo[1]) * f * lev.h[1])
    np.testing.assert_allclose(j @ X, area * wl.tau, rtol=1e-13)
