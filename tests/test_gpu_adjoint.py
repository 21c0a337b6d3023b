"""Adjoint / gradient path on the GPU against the oracle (the 2D dG(1) channel c4_2d_k1 and small 2D/3D cases).

Right-hand sides, functional weights and (dJ/dnu) x must match the oracle to rounding (1e-12).
Autograd gradients (one forward and one adjoint FGMRES solve, rtol 1e-13) must match the oracle's
adjoint gradient from direct solves to 1e-7 and central finite differences (h = 1e-6) of GPU
solves to 1e-5.
"""
import numpy as np
import pytest

import synth
from helpers import gpu_hierarchy, lattice_to_gpu, rel_max

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SMALL = {
    "2d_k1": synth.small_workload(2, 1, (8, 3), 2, obstacle=True, seed=51),
    "2d_k2": synth.small_workload(2, 2, (6, 3), 2, obstacle=True, seed=52),
    "3d_k1": synth.small_workload(3, 1, (4, 2, 2), 2, obstacle=True, seed=56),
}


def wake_level1(wl):
    lo = (wl.obstacle_hi[0], wl.obstacle_lo[1]) + ((0,) if wl.dim == 3 else ())
    hi = (wl.obstacle_hi[0] + 2, wl.obstacle_hi[1]) + ((wl.coarse_cells[2],) if wl.dim == 3 else ())
    return lo, hi


def oracle_fine(wl):
    from oracle import adjoint, fem
    f = 2 ** (wl.n_levels - 1)
    lev = fem.Level(wl.dim, wl.k, wl.fine_cells, wl.length, tuple(x * f for x in wl.obstacle_lo),
                    tuple(x * f for x in wl.obstacle_hi))
    X_lin = lev.dofs_from_lattice(synth.linearisation_point(wl))
    lo, hi = wake_level1(wl)
    j = adjoint.functional_weights(lev, tuple(x * f for x in lo[:wl.dim]), tuple(x * f for x in hi[:wl.dim]), wl.tau)
    return lev, X_lin, j


@pytest.mark.parametrize("name", list(SMALL))
def test_rhs_functional_and_dnu_parity(name):
    from oracle import adjoint
    wl = SMALL[name]
    lev, X_lin, j = oracle_fine(wl)
    h = gpu_hierarchy(wl, factor=False)
    U, nu = 0.3, wl.nu
    b = torch.empty(lev.N, dtype=torch.float64, device="cuda")
    h.assemble_rhs(U, nu, b, which=0)
    assert rel_max(b.cpu().numpy(), adjoint.newton_rhs(lev, X_lin, U, nu, wl.tau)) < 1e-12
    h.assemble_rhs(U, nu, b, which=1)
    assert rel_max(b.cpu().numpy(), adjoint.db_dU(lev, X_lin, nu, wl.tau)) < 1e-12
    h.assemble_rhs(U, nu, b, which=2)
    assert rel_max(b.cpu().numpy(), adjoint.db_dnu(lev, X_lin, U, wl.tau)) < 1e-12
    lo, hi = wake_level1(wl)
    jg = torch.empty_like(b)
    h.functional_weights(lo, hi, jg)
    assert rel_max(jg.cpu().numpy(), j) < 1e-13
    x = np.random.default_rng(57).standard_normal(lev.N)
    y = torch.empty_like(b)
    h.jacobian_dnu_apply(torch.from_numpy(x).cuda(), y)
    assert rel_max(y.cpu().numpy(), adjoint.dJ_dnu_apply(lev, X_lin, wl.tau, x)) < 1e-12
    h.close()


def test_autograd_gradients_c4_2d_k1():
    from oracle import adjoint
    from paper_2107_10561_gb300.adjoint import GMGSolveFunctional, SlabFunctional
    wl = synth.WORKLOADS["c4_2d_k1"]
    lev, X_lin, j = oracle_fine(wl)
    h = gpu_hierarchy(wl, factor=False)
    Xg = lattice_to_gpu(h, synth.linearisation_point(wl))
    lo, hi = wake_level1(wl)
    sf = SlabFunctional(h, Xg, lo, hi, rtol=1e-13)
    U = torch.tensor(0.3, dtype=torch.float64, requires_grad=True)
    nu = torch.tensor(wl.nu, dtype=torch.float64, requires_grad=True)
    J = GMGSolveFunctional.apply(U, nu, sf)
    J.backward()
    assert sf.last_info["forward"]["converged"] and sf.last_info["adjoint"]["converged"]
    Jo, gUo, gnuo, _, _ = adjoint.adjoint_gradient(lev, X_lin, 0.3, wl.nu, wl.tau, j)
    assert abs(float(J.detach()) - Jo) <= 1e-9 * abs(Jo)
    assert abs(float(U.grad) - gUo) <= 1e-7 * abs(gUo), (float(U.grad), gUo)
    assert abs(float(nu.grad) - gnuo) <= 1e-7 * abs(gnuo), (float(nu.grad), gnuo)
    # central differences of GPU solves
    hh = 1e-6
    f = lambda Uv, nuv: sf.value_and_state(Uv, nuv)[0]
    fdU = (f(0.3 + hh, wl.nu) - f(0.3 - hh, wl.nu)) / (2 * hh)
    fdnu = (f(0.3, wl.nu + hh) - f(0.3, wl.nu - hh)) / (2 * hh)
    assert abs(float(U.grad) - fdU) <= 1e-5 * abs(fdU), (float(U.grad), fdU)
    assert abs(float(nu.grad) - fdnu) <= 1e-5 * abs(fdnu), (float(nu.grad), fdnu)
    h.close()


@pytest.mark.parametrize("name", list(SMALL))
def test_assemble_load_at_an_explicit_point(name):
    """stm_assemble_load(U, nu, w): b(U, nu) + c(w, w) for a point w other than the assembled one equals
    the oracle's Newton-step load at w, and leaves the assembled Jacobian untouched."""
    from oracle import adjoint
    wl = SMALL[name]
    lev, X_lin, _ = oracle_fine(wl)
    h = gpu_hierarchy(wl, factor=False)
    w2 = X_lin + 0.05 * np.random.default_rng(58).standard_normal(lev.N)
    x = torch.from_numpy(np.random.default_rng(59).standard_normal(lev.N)).cuda()
    y0, y1 = torch.empty_like(x), torch.empty_like(x)
    h.spmv(h.finest, x, y0)
    b = torch.empty_like(x)
    h.assemble_load(0.3, wl.nu, b, w=torch.from_numpy(w2).cuda())
    assert rel_max(b.cpu().numpy(), adjoint.newton_rhs(lev, w2, 0.3, wl.nu, wl.tau)) < 1e-12
    h.spmv(h.finest, x, y1)
    assert torch.equal(y0, y1)
    h.assemble_load(0.3, wl.nu, b)  # w = the assembled point
    assert rel_max(b.cpu().numpy(), adjoint.newton_rhs(lev, X_lin, 0.3, wl.nu, wl.tau)) < 1e-12
    h.close()


@pytest.mark.parametrize("name", list(SMALL))
def test_adjoint_gradient_entry_point(name):
    """stm_adjoint_gradient (adjoint FGMRES solve and the two gradient combinations inside the library)
    against the oracle's adjoint gradient from direct solves; lambda against the oracle's J^T solve."""
    from oracle import adjoint
    wl = SMALL[name]
    lev, X_lin, j = oracle_fine(wl)
    h = gpu_hierarchy(wl)
    U = 0.3
    b = torch.empty(lev.N, dtype=torch.float64, device="cuda")
    h.assemble_load(U, wl.nu, b)
    X = torch.zeros_like(b)
    h.gmres_solve(b, X, rtol=1e-13)
    lam = torch.empty_like(b)
    gU, gnu, info = h.adjoint_gradient(U, wl.nu, torch.from_numpy(j).cuda(), X, lam=lam, rtol=1e-13)
    assert info["converged"] and info["history"] and info["history"][0] == pytest.approx(1.0)
    Jo, gUo, gnuo, _, lam_o = adjoint.adjoint_gradient(lev, X_lin, U, wl.nu, wl.tau, j)
    assert abs(gU - gUo) <= 1e-7 * abs(gUo), (gU, gUo)
    assert abs(gnu - gnuo) <= 1e-7 * abs(gnuo), (gnu, gnuo)
    assert rel_max(lam.cpu().numpy(), lam_o) < 1e-8
    h.close()
