"""The viscosity / damping study of Sec. 5.3 (Table 5.4) on a reduced channel: for each (nu, omega_d)
the GPU Newton solve takes the same Newton steps as the oracle's, and every inner GMG-FGMRES solve
the same number of iterations within +-1 (V(4,4) cycles, tau = 0.005, inner rtol 1e-8)."""
import dataclasses

import pytest

import synth
from helpers import gpu_hierarchy, lattice_to_gpu

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

BASE = synth.small_workload(2, 1, (8, 2), 3, obstacle=True)


@pytest.mark.timeout(600)
@pytest.mark.parametrize("nu", [1e-3, 3e-4, 1e-4])
@pytest.mark.parametrize("omega", [1.0, 0.7])
def test_newton_and_gmres_counts_match_oracle(nu, omega):
    from oracle import newton
    from oracle.fem import Level
    wl = dataclasses.replace(BASE, nu=nu, omega=omega, nu1=4, nu2=4, tau=0.005)
    f = 2 ** (wl.n_levels - 1)
    lev = Level(wl.dim, wl.k, wl.fine_cells, wl.length, tuple(x * f for x in wl.obstacle_lo),
                tuple(x * f for x in wl.obstacle_hi))
    st = synth.linearisation_point(wl)
    _, io = newton.newton_solve(wl, lev.dofs_from_lattice(st), 0.3, linear="gmg", lin_rtol=1e-8)
    h = gpu_hierarchy(wl, "f64", factor=False)
    X = lattice_to_gpu(h, st)
    ig = h.newton_solve(X, 0.3, rtol=1e-8, raise_on_fail=False)
    h.close()
    assert ig["converged"] == io["converged"]
    assert ig["newton_iters"] == len(io["gmres_iters"]), (ig, io)
    for a, b in zip(ig["gmres_step"], io["gmres_iters"]):
        assert abs(a - b) <= 1, (ig["gmres_step"], io["gmres_iters"])
