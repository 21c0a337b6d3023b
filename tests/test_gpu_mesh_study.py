"""V(1,1) and V(4,4) cycles on refined meshes (the mesh-independence setting of Tables 5.1 and 5.5,
Sec. 5.1 and 5.4): the GPU FGMRES takes the oracle's number of iterations within +-1 and reaches
the direct solution, for one and two refinements of the same coarse grid, in 2D and 3D."""
import dataclasses

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from helpers import gpu_hierarchy, lattice_to_gpu, oracle_hierarchy, rel_max

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BASES = {
    "2d_k1_L2": synth.small_workload(2, 1, (6, 3), 2, obstacle=True, seed=81),
    "2d_k1_L3": synth.small_workload(2, 1, (6, 3), 3, obstacle=True, seed=81),
    "3d_k1_L2": synth.small_workload(3, 1, (3, 2, 2), 2, obstacle=True, seed=82),
}


@pytest.mark.parametrize("name", list(BASES))
@pytest.mark.parametrize("sweeps", [1, 4])
def test_cycle_depth_iterations_match_oracle(name, sweeps):
    wl = dataclasses.replace(BASES[name], nu1=sweeps, nu2=sweeps)
    o = oracle_hierarchy(wl)
    b = o.fine.dofs_from_lattice(synth.random_rhs(wl))
    _, info_o = o.solve(b, rtol=1e-8)
    h = gpu_hierarchy(wl)
    x = torch.zeros(b.size, dtype=torch.float64, device="cuda")
    info = h.gmres_solve(torch.from_numpy(b).cuda(), x, rtol=1e-8, restart=wl.restart)
    assert info["converged"] and abs(info["iters"] - info_o["iters"]) <= 1, (info, info_o)
    assert rel_max(x.cpu().numpy(), spla.spsolve(o.J[-1].tocsc(), b)) < 1e-7
    h.close()


def test_more_sweeps_fewer_iterations():
    """V(4,4) needs no more FGMRES iterations than V(1,1) on the same system (Tables 5.1, 5.5)."""
    its = {}
    for sweeps in (1, 4):
        wl = dataclasses.replace(BASES["2d_k1_L3"], nu1=sweeps, nu2=sweeps)
        h = gpu_hierarchy(wl)
        b = lattice_to_gpu(h, synth.random_rhs(wl))
        x = torch.zeros_like(b)
        its[sweeps] = h.gmres_solve(b, x, rtol=1e-8)["iters"]
        h.close()
    assert its[4] <= its[1], its
