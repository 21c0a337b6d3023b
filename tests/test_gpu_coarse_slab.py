"""Direct coarse solve of Algorithm 1 on coarse levels large enough for the twisted slab factors: d =
J_1^{-1} r and d = J_1^{-T} r against a sparse direct solve of the oracle's J_1 (1e-10 relative), for one
vector and for 32 columns inside the multi-right-hand-side V-cycle (through the coarse solve of a
two-level V(0,0) cycle: P J_1^{-1} P^T r). Coarse grids (all minus the obstacle):
  - 16x4x4 (the 3D channel's level 1, 18,000 DoFs): 16 slabs, twist at slab 8, chains of 7 and 6 steps;
  - 9x4x4: an odd slab count, twist at slab 4, chains of equal length;
  - 2x8x8: two slabs, no chain step, one back-substitution step.
Small coarse levels keep the explicit inverse and are covered by test_gpu_parity.test_coarse_solve."""
import dataclasses

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from helpers import gpu_hierarchy, rel_max

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=[(16, 4, 4), (9, 4, 4), (2, 8, 8)], ids=["16x4x4", "9x4x4", "2x8x8"])
def pair(request):
    from oracle import fem
    wl = dataclasses.replace(synth.WORKLOADS["c3_3d_k1"], n_levels=2, coarse_cells=request.param)
    lev0 = fem.Level(wl.dim, wl.k, wl.coarse_cells, wl.length, wl.obstacle_lo, wl.obstacle_hi)
    st = fem.fine_lattice_to_level(synth.linearisation_point(wl), wl.fine_cells, lev0)
    J0 = fem.assemble_jacobian(lev0, lev0.dofs_from_lattice(st), wl.tau, wl.nu, wl.gamma1, wl.gamma2)
    h = gpu_hierarchy(wl)
    yield wl, lev0, J0, h
    h.close()


@pytest.mark.parametrize("transpose", [False, True])
def test_slab_coarse_solve(pair, transpose):
    wl, lev0, J0, h = pair
    assert lev0.N >= 8000
    rng = np.random.default_rng(81)
    lu = spla.splu((J0.T if transpose else J0).tocsc())
    for _ in range(2):  # twice: the work vectors and the cooperative launch are reused
        r = rng.standard_normal(lev0.N)
        d = torch.zeros(lev0.N, dtype=torch.float64, device="cuda")
        h.coarse_solve(torch.from_numpy(r).cuda(), d, transpose=transpose)
        assert rel_max(d.cpu().numpy(), lu.solve(r)) < 1e-10


def test_slab_coarse_solve_32_columns(pair):
    """The 32-column coarse solve inside the multi-RHS V-cycle: with V(0,0) on two levels the
    preconditioner is M^{-1} b = P J_1^{-1} P^T b, and one FGMRES iteration from x = 0 returns a scalar
    multiple of it for every column; directions compared column by column (1e-9)."""
    from oracle import fem
    wl, lev0, J0, h = pair
    wl0 = dataclasses.replace(wl, nu1=0, nu2=0)
    h2 = gpu_hierarchy(wl0, "bf16")
    lev1 = fem.Level(wl.dim, wl.k, wl.fine_cells, wl.length, tuple(2 * x for x in wl.obstacle_lo),
                     tuple(2 * x for x in wl.obstacle_hi))
    P = fem.prolongation(lev0, lev1)
    lu = spla.splu(J0.tocsc())
    B = np.random.default_rng(82).standard_normal((32, lev1.N))
    X = torch.zeros(32, lev1.N, dtype=torch.float64, device="cuda")
    h2.gmres_solve_multi(torch.from_numpy(B).cuda(), X, rtol=1e-10, max_iter=1, raise_on_fail=False)
    Xh = X.cpu().numpy()
    for c in range(32):
        e = P @ lu.solve(P.T @ B[c])
        x = Xh[c] * np.sign(Xh[c] @ e)
        assert rel_max(x / np.linalg.norm(x), e / np.linalg.norm(e)) < 1e-9, c
    h2.close()
