"""Multi-right-hand-side path (32 columns sharing one hierarchy) against the single-RHS path and
the oracle.

One multi-RHS smoothing step equals, column by column, the oracle's additive sweep taken with the
oracle's cell inverses rounded to the storage precision (one rounding from FP64), and the
single-RHS GPU step: to 1e-12 with FP64
inverses (same arithmetic, other summation order), 1e-5 with FP32 inverses (FP32 accumulation),
and 1e-4 with BF16 inverses on the tensor cores (the gathered block enters as two BF16 parts, i.e.
to about 2^-16 relative; FP32 accumulation). The lock-stepped FGMRES reaches the same solutions as
one solve per column and as the direct solve.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from helpers import gpu_hierarchy, lattice_to_gpu, rel_max

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    "3d_k1": synth.small_workload(3, 1, (3, 2, 2), 2, obstacle=True, seed=61),
    "2d_k2": synth.small_workload(2, 2, (6, 3), 2, obstacle=True, seed=62),
    "2d_k1": synth.small_workload(2, 1, (6, 3), 2, obstacle=True, seed=63),
}
TOL = {"f64": 1e-12, "f32": 1e-5, "bf16": 1e-4}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("nrhs", [32, 5])
def test_multi_sweep_equals_single_sweeps(name, prec, nrhs):
    wl = CASES[name]
    h = gpu_hierarchy(wl, prec)
    g = h.finest
    n = h.n_dofs(g)
    rng = np.random.default_rng(64)
    R = torch.from_numpy(rng.standard_normal((nrhs, n))).cuda()
    D = torch.from_numpy(rng.standard_normal((nrhs, n))).cuda()
    Dm = D.clone()
    h.vanka_sweep_multi(g, R, Dm)
    for c in range(nrhs):
        d = D[c].clone()
        h.vanka_sweep(g, R[c].contiguous(), d)
        assert rel_max(Dm[c].cpu().numpy(), d.cpu().numpy()) < TOL[prec], (c, prec)
    h.close()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("nrhs", [32, 7])
def test_multi_sweep_against_oracle(name, prec, nrhs):
    """Every column of one multi-RHS additive step against oracle.solvers.vanka_step (Eq. LocVanka,
    damped, multiplicity-weighted) on the oracle's J, with the oracle's inverses rounded to the
    storage precision as the GPU stores them."""
    from helpers import oracle_hierarchy, round_storage
    from oracle import solvers
    wl = CASES[name]
    o = oracle_hierarchy(wl)
    h = gpu_hierarchy(wl, prec)
    g = h.finest
    lev = o.fine
    inv = round_storage(o.inv[-1], prec)
    rng = np.random.default_rng(65)
    R = rng.standard_normal((nrhs, lev.N))
    D = rng.standard_normal((nrhs, lev.N))
    Dm = torch.from_numpy(D).cuda()
    h.vanka_sweep_multi(g, torch.from_numpy(R).cuda(), Dm)
    got = Dm.cpu().numpy()
    for c in range(nrhs):
        expect = solvers.vanka_step(lev, o.J[-1], inv, D[c], R[c], wl.omega)
        assert rel_max(got[c], expect) < TOL[prec], (c, prec)
    h.close()


def _inflow_sweep_rhs(h, wl, nrhs):
    """Columns b(U_j, nu) + c(w, w), U_j = linspace(0.2, 0.45, nrhs) (the multi-RHS workload)."""
    n = h.n_dofs()
    B = torch.empty((nrhs, n), dtype=torch.float64, device="cuda")
    for c, U in enumerate(synth.inflow_sweep(nrhs)):
        b = torch.empty(n, dtype=torch.float64, device="cuda")
        h.assemble_rhs(U, wl.nu, b, which=0)
        B[c] = b
    return B


@pytest.mark.parametrize("prec", ["bf16", "f64"])
def test_multi_gmres_matches_single_solves(prec):
    wl = CASES["3d_k1"]
    h = gpu_hierarchy(wl, prec)
    nrhs = 32
    B = _inflow_sweep_rhs(h, wl, nrhs)
    X = torch.zeros_like(B)
    infos = h.gmres_solve_multi(B, X, rtol=1e-10)
    assert all(i["converged"] and i["rel_res_true"] <= 2e-10 for i in infos), infos[:3]
    for c in (0, 7, 31):
        x = torch.zeros_like(B[c])
        info = h.gmres_solve(B[c].contiguous(), x, rtol=1e-10)
        assert rel_max(X[c].cpu().numpy(), x.cpu().numpy()) < 1e-7
        assert abs(infos[c]["iters"] - info["iters"]) <= 2, (infos[c], info)
    # against the direct solve of the oracle's matrix
    from helpers import oracle_hierarchy
    o = oracle_hierarchy(wl)
    for c in (0, 31):
        xd = spla.spsolve(o.J[-1].tocsc(), B[c].cpu().numpy())
        assert rel_max(X[c].cpu().numpy(), xd) < 1e-6
    h.close()


@pytest.mark.parametrize("name", ["3d_k1", "2d_k2", "2d_k1"])
@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("nf,na", [(16, 16), (5, 11), (16, 0), (0, 3)])
def test_fused_forward_adjoint_sweep_against_oracle(name, prec, nf, na):
    """stm_vanka_sweep_fused: forward columns against oracle.solvers.vanka_step on J, adjoint columns
    against the transposed oracle step (J^T, J_T^{-T}), one pass over the inverses on the GPU."""
    from helpers import oracle_hierarchy, round_storage
    from oracle import solvers
    wl = CASES[name]
    o = oracle_hierarchy(wl)
    h = gpu_hierarchy(wl, prec)
    g = h.finest
    lev = o.fine
    inv = round_storage(o.inv[-1], prec)
    rng = np.random.default_rng(66)
    Rf, Df = rng.standard_normal((nf, lev.N)), rng.standard_normal((nf, lev.N))
    Ra, Da = rng.standard_normal((na, lev.N)), rng.standard_normal((na, lev.N))
    dRf, dDf = torch.from_numpy(Rf).cuda(), torch.from_numpy(Df).cuda()
    dRa, dDa = torch.from_numpy(Ra).cuda(), torch.from_numpy(Da).cuda()
    h.vanka_sweep_fused(g, dRf if nf else None, dDf if nf else None, dRa if na else None, dDa if na else None)
    gf, ga = dDf.cpu().numpy(), dDa.cpu().numpy()
    for c in range(nf):
        expect = solvers.vanka_step(lev, o.J[-1], inv, Df[c], Rf[c], wl.omega)
        assert rel_max(gf[c], expect) < TOL[prec], ("forward", c)
    for c in range(na):
        expect = solvers.vanka_step(lev, o.J[-1], inv, Da[c], Ra[c], wl.omega, transpose=True)
        assert rel_max(ga[c], expect) < TOL[prec], ("adjoint", c)
    h.close()
