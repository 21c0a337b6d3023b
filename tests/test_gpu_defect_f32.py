"""FP32 defects inside the V-cycle (defect_precision = "f32"): the smoother's r - J_g d runs over
FP32 copies of J_g's values with FP32 products and sums, while FGMRES, its Arnoldi products and the
true residual stay FP64 (Sec. 3: flexible GMRES keeps every preconditioned vector).

A single sweep is checked against the oracle's sweep (Sec. 4.2, Eq. LocVanka) whose defect is the
exact value t = r - fl32(J) fl32(d), element by element, within the error bound of an FP32 dot
product of m terms in any summation order (fused multiply-adds only tighten it):
    |delta t_i| <= gamma_m sum_j |fl32(J)_ij| |fl32(d)_j|,   gamma_m = m u / (1 - m u),  u = 2^-24,
carried through the smoother's update as |delta d_new| <= omega W sum_T |J_T^{-1}| |delta t_T|
(additive), or through the owning cell's |J_T^{-1}| (overwrite). Solves must still reach the FP64
tolerance and the direct solution.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from helpers import gpu_params, lattice_to_gpu, oracle_hierarchy, rel_max

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    "2d_k1_obs": synth.small_workload(2, 1, (6, 3), 2, obstacle=True, seed=21),
    "2d_k2_obs_3lev": synth.small_workload(2, 2, (4, 2), 3, obstacle=True, seed=22),
    "3d_k1_obs": synth.small_workload(3, 1, (3, 2, 2), 2, obstacle=True, seed=23),
    "c1": synth.WORKLOADS["c1_2d_k1"],
}
U = 2.0 ** -24
_oracles = {}


def _oracle(name, smoother="additive"):
    key = (name, smoother)
    if key not in _oracles:
        _oracles[key] = oracle_hierarchy(CASES[name], variant=smoother)
    return _oracles[key]


def _hier(name, prec="f64", smoother="additive", defect="f32", reassemble=False):
    """GPU hierarchy at the seeded linearisation point; with reassemble=True it is first assembled
    and factored at the zero state, so the FP32 copies must follow the second assembly."""
    from paper_2107_10561_gb300 import Hierarchy
    wl = CASES[name]
    h = Hierarchy(gpu_params(wl, prec, smoother, defect_precision=defect))
    X = lattice_to_gpu(h, synth.linearisation_point(wl))
    if reassemble:
        h.assemble_jacobian(torch.zeros_like(X))
        h.factor_cells()
    h.assemble_jacobian(X)
    h.factor_cells()
    torch.cuda.synchronize()
    return h


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("name", ["2d_k1_obs", "2d_k2_obs_3lev", "3d_k1_obs"])
@pytest.mark.parametrize("transpose", [False, True])
def test_defect_within_fp32_dot_bound(name, transpose):
    """stm_defect on every level: |t - (r - fl32(A) fl32(d))| <= gamma_m sum_j |fl32(A)_ij| |fl32(d)_j|
    element by element; with defect_precision = "f64" it is r - A d to rounding."""
    wl = CASES[name]
    o = _oracle(name)
    h = _hier(name, "bf16")
    h64 = _hier(name, "bf16", defect="f64")
    rng = np.random.default_rng(72)
    for g in range(wl.n_levels):
        A = (o.J[g].T if transpose else o.J[g]).tocsr()
        A32 = A.astype(np.float32).astype(np.float64)
        r = rng.standard_normal(A.shape[0])
        d = rng.standard_normal(A.shape[0])
        d32 = d.astype(np.float32).astype(np.float64)
        m = np.diff(A32.indptr).astype(np.float64)
        bound = m * U / (1.0 - m * U) * (abs(A32) @ np.abs(d32)) + 1e-15 * np.abs(r)
        t = torch.empty(A.shape[0], dtype=torch.float64, device="cuda")
        h.defect(g, dev(r), dev(d), t, transpose=transpose)
        err = np.abs(t.cpu().numpy() - (r - A32 @ d32))
        assert np.all(err <= bound), (g, float((err - bound).max()))
        h64.defect(g, dev(r), dev(d), t, transpose=transpose)
        assert rel_max(t.cpu().numpy(), r - A @ d) < 1e-13
    h.close()
    h64.close()


# FP64 values whose rounding to FP32 exercises each branch of round-to-nearest-even: exact, below
# and above half an ulp, ties to an even and to an odd fraction, a carry into the exponent, both
# ends of the normal FP32 range, subnormal results (a carry into the normal range, the tie at half
# the smallest subnormal), results that round to zero (an FP64 subnormal included), negative values
_ROUNDING_CASES = [1.0, 1.0 + 2.0**-25, 1.0 + 2.0**-24 - 2.0**-40, 1.0 + 2.0**-24, 1.0 + 3 * 2.0**-24,
                   1.0 + 2.0**-24 + 2.0**-40, 2.0 - 2.0**-25, -(1.0 + 3 * 2.0**-24), 0.1, -1.0 / 3.0,
                   2.0**-126, 2.0**-126 * (1 - 2.0**-30), 1.5 * 2.0**-127, 2.0**-149 * 0.75,
                   2.0**-150, 2.0**-150 * (1 + 2.0**-40), 2.0**-151, 5e-324, 1.5 * 2.0**127,
                   (2.0 - 2.0**-23) * 2.0**127, 3.0e-30, 7.0e29]


@pytest.mark.parametrize("transpose", [False, True])
def test_defect_rounds_d_to_nearest_even(transpose):
    """One nonzero d_j = v per call, r = 0: every row then holds a single FP32 product, so
    t_i = -fl32(fl32(A_ij) * rn32(v)) exactly, with rn32 the IEEE round-to-nearest-even conversion
    (numpy's float32 cast) and fl32 the IEEE FP32 product. Covers a velocity and a pressure column.
    Exact on the entries above 1e-6 of the column's largest; the others are assembly rounding noise
    (the GPU's J matches the oracle's to 1e-13 of its largest entry), held to that level instead."""
    name = "2d_k1_obs"
    wl = CASES[name]
    o = _oracle(name)
    g = wl.n_levels - 1
    lev = o.levels[g]
    A = (o.J[g].T if transpose else o.J[g]).tocsc()
    h = _hier(name, "bf16")
    n = lev.N
    cols = [lev.R // 2 + 1, lev.dim * lev.R + lev.np_ * (lev.C // 2)]  # a velocity and a pressure DoF
    r = torch.zeros(n, dtype=torch.float64, device="cuda")
    t = torch.empty_like(r)
    with np.errstate(over="ignore", under="ignore"):
        for j in cols:
            colj = A.getcol(j).toarray().ravel().astype(np.float32)
            assert np.count_nonzero(colj) > 4
            for v in _ROUNDING_CASES:
                d = np.zeros(n)
                d[j] = v
                h.defect(g, r, dev(d), t, transpose=transpose)
                expect = -(colj * np.float32(v)).astype(np.float64)
                got = t.cpu().numpy()
                big = np.abs(colj) >= 1e-6 * np.abs(colj).max()
                assert np.array_equal(got[big], expect[big]), (j, v, np.abs(got - expect)[big].max())
                floor = 1e-12 * float(np.abs(colj).max()) * abs(v)
                assert np.all(np.abs(got[~big] - expect[~big]) <= floor), (j, v)
    h.close()


def test_defect_arguments_checked():
    from paper_2107_10561_gb300 import _lib
    h = _hier("2d_k1_obs", "bf16")
    n = h.n_dofs(h.finest)
    r = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.StmError) as e:
        h.defect(h.finest, r, r.clone(), r)  # t aliases r
    assert e.value.status == _lib.STM_ERR_INVALID_ARG
    h.close()


@pytest.mark.parametrize("name,reassemble", [("2d_k1_obs", False), ("2d_k2_obs_3lev", False),
                                             ("3d_k1_obs", False), ("2d_k1_obs", True)])
@pytest.mark.parametrize("smoother", ["additive", "overwrite"])
@pytest.mark.parametrize("transpose", [False, True])
def test_single_sweep_within_fp32_dot_bound(name, reassemble, smoother, transpose):
    from oracle import solvers
    wl = CASES[name]
    o = _oracle(name, smoother)
    g = wl.n_levels - 1
    lev, J, inv = o.levels[g], o.J[g].tocsr(), o.inv[g]
    A = J.T.tocsr() if transpose else J
    A32 = A.astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(71)
    r = rng.standard_normal(lev.N)
    d = rng.standard_normal(lev.N)
    d32 = d.astype(np.float32).astype(np.float64)
    t = r - A32 @ d32
    # the oracle's sweep computes r' - A d; r' = t + A d hands it the defect t
    expect = solvers.vanka_step(lev, J, inv, d, t + A @ d, wl.omega, smoother, transpose)
    m = np.diff(A32.indptr).astype(np.float64)
    gam = m * U / (1.0 - m * U)
    tb = gam * (abs(A32) @ np.abs(d32))
    zero = np.zeros(lev.N)
    bound = solvers.vanka_step(lev, J, np.abs(inv), zero, tb, wl.omega, smoother, transpose)
    # FP64 rounding of the rest of the step (inverse apply, combine, the r' round trip)
    mag = solvers.vanka_step(lev, J, np.abs(inv), zero, np.abs(t) + abs(A) @ np.abs(d), wl.omega, smoother,
                             transpose)
    slack = 1e-13 * (mag + np.abs(d))
    h = _hier(name, "f64", smoother, reassemble=reassemble)
    dg = dev(d)
    h.vanka_sweep(g, dev(r), dg, transpose=transpose)
    err = np.abs(dg.cpu().numpy() - expect)
    assert np.all(err <= bound + slack), float((err - bound - slack).max())
    # the FP32 path ran: an FP64-defect sweep gives a different result
    h64 = _hier(name, "f64", smoother, defect="f64")
    d64 = dev(d)
    h64.vanka_sweep(g, dev(r), d64, transpose=transpose)
    assert not torch.equal(dg, d64)
    h.close()
    h64.close()


@pytest.mark.parametrize("name", ["c1", "3d_k1_obs", "2d_k2_obs_3lev"])
@pytest.mark.parametrize("transpose", [False, True])
def test_solve_reaches_fp64_solution(name, transpose):
    """BF16 inverses with FP32 defects: FGMRES reaches 1e-8 and the direct solution; the FP32
    defects cost at most one extra iteration against FP64 defects."""
    wl = CASES[name]
    o = _oracle(name)
    b = o.fine.dofs_from_lattice(synth.random_rhs(wl))
    A = o.J[-1].T if transpose else o.J[-1]
    xd = spla.spsolve(A.tocsc(), b)
    its = {}
    for defect in ("f32", "f64"):
        h = _hier(name, "bf16", defect=defect)
        x = torch.zeros_like(dev(b))
        info = h.gmres_solve(dev(b), x, rtol=1e-8, transpose=transpose)
        assert info["converged"] and info["rel_res_true"] <= 2e-8, (defect, info)
        assert rel_max(x.cpu().numpy(), xd) < 1e-6
        its[defect] = info["iters"]
        h.close()
    assert its["f32"] <= its["f64"] + 1, its


def test_coloured_solve_converges():
    """The coloured smoother takes one defect per colour; with FP32 defects the solve still reaches
    1e-8 and the direct solution."""
    name = "2d_k2_obs_3lev"
    wl = CASES[name]
    o = _oracle(name)
    b = o.fine.dofs_from_lattice(synth.random_rhs(wl))
    h = _hier(name, "bf16", "coloured")
    x = torch.zeros_like(dev(b))
    info = h.gmres_solve(dev(b), x, rtol=1e-8)
    assert info["converged"] and info["rel_res_true"] <= 2e-8, info
    assert rel_max(x.cpu().numpy(), spla.spsolve(o.J[-1].tocsc(), b)) < 1e-6
    h.close()


def test_newton_with_fp32_defects_matches_oracle():
    """Damped Newton (Sec. 3) with BF16 inverses and FP32 defects: the nonlinear residual is FP64,
    so the steps, step lengths and final iterate follow the oracle's Newton with exact solves."""
    from oracle import newton
    from oracle.fem import Level
    wl = synth.small_workload(2, 2, (8, 2), 2, obstacle=True)
    f = 2 ** (wl.n_levels - 1)
    lev = Level(wl.dim, wl.k, wl.fine_cells, wl.length, tuple(x * f for x in wl.obstacle_lo),
                tuple(x * f for x in wl.obstacle_hi))
    st = synth.linearisation_point(wl, amp=2.0)
    Xo, io = newton.newton_solve(wl, lev.dofs_from_lattice(st), 0.3, linear="lu", abs_tol=1e-10, reduction=1e30)
    from paper_2107_10561_gb300 import Hierarchy
    h = Hierarchy(gpu_params(wl, "bf16", defect_precision="f32"))
    X = lattice_to_gpu(h, st)
    ig = h.newton_solve(X, 0.3, rtol=1e-12, abs_tol=1e-10, reduction=1e30)
    assert io["converged"] and ig["converged"]
    assert ig["newton_iters"] == len(io["lam"]) and ig["lam"] == io["lam"]
    assert rel_max(X.cpu().numpy(), Xo) < 1e-8
    h.close()


def test_bf16_defects_rejected():
    from paper_2107_10561_gb300 import Hierarchy, _lib
    with pytest.raises(_lib.StmError) as e:
        Hierarchy(gpu_params(CASES["2d_k1_obs"], "bf16", defect_precision="bf16"))
    assert e.value.status == _lib.STM_ERR_INVALID_ARG


def _composed_vcycle(h, wl, r, transpose):
    """Algorithm 1 spelled out through the public entry points: sweeps, defect, restriction, coarse
    solve, prolongation. Inside stm_vcycle the FP32 defects read d as rounded by the kernel that last
    wrote it; here every defect rounds d itself, so equal results show those copies are current."""
    G = wl.n_levels
    zeros = lambda g: torch.zeros(h.n_dofs(g), dtype=torch.float64, device="cuda")
    rs, ds = {G - 1: r}, {}
    for g in range(G - 1, 0, -1):
        d = zeros(g)
        for _ in range(wl.nu1):
            h.vanka_sweep(g, rs[g], d, transpose=transpose)
        t = zeros(g)
        h.defect(g, rs[g], d, t, transpose=transpose)
        rs[g - 1] = zeros(g - 1)
        h.restrict(g, t, rs[g - 1])
        ds[g] = d
    ds[0] = zeros(0)
    h.coarse_solve(rs[0], ds[0], transpose=transpose)
    for g in range(1, G):
        h.prolongate_add(g, ds[g - 1], ds[g])
        for _ in range(wl.nu2):
            h.vanka_sweep(g, rs[g], ds[g], transpose=transpose)
    return ds[G - 1]


@pytest.mark.parametrize("defect", ["f32", "f64"])
@pytest.mark.parametrize("smoother", ["additive", "overwrite", "coloured"])
@pytest.mark.parametrize("transpose", [False, True])
def test_vcycle_equals_its_public_steps(defect, smoother, transpose):
    name = "2d_k2_obs_3lev"
    wl = CASES[name]
    h = _hier(name, "bf16", smoother, defect=defect)
    r = dev(np.random.default_rng(73).standard_normal(h.n_dofs(h.finest)))
    d = torch.zeros_like(r)
    h.vcycle(r, d, transpose=transpose)
    assert torch.equal(d, _composed_vcycle(h, wl, r, transpose))
    h.close()
