"""GPU path (libstm through its C-ABI) against the FP64 oracle on seeded inputs.

Tolerances: a single FP64 smoother sweep to 1e-12 relative, converged solutions to 1e-8 relative,
FGMRES iteration counts within +-1 (CGS2 on the GPU vs MGS in the oracle). The assembled matrix
and the transfers agree to rounding (1e-13 / 1e-14); the cell inverses to the rounding error of
an explicit inverse, eps * cond(J_T) (bounded here by 1e-9 relative).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from helpers import gpu_hierarchy, lattice_to_gpu, oracle_hierarchy, oracle_lattice_index, rel_max

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    "2d_k1_obs": synth.small_workload(2, 1, (6, 3), 2, obstacle=True, seed=21),
    "2d_k2_obs_3lev": synth.small_workload(2, 2, (4, 2), 3, obstacle=True, seed=22),
    "3d_k1_obs": synth.small_workload(3, 1, (3, 2, 2), 2, obstacle=True, seed=23),
    "c1": synth.WORKLOADS["c1_2d_k1"],
}

_cache = {}


def pair(name, smoother="additive", prec="f64"):
    key = (name, smoother, prec)
    if key not in _cache:
        wl = CASES[name]
        o = _cache.get(("oracle", name, smoother))
        if o is None:
            o = oracle_hierarchy(wl, variant=smoother)
            _cache[("oracle", name, smoother)] = o
        _cache[key] = (wl, o, gpu_hierarchy(wl, prec, smoother))
    return _cache[key]


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("name", list(CASES))
def test_dof_numbering(name):
    wl, o, h = pair(name)
    for g, lev in enumerate(o.levels):
        np.testing.assert_array_equal(h.dof_lattice_index(g), oracle_lattice_index(lev))


@pytest.mark.parametrize("name", list(CASES))
def test_jacobian_all_levels(name):
    wl, o, h = pair(name)
    for g in range(wl.n_levels):
        Jg = h.copy_jacobian(g)
        Jo = o.J[g]
        diff = abs(Jg - Jo).max()
        assert diff <= 1e-13 * abs(Jo).max(), (g, diff)


@pytest.mark.parametrize("name", ["2d_k1_obs", "2d_k2_obs_3lev", "3d_k1_obs"])
def test_cell_inverses(name):
    from oracle import solvers
    wl, o, h = pair(name)
    for g in range(1, wl.n_levels):
        inv = h.copy_cell_inverses(g)
        JT = solvers.cell_matrices(o.J[g], o.levels[g].idx)
        eye = np.einsum("cij,cjk->cik", inv, JT)
        assert np.abs(eye - np.eye(JT.shape[1])).max() < 1e-9
        assert rel_max(inv, o.inv[g]) < 1e-9


@pytest.mark.parametrize("name", ["2d_k1_obs", "2d_k2_obs_3lev", "3d_k1_obs"])
@pytest.mark.parametrize("smoother", ["additive", "coloured", "overwrite"])
@pytest.mark.parametrize("transpose", [False, True])
def test_single_sweep(name, smoother, transpose):
    """One FP64 smoothing step from a random d: 1e-12 relative to the oracle."""
    from oracle import solvers
    wl, o, h = pair(name, smoother)
    g = wl.n_levels - 1
    rng = np.random.default_rng(31)
    r = rng.standard_normal(o.levels[g].N)
    d = rng.standard_normal(o.levels[g].N)
    expect = solvers.vanka_step(o.levels[g], o.J[g], o.inv[g], d, r, wl.omega, smoother, transpose)
    dg = dev(d)
    h.vanka_sweep(g, dev(r), dg, transpose=transpose)
    assert rel_max(dg.cpu().numpy(), expect) < 1e-12


@pytest.mark.parametrize("name", list(CASES))
def test_spmv_and_transpose(name):
    wl, o, h = pair(name)
    rng = np.random.default_rng(32)
    for g in range(wl.n_levels):
        x = rng.standard_normal(o.levels[g].N)
        for tr in (False, True):
            y = torch.zeros(o.levels[g].N, dtype=torch.float64, device="cuda")
            h.spmv(g, dev(x), y, transpose=tr)
            A = o.J[g].T if tr else o.J[g]
            assert rel_max(y.cpu().numpy(), A @ x) < 1e-13


@pytest.mark.parametrize("name", list(CASES))
def test_transfers(name):
    wl, o, h = pair(name)
    rng = np.random.default_rng(33)
    for g in range(1, wl.n_levels):
        xf = rng.standard_normal(o.levels[g].N)
        xc = rng.standard_normal(o.levels[g - 1].N)
        rc = torch.zeros(o.levels[g - 1].N, dtype=torch.float64, device="cuda")
        h.restrict(g, dev(xf), rc)
        assert rel_max(rc.cpu().numpy(), o.P[g].T @ xf) < 1e-14
        base = rng.standard_normal(o.levels[g].N)
        yf = dev(base)
        h.prolongate_add(g, dev(xc), yf)
        assert rel_max(yf.cpu().numpy(), base + o.P[g] @ xc) < 1e-14


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("transpose", [False, True])
def test_coarse_solve(name, transpose):
    wl, o, h = pair(name)
    r = np.random.default_rng(34).standard_normal(o.levels[0].N)
    d = torch.zeros_like(dev(r))
    h.coarse_solve(dev(r), d, transpose=transpose)
    A = (o.J[0].T if transpose else o.J[0]).tocsc()
    assert rel_max(d.cpu().numpy(), spla.spsolve(A, r)) < 1e-10


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("smoother", ["additive", "coloured"])
def test_vcycle(name, smoother):
    wl, o, h = pair(name, smoother)
    r = np.random.default_rng(35).standard_normal(o.fine.N)
    d = torch.zeros_like(dev(r))
    h.vcycle(dev(r), d)
    assert rel_max(d.cpu().numpy(), o.vcycle(r)) < 1e-10


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("smoother", ["additive", "coloured", "overwrite"])
def test_gmres_solution_and_iterations(name, smoother):
    wl, o, h = pair(name, smoother)
    b = o.fine.dofs_from_lattice(synth.random_rhs(wl))
    x_o, info_o = o.solve(b)
    x = torch.zeros_like(dev(b))
    info = h.gmres_solve(dev(b), x, rtol=wl.rtol, restart=wl.restart)
    assert info["converged"] and info["rel_res_true"] <= 2 * wl.rtol
    assert abs(info["iters"] - info_o["iters"]) <= 1, (info, info_o)
    xd = spla.spsolve(o.J[-1].tocsc(), b)
    assert rel_max(x.cpu().numpy(), xd) < 1e-8
    assert rel_max(x.cpu().numpy(), x_o) < 1e-8


@pytest.mark.parametrize("name", ["2d_k1_obs", "3d_k1_obs"])
def test_adjoint_solve(name):
    wl, o, h = pair(name)
    b = np.random.default_rng(36).standard_normal(o.fine.N)
    x_o, info_o = o.solve(b, transpose=True)
    x = torch.zeros_like(dev(b))
    info = h.gmres_solve(dev(b), x, rtol=wl.rtol, transpose=True)
    assert abs(info["iters"] - info_o["iters"]) <= 1
    assert rel_max(x.cpu().numpy(), spla.spsolve(o.J[-1].T.tocsc(), b)) < 1e-8


@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("name", ["c1", "3d_k1_obs"])
def test_mixed_precision_inverses(name, prec):
    """FP32/BF16 cell inverses inside FP64 FGMRES still reach 1e-8 and the FP64 solution."""
    wl, o, h = pair(name, "additive", prec)
    b = o.fine.dofs_from_lattice(synth.random_rhs(wl))
    x = torch.zeros_like(dev(b))
    info = h.gmres_solve(dev(b), x, rtol=1e-8)
    assert info["converged"] and info["rel_res_true"] <= 2e-8
    xd = spla.spsolve(o.J[-1].tocsc(), b)
    err = rel_max(x.cpu().numpy(), xd)
    assert err < 1e-6, err
    inv = h.copy_cell_inverses(wl.n_levels - 1)
    bound = 2**-8 if prec == "bf16" else 2**-23
    assert rel_max(inv, o.inv[-1]) < 2 * bound


def test_host_buffer_solve_matches_device_solve():
    wl, o, h = pair("c1")
    b = o.fine.dofs_from_lattice(synth.random_rhs(wl))
    x = torch.zeros_like(dev(b))
    h.gmres_solve(dev(b), x, rtol=1e-10)
    bh = torch.from_numpy(b).pin_memory()
    xh = torch.zeros_like(bh).pin_memory()
    info = h.gmres_solve_host(bh, xh, rtol=1e-10)
    assert info["converged"]
    np.testing.assert_array_equal(xh.numpy(), x.cpu().numpy())


def test_deterministic_repeat():
    wl, o, h = pair("2d_k1_obs")
    b = dev(np.random.default_rng(37).standard_normal(o.fine.N))
    x1, x2 = torch.zeros_like(b), torch.zeros_like(b)
    h.gmres_solve(b, x1)
    h.gmres_solve(b, x2)
    assert torch.equal(x1, x2)


def test_error_statuses():
    from paper_2107_10561_gb300 import Hierarchy, _lib
    wl, o, h = pair("2d_k1_obs")
    # maximum iterations reached -> NOT_CONVERGED with the last iterate and info filled
    b = dev(np.random.default_rng(38).standard_normal(o.fine.N))
    x = torch.zeros_like(b)
    info = h.gmres_solve(b, x, rtol=1e-14, max_iter=1, raise_on_fail=False)
    assert info["status"] == "STM_ERR_NOT_CONVERGED" and info["iters"] == 1
    # non-finite right-hand side
    bn = b.clone()
    bn[3] = float("nan")
    info = h.gmres_solve(bn, x, raise_on_fail=False)
    assert info["status"] == "STM_ERR_NONFINITE"
    # invalid parameters
    with pytest.raises(_lib.StmError) as e:
        Hierarchy(_bad_params(wl))
    assert e.value.status == _lib.STM_ERR_INVALID_ARG
    # wrong sizes are rejected by the binding before reaching the library
    with pytest.raises(ValueError):
        h.vcycle(b[:-1], x[:-1])


def _bad_params(wl):
    from helpers import gpu_params
    p = gpu_params(wl)
    p.dim = 4
    return p


def test_singular_cell_reported():
    """A non-finite linearisation point (injected on the host) makes every cell pivot non-finite:
    factor_cells reports STM_ERR_SINGULAR_CELL with the level and cell, without faulting."""
    from paper_2107_10561_gb300 import _lib
    wl = CASES["2d_k1_obs"]
    h = gpu_hierarchy(wl, factor=False)
    X = lattice_to_gpu(h, synth.linearisation_point(wl))
    X[:] = float("nan")
    h.assemble_jacobian(X)
    with pytest.raises(_lib.StmError) as e:
        h.factor_cells()
    assert e.value.status == _lib.STM_ERR_SINGULAR_CELL
    assert e.value.bad_level >= 1 and e.value.bad_cell >= 0


@pytest.mark.parametrize("name", ["2d_k1_obs", "2d_k2_obs_3lev", "3d_k1_obs"])
@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_single_sweep_mixed_precision(name, prec):
    """Additive step with FP32/BF16 inverses against the oracle with the same storage rounding
    (inverse rounded to the storage type, residual to FP32, products summed in FP64); the GPU
    accumulates in FP32, hence 1e-5 relative."""
    from oracle import solvers
    wl, o, h = pair(name, "additive", prec)
    g = wl.n_levels - 1
    lev = o.levels[g]
    rng = np.random.default_rng(38)
    r = rng.standard_normal(lev.N)
    d = rng.standard_normal(lev.N)
    from helpers import round_storage
    inv_r = round_storage(o.inv[g], prec)
    t = (r - o.J[g] @ d).astype(np.float32).astype(np.float64)
    y = np.einsum("cij,cj->ci", inv_r, t[lev.idx])
    corr = np.zeros(lev.N)
    np.add.at(corr, lev.idx.ravel(), y.ravel())
    expect = d + wl.omega * corr / solvers.multiplicity(lev)
    dg = dev(d)
    h.vanka_sweep(g, dev(r), dg)
    assert rel_max(dg.cpu().numpy(), expect) < 1e-5


def test_vcycles_replayed_as_graphs():
    """A plain solve replays its V-cycles from CUDA graphs (a refused capture would fall back to direct
    launches silently otherwise); with event profiling on they are launched directly."""
    wl, o, h = pair("3d_k1_obs")
    b = dev(np.random.default_rng(41).standard_normal(o.fine.N))
    x = torch.zeros_like(b)
    assert h.gmres_solve(b, x)["graphs"]
    h.profile_enable(True)
    x.zero_()
    assert not h.gmres_solve(b, x)["graphs"]
    h.profile_enable(False)
