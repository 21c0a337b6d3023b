"""Allocation-free additive Vanka correction, checked against the regular smoother.

Some callers cannot allocate device memory while they run: their device memory belongs to
another component's pool allocator, or the implicit device synchronisation of cudaMalloc/cudaFree
is not acceptable in their loop. stm_vanka_apply_noalloc serves them: it takes every input and
output from the caller and keeps its scratch in a fixed static device array.

This test calls it through the C-ABI twice in a row and compares both results with one additive
sweep of stm_vanka_sweep on the same cell inverses and residual (1e-12 relative, the single-sweep
tolerance of the other parity tests; the two differ only in FP64 summation order). The second call
also shows that the scratch left behind by the first call is cleared. It then feeds the oracle's own
cell inverses and residual through the same entry point and compares the result with the oracle's
additive sweep (same tolerance).
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
    return np.abs(a - b).max() / np.abs(b).max()


def test_noalloc_additive_correction_matches_vanka_sweep():
    from helpers import gpu_hierarchy
    from oracle import fem
    from paper_2107_10561_gb300 import _lib
    from paper_2107_10561_gb300.solver import vanka_apply_noalloc

    wl = synth.small_workload(2, 1, (6, 3), 2, obstacle=True, seed=41)
    h = gpu_hierarchy(wl, "f64", "additive")
    g = h.finest
    f = 2 ** (wl.n_levels - 1)
    lev = fem.Level(wl.dim, wl.k, wl.fine_cells, wl.length, tuple(x * f for x in wl.obstacle_lo),
                    tuple(x * f for x in wl.obstacle_hi))
    idx = torch.from_numpy(lev.idx.astype(np.int32)).cuda()
    inv_cm = torch.from_numpy(np.ascontiguousarray(h.copy_cell_inverses(g).transpose(0, 2, 1))).cuda()

    rng = np.random.default_rng(42)
    r = torch.from_numpy(rng.standard_normal(lev.N)).cuda()
    d0 = torch.from_numpy(rng.standard_normal(lev.N)).cuda()
    d_ref = d0.clone()
    h.vanka_sweep(g, r, d_ref)  # regular entry point: d + omega W sum_T R_T^T J_T^{-1} R_T (r - J d)
    Jd = torch.empty_like(d0)
    h.spmv(g, d0, Jd)
    t = r - Jd
    for _ in range(2):
        d = d0.clone()
        vanka_apply_noalloc(inv_cm, idx, t, d, wl.omega)
        torch.cuda.synchronize()
        assert _rel(d, d_ref) < 1e-12

    # the oracle's inverses and residual through the same entry point give the oracle's sweep
    from helpers import oracle_hierarchy
    from oracle import solvers

    ho = oracle_hierarchy(wl)
    lo, Jo, invo = ho.fine, ho.J[-1], ho.inv[-1]
    r_np, d_np = r.cpu().numpy(), d0.cpu().numpy()
    expect = solvers.vanka_step(lo, Jo, invo, d_np, r_np, wl.omega)
    t_o = torch.from_numpy(r_np - Jo @ d_np).cuda()
    inv_o = torch.from_numpy(np.ascontiguousarray(invo.transpose(0, 2, 1))).cuda()
    idx_o = torch.from_numpy(lo.idx.astype(np.int32)).cuda()
    for _ in range(2):
        d = d0.clone()
        vanka_apply_noalloc(inv_o, idx_o, t_o, d, wl.omega)
        torch.cuda.synchronize()
        got = d.cpu().numpy()
        assert np.abs(got - expect).max() / np.abs(expect).max() < 1e-12

    # sizes beyond the fixed scratch capacity are rejected before any launch
    big = torch.zeros(2**20 + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.StmError) as e:
        vanka_apply_noalloc(inv_cm, idx, big, big.clone(), wl.omega)
    assert e.value.status == _lib.STM_ERR_INVALID_ARG
    h.close()
