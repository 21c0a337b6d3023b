"""Pins of the oracle's transfer, cell inverses, Vanka smoothers, V-cycle and FGMRES (CPU only)."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import fem, solvers


def _levels(dim, k, coarse, obstacle):
    L = (2.2, 0.41) if dim == 2 else (2.5, 0.41, 0.41)
    if obstacle:
        lo = (1, 1) + ((0,) if dim == 3 else ())
        hi = (2, 2) + ((coarse[2],) if dim == 3 else ())
    else:
        lo = hi = (0,) * dim
    c = fem.Level(dim, k, coarse, L, lo, hi)
    f = fem.Level(dim, k, tuple(2 * x for x in coarse), L, tuple(2 * x for x in lo), tuple(2 * x for x in hi))
    return c, f


def _node_coords(lev):
    return np.stack(np.unravel_index(lev.lat_of_node, lev.lshape[::-1])[::-1], axis=1) * (lev.h / 2)


@pytest.mark.parametrize("dim,k,coarse,obstacle", [(2, 1, (4, 3), True), (2, 2, (4, 2), False), (3, 1, (3, 3, 2), True)])
def test_prolongation_reproduces_coarse_polynomials(dim, k, coarse, obstacle):
    """Sec. 4.1: P interpolates; every function of the coarse space is reproduced exactly."""
    c, f = _levels(dim, k, coarse, obstacle)
    P = fem.prolongation(c, f)
    rng = np.random.default_rng(0)
    # a global polynomial of degree <= 2 per variable lies in Q2 on every cell
    def q(x):
        out = 1.0 + 0.3 * x[:, 0] - 0.7 * x[:, 0] ** 2 * x[:, 1] ** 2 + x[:, 1]
        if dim == 3:
            out = out + x[:, 2] ** 2 * x[:, 0]
        return out
    xc, xf = _node_coords(c), _node_coords(f)
    # pressure: a linear function, coefficients of the orthonormal Legendre basis per cell
    a = rng.standard_normal(dim + 1)
    def pcoef(lev):
        # p(x) = a0 + sum a_m x_m ; on a cell with origin o and size h: x_m = o_m + h_m xhat_m
        o = lev.cell_origin()
        out = np.zeros((lev.C, dim + 1))
        out[:, 0] = a[0] + (a[1:] * (o + lev.h / 2)).sum(1)
        for m in range(dim):
            out[:, 1 + m] = a[1 + m] * lev.h[m] / (2 * math.sqrt(3.0))
        return out.ravel()
    Xc = np.concatenate([np.concatenate([q(xc) * (i + 1) for i in range(dim)] + [pcoef(c)]) * (l + 1) for l in range(k + 1)])
    Xf = np.concatenate([np.concatenate([q(xf) * (i + 1) for i in range(dim)] + [pcoef(f)]) * (l + 1) for l in range(k + 1)])
    np.testing.assert_allclose(P @ Xc, Xf, atol=1e-12)


def test_q2_prolongation_weights_and_pressure_child_map():
    c, f = _levels(2, 0, (1, 1), False)
    P = fem.prolongation(c, f).toarray()
    # fine node at x = 1/4 (lattice (1,0)) -> coarse nodes (0,0), (1,0), (2,0) with 3/8, 3/4, -1/8
    nf = f.node_of_lat[1]
    row = P[nf, :c.R]
    np.testing.assert_allclose([row[c.node_of_lat[0]], row[c.node_of_lat[1]], row[c.node_of_lat[2]]],
                               [3 / 8, 3 / 4, -1 / 8], atol=1e-15)
    # pressure: left child c0' = c0 - (sqrt3/2) c1, c1' = c1/2, c2' = c2 - (sqrt3/2)... (x only)
    Pp = P[2 * f.R:, 2 * c.R:]
    s = math.sqrt(3.0) / 2
    child_ll = Pp[0:3]  # fine cell (0,0)
    np.testing.assert_allclose(child_ll, [[1, -s, -s], [0, 0.5, 0], [0, 0, 0.5]], atol=1e-14)
    child_rl = Pp[3:6]  # fine cell (1,0)
    np.testing.assert_allclose(child_rl, [[1, s, -s], [0, 0.5, 0], [0, 0, 0.5]], atol=1e-14)


def _hier(wl, variant=solvers.ADDITIVE):
    return solvers.Hierarchy(wl, synth.linearisation_point(wl), variant=variant)


@pytest.fixture(scope="module")
def h2d():
    return _hier(synth.small_workload(2, 1, (6, 3), 2, obstacle=True, seed=11))


def test_cell_inverse_identity(h2d):
    g = 1
    lev = h2d.levels[g]
    JT = solvers.cell_matrices(h2d.J[g], lev.idx)
    err = np.abs(np.einsum("cij,cjk->cik", h2d.inv[g], JT) - np.eye(lev.n)).max()
    assert err < 1e-10


def test_partition_of_unity(h2d):
    lev = h2d.fine
    m = solvers.multiplicity(lev)
    acc = np.zeros(lev.N)
    np.add.at(acc, lev.idx.ravel(), 1.0)
    np.testing.assert_allclose(acc / m, 1.0)
    assert m.min() >= 1
    assert m.max() == 2**lev.dim


def test_colours_share_no_dof(h2d):
    lev = h2d.fine
    for col in range(2**lev.dim):
        cells = np.nonzero(lev.colour == col)[0]
        dofs = lev.idx[cells].ravel()
        assert np.unique(dofs).size == dofs.size


@pytest.mark.parametrize("variant", [solvers.ADDITIVE, solvers.COLOURED, solvers.OVERWRITE])
@pytest.mark.parametrize("transpose", [False, True])
def test_smoother_fixed_point(h2d, variant, transpose):
    g = 1
    lev, J = h2d.levels[g], h2d.J[g]
    r = np.random.default_rng(1).standard_normal(lev.N)
    A = (J.T if transpose else J).tocsc()
    d = spla.spsolve(A, r)
    d2 = solvers.vanka_step(lev, J, h2d.inv[g], d, r, 0.7, variant, transpose)
    np.testing.assert_allclose(d2, d, atol=1e-9 * np.abs(d).max())


@pytest.mark.parametrize("dim,k", [(2, 1), (2, 2), (3, 1)])
def test_one_cell_vanka_is_exact_solve(dim, k):
    """Single cell: J_T = J, so one undamped sweep from zero gives J^{-1} r."""
    L = (1.0,) * dim
    lev = fem.Level(dim, k, (1,) * dim, L, (0,) * dim, (0,) * dim)
    w = np.random.default_rng(2).standard_normal(lev.N)
    J = fem.assemble_jacobian(lev, w, 0.01, 1e-3)
    inv = solvers.cell_inverses(J, lev.idx)
    r = np.random.default_rng(3).standard_normal(lev.N)
    x = np.linalg.solve(J.toarray(), r)
    for variant in (solvers.ADDITIVE, solvers.COLOURED, solvers.OVERWRITE):
        d = solvers.vanka_step(lev, J, inv, np.zeros(lev.N), r, 1.0, variant)
        np.testing.assert_allclose(d, x, atol=1e-12 * np.abs(x).max())


def test_additive_sweep_against_explicit_sum(h2d):
    """d + omega W sum_T R_T^T J_T^{-1} R_T (r - J d) written with explicit restriction matrices."""
    g = 1
    lev, J = h2d.levels[g], h2d.J[g]
    rng = np.random.default_rng(4)
    r, d = rng.standard_normal(lev.N), rng.standard_normal(lev.N)
    JT = solvers.cell_matrices(J, lev.idx)
    B = np.zeros((lev.N, lev.N))
    for c in range(lev.C):
        Rt = sp.csr_matrix((np.ones(lev.n), (np.arange(lev.n), lev.idx[c])), shape=(lev.n, lev.N)).toarray()
        B += Rt.T @ np.linalg.solve(JT[c], Rt)
    m = np.zeros(lev.N)
    for c in range(lev.C):
        m[lev.idx[c]] += 1
    expect = d + 0.7 * (B @ (r - J @ d)) / m
    got = solvers.vanka_step(lev, J, h2d.inv[g], d, r, 0.7)
    np.testing.assert_allclose(got, expect, atol=1e-11 * np.abs(expect).max())


def test_two_grid_without_smoothing_is_coarse_correction(h2d):
    """V(0,0) on two levels returns P J_1^{-1} P^T r (Algorithm 1 with no smoothing steps)."""
    import dataclasses
    wl0 = h2d.wl
    h2d.wl = dataclasses.replace(wl0, nu1=0, nu2=0)
    try:
        r = np.random.default_rng(5).standard_normal(h2d.fine.N)
        d = h2d.vcycle(r)
        expect = h2d.P[1] @ spla.spsolve(h2d.J[0].tocsc(), h2d.P[1].T @ r)
        np.testing.assert_allclose(d, expect, atol=1e-10 * np.abs(expect).max())
    finally:
        h2d.wl = wl0


def test_fgmres_full_krylov_is_exact():
    """Unpreconditioned GMRES with restart >= n terminates with the exact solution (textbook)."""
    rng = np.random.default_rng(6)
    A = rng.standard_normal((25, 25)) + 5 * np.eye(25)
    b = rng.standard_normal(25)
    x, info = solvers.fgmres(lambda v: A @ v, lambda v: v, b, restart=30, rtol=1e-13)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), atol=1e-10)
    assert info["iters"] <= 25


@pytest.mark.parametrize("variant", [solvers.ADDITIVE, solvers.COLOURED, solvers.OVERWRITE])
def test_gmres_solution_matches_direct_solve_c1(variant):
    wl = synth.WORKLOADS["c1_2d_k1"]
    h = _hier(wl, variant)
    b = h.fine.dofs_from_lattice(synth.random_rhs(wl))
    x, info = h.solve(b)
    assert info["converged"]
    xd = spla.spsolve(h.J[-1].tocsc(), b)
    assert np.abs(x - xd).max() / np.abs(xd).max() < 1e-8
    assert info["iters"] < 60


def test_transposed_solve_matches_direct(h2d):
    b = np.random.default_rng(8).standard_normal(h2d.fine.N)
    x, info = h2d.solve(b, transpose=True)
    assert info["converged"]
    xd = spla.spsolve(h2d.J[-1].T.tocsc(), b)
    assert np.abs(x - xd).max() / np.abs(xd).max() < 1e-8


def test_mesh_independent_iterations():
    """Sec. 5.1: GMG-preconditioned GMRES iteration counts stay (almost) grid independent."""
    its = []
    for levels in (2, 3):
        wl = synth.small_workload(2, 1, (8, 2), levels, obstacle=True, seed=12)
        h = _hier(wl)
        b = h.fine.dofs_from_lattice(synth.random_rhs(wl))
        _, info = h.solve(b)
        its.append(info["iters"])
    assert abs(its[1] - its[0]) <= 3, its
