"""Pins of the oracle's coloured multiplicative and literal overwrite Vanka sweeps (CPU only).

Sec. 4.2 leaves the update of DoFs shared by several cells to the order of the cell loop ("the last
update wins"). The oracle offers two order-defined readings besides the additive one:
  * coloured: the 2^d colours are visited in ascending order, each colour's cells see the residual
    refreshed after the previous colour (block Gauss-Seidel over colours);
  * overwrite: one residual for all cells, and every DoF keeps the correction of the highest-index
    cell containing it.
The checks below are written with dense matrices and explicit index sets, so that a Jacobi-style
coloured loop (one residual for every colour), a reversed colour order, or an overwrite that keeps
the lowest-index cell each fail at least one of them.
"""
import numpy as np
import pytest

from oracle import fem, solvers


def _mesh(cells, k=1, seed=0):
    lev = fem.Level(2, k, cells, (1.0, 0.5), (0, 0), (0, 0))
    rng = np.random.default_rng(seed)
    X = 0.3 * rng.standard_normal(lev.N)
    J = fem.assemble_jacobian(lev, X, 0.01, 1e-3)
    inv = solvers.cell_inverses(J, lev.idx)
    r, d = rng.standard_normal(lev.N), rng.standard_normal(lev.N)
    return lev, J, inv, r, d


def _local_solve(Jd, dofs, rhs):
    return np.linalg.solve(Jd[np.ix_(dofs, dofs)], rhs[dofs])


@pytest.mark.parametrize("omega", [1.0, 0.6])
def test_coloured_two_cells_is_block_gauss_seidel(omega):
    """1x2 cells, two colours sharing one face: cell 0 is corrected first, then cell 1 from the
    residual recomputed after cell 0's correction."""
    lev, J, inv, r, d = _mesh((2, 1))
    assert list(lev.colour) == [0, 1]
    Jd = J.toarray()
    A, B = lev.idx[0], lev.idx[1]
    assert np.intersect1d(A, B).size > 0  # the shared face couples the two local solves
    d1 = d.copy()
    d1[A] += omega * _local_solve(Jd, A, r - Jd @ d)
    d2 = d1.copy()
    d2[B] += omega * _local_solve(Jd, B, r - Jd @ d1)
    got = solvers.vanka_step(lev, J, inv, d, r, omega, solvers.COLOURED)
    np.testing.assert_allclose(got, d2, rtol=0, atol=1e-10 * np.abs(d2).max())
    # the Jacobi reading (one residual for both cells) differs on this mesh
    t0 = r - Jd @ d
    jac = d.copy()
    jac[A] += omega * _local_solve(Jd, A, t0)
    jac[B] = d[B] + omega * _local_solve(Jd, B, t0)
    assert np.abs(jac - d2).max() > 1e-6 * np.abs(d2).max()


def test_coloured_four_cells_in_ascending_colour_order():
    """2x2 cells, one cell per colour: cells 0, 1, 2, 3 (colours 0, 1, 2, 3) in that order."""
    lev, J, inv, r, d = _mesh((2, 2), seed=1)
    assert list(lev.colour) == [0, 1, 2, 3]
    Jd = J.toarray()
    x = d.copy()
    for c in range(4):
        x[lev.idx[c]] += 0.8 * _local_solve(Jd, lev.idx[c], r - Jd @ x)
    got = solvers.vanka_step(lev, J, inv, d, r, 0.8, solvers.COLOURED)
    np.testing.assert_allclose(got, x, rtol=0, atol=1e-10 * np.abs(x).max())


@pytest.mark.parametrize("k", [1, 2])
def test_coloured_undamped_leaves_no_residual_on_last_colour(k):
    """omega = 1 on 3x2 cells, where colour 3 (the last) holds the single cell (1, 1): that cell is
    solved exactly against the residual that includes every earlier colour's correction, and nothing
    changes its DoFs afterwards, so r - J d vanishes on them. A sweep that reused one residual, or
    visited the colours in another order, leaves a residual there."""
    lev, J, inv, r, d = _mesh((3, 2), k=k, seed=2)
    last = np.nonzero(lev.colour == 3)[0]
    assert last.size == 1
    got = solvers.vanka_step(lev, J, inv, d, r, 1.0, solvers.COLOURED)
    res = r - J @ got
    dofs = lev.idx[last[0]]
    assert np.abs(res[dofs]).max() < 1e-9 * np.abs(r).max()
    first = np.unique(lev.idx[np.nonzero(lev.colour == 0)[0]].ravel())
    assert np.abs(res[np.setdiff1d(first, dofs)]).max() > 1e-6 * np.abs(r).max()


def test_overwrite_two_cells_highest_index_wins():
    """1x2 cells: one residual t = r - J d; DoFs of cell 1 (the shared face included) take cell 1's
    correction, the others cell 0's."""
    lev, J, inv, r, d = _mesh((2, 1), seed=3)
    Jd = J.toarray()
    t = r - Jd @ d
    A, B = lev.idx[0], lev.idx[1]
    expect = d.copy()
    expect[A] = d[A] + 0.7 * _local_solve(Jd, A, t)
    expect[B] = d[B] + 0.7 * _local_solve(Jd, B, t)
    got = solvers.vanka_step(lev, J, inv, d, r, 0.7, solvers.OVERWRITE)
    np.testing.assert_allclose(got, expect, rtol=0, atol=1e-10 * np.abs(expect).max())
    shared = np.intersect1d(A, B)
    yA = d.copy()
    yA[A] = d[A] + 0.7 * _local_solve(Jd, A, t)
    assert np.abs(got[shared] - yA[shared]).max() > 1e-6 * np.abs(expect).max()


def test_overwrite_centre_node_takes_last_cell():
    """2x2 cells: the centre node belongs to all four cells and carries the correction of cell 3;
    a DoF owned by cells 0 and 1 only carries cell 1's."""
    lev, J, inv, r, d = _mesh((2, 2), seed=4)
    Jd = J.toarray()
    t = r - Jd @ d
    got = solvers.vanka_step(lev, J, inv, d, r, 1.0, solvers.OVERWRITE)
    corr = [d[lev.idx[c]] + _local_solve(Jd, lev.idx[c], t) for c in range(4)]
    owners = {}
    for c in range(4):
        for a, i in enumerate(lev.idx[c]):
            owners.setdefault(int(i), []).append((c, a))
    for i, lst in owners.items():
        c, a = max(lst)
        assert abs(got[i] - corr[c][a]) <= 1e-10 * np.abs(got).max(), (i, lst)
    four = [i for i, lst in owners.items() if len(lst) == 4]
    two01 = [i for i, lst in owners.items() if sorted(c for c, _ in lst) == [0, 1]]
    assert four and two01
