"""Parity at the benchmark's full sizes, in the launch configuration bench.py times.

The 2D dG(2) channel c2_2d_k2 (536,448 DoFs, 5 levels): the complete oracle is affordable, so the whole FGMRES solve is
compared (both to rtol 1e-10; iterations +-1, solutions within 1e-8 with FP64 inverses and 1e-7
with BF16 inverses).
The 3D dG(1) channel c3_3d_k1 (962,208 DoFs, 3 levels): sampled outputs the oracle computes one by one: rows of J (from the
element matrices of the cells around a DoF), cell inverses (J_T from its 3x3x3 cell neighbourhood),
and one smoothing step at sampled DoFs; plus properties that hold at any size (true residual of
the converged solve, exact prolongation of a coarse polynomial).
"""
import numpy as np
import pytest

import synth
from helpers import gpu_hierarchy, rel_max

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.mark.timeout(900)
def test_c2_2d_k2_full_solve_against_oracle():
    """Both solves to rtol 1e-10: the iterates then agree with each other to ~cond * 1e-10."""
    from oracle import solvers
    wl = synth.WORKLOADS["c2_2d_k2"]
    o = solvers.Hierarchy(wl, synth.linearisation_point(wl))
    b = o.fine.dofs_from_lattice(synth.random_rhs(wl))
    x_o, info_o = o.solve(b, rtol=1e-10)
    assert info_o["converged"]
    for prec, tol in (("f64", 1e-8), ("bf16", 1e-7)):
        h = gpu_hierarchy(wl, prec)
        x = torch.zeros(o.fine.N, dtype=torch.float64, device="cuda")
        info = h.gmres_solve(torch.from_numpy(b).cuda(), x, rtol=1e-10)
        assert info["converged"] and info["rel_res_true"] <= 2e-10
        if prec == "f64":
            assert abs(info["iters"] - info_o["iters"]) <= 1, (info, info_o)
        assert rel_max(x.cpu().numpy(), x_o) < tol
        h.close()


@pytest.mark.timeout(900)
def test_c3_3d_k1_two_level_full_solve_against_oracle():
    """The 3D dG(1) channel of c3_3d_k1 with one refinement level fewer (fine 32x8x8 minus the obstacle,
    127,920 DoFs, n = 170): the complete oracle solve is affordable there. Both solves to rtol 1e-10;
    FP64 inverses: iterations +-1 and the solution within 1e-8; FP32 / BF16 inverses (FP64 defects):
    the solution within 1e-7."""
    import dataclasses

    from oracle import solvers
    wl = dataclasses.replace(synth.WORKLOADS["c3_3d_k1"], n_levels=2)
    o = solvers.Hierarchy(wl, synth.linearisation_point(wl))
    b = o.fine.dofs_from_lattice(synth.random_rhs(wl))
    x_o, info_o = o.solve(b, rtol=1e-10)
    assert info_o["converged"]
    for prec, tol in (("f64", 1e-8), ("f32", 1e-7), ("bf16", 1e-7)):
        h = gpu_hierarchy(wl, prec)
        x = torch.zeros(o.fine.N, dtype=torch.float64, device="cuda")
        info = h.gmres_solve(torch.from_numpy(b).cuda(), x, rtol=1e-10)
        assert info["converged"] and info["rel_res_true"] <= 1e-10
        if prec == "f64":
            assert abs(info["iters"] - info_o["iters"]) <= 1, (info, info_o)
        assert rel_max(x.cpu().numpy(), x_o) < tol, prec
        h.close()


# ---------------------------------------------------------------------------------------------
# c3_3d_k1: sampled checks
# ---------------------------------------------------------------------------------------------
def _fine_level(wl):
    from oracle import fem
    f = 2 ** (wl.n_levels - 1)
    return fem.Level(wl.dim, wl.k, wl.fine_cells, wl.length, tuple(x * f for x in wl.obstacle_lo),
                     tuple(x * f for x in wl.obstacle_hi))


class LocalAssembler:
    """Rows and cell blocks of the assembled J from element matrices of the cells that touch them."""

    def __init__(self, wl, lev, X_lin):
        self.wl, self.lev, self.X = wl, lev, X_lin
        self.cache = {}
        self.cells_of_node = {}
        cn = lev.cell_nodes
        for c in range(lev.C):
            for nd in cn[c]:
                self.cells_of_node.setdefault(int(nd), []).append(c)

    def element(self, cells):
        from oracle import fem
        need = [c for c in cells if c not in self.cache]
        if need:
            E = fem.element_matrices(self.lev, np.array(need), self.X, self.wl.tau, self.wl.nu, self.wl.gamma1,
                                     self.wl.gamma2)
            for c, e in zip(need, E):
                self.cache[c] = e
        return [self.cache[c] for c in cells]

    def cells_of_dof(self, dof):
        lev = self.lev
        a, r = divmod(dof, lev.block)
        if r < lev.dim * lev.R:
            return self.cells_of_node[int(r % lev.R)]
        return [int((r - lev.dim * lev.R) // lev.np_)]

    def row(self, dof):
        if ("row", dof) in self.cache:
            return self.cache[("row", dof)]
        out = {}
        cells = self.cells_of_dof(dof)
        for c, E in zip(cells, self.element(cells)):
            loc = np.nonzero(self.lev.idx[c] == dof)[0][0]
            for j, col in enumerate(self.lev.idx[c]):
                out[int(col)] = out.get(int(col), 0.0) + E[loc, j]
        self.cache[("row", dof)] = out
        return out

    def cell_matrix(self, c):
        idx = self.lev.idx[c]
        pos = {int(g): k for k, g in enumerate(idx)}
        JT = np.zeros((len(idx), len(idx)))
        touching = sorted({cc for nd in self.lev.cell_nodes[c] for cc in self.cells_of_node[int(nd)]})
        for cc, E in zip(touching, self.element(touching)):
            for i, gi in enumerate(self.lev.idx[cc]):
                if int(gi) not in pos:
                    continue
                for j, gj in enumerate(self.lev.idx[cc]):
                    if int(gj) in pos:
                        JT[pos[int(gi)], pos[int(gj)]] += E[i, j]
        return JT


@pytest.fixture(scope="module")
def c3():
    wl = synth.WORKLOADS["c3_3d_k1"]
    lev = _fine_level(wl)
    X_lin = lev.dofs_from_lattice(synth.linearisation_point(wl))
    h = gpu_hierarchy(wl, "f64")
    yield wl, lev, X_lin, h, LocalAssembler(wl, lev, X_lin)
    h.close()


@pytest.mark.timeout(600)
def test_c3_3d_k1_sampled_jacobian_rows(c3):
    wl, lev, X_lin, h, la = c3
    J = h.copy_jacobian(h.finest)
    rng = np.random.default_rng(71)
    for dof in rng.choice(lev.N, 40, replace=False):
        ref = la.row(int(dof))
        got = J[int(dof)]
        cols = np.array(sorted(ref))
        vals = np.array([ref[c] for c in cols])
        g = np.asarray(got[:, cols].todense()).ravel()
        assert np.abs(g - vals).max() <= 1e-13 * max(np.abs(vals).max(), 1e-300), dof
        # entries of the GPU row outside the oracle's support are structural zeros
        extra = np.setdiff1d(got.indices, cols)
        assert np.abs(np.asarray(got[:, extra].todense())).max(initial=0.0) <= 1e-15 * np.abs(vals).max()


@pytest.mark.timeout(600)
def test_c3_3d_k1_sampled_cell_inverses_and_sweep(c3):
    wl, lev, X_lin, h, la = c3
    inv_all = h.copy_cell_inverses(h.finest)
    rng = np.random.default_rng(72)
    cells = rng.choice(lev.C, 6, replace=False)
    for c in cells:
        JT = la.cell_matrix(int(c))
        Inv = np.linalg.inv(JT)
        assert rel_max(inv_all[c], Inv) < 1e-9
        assert np.abs(inv_all[c] @ JT - np.eye(JT.shape[0])).max() < 1e-9
    # one additive smoothing step, checked at the DoFs of one sampled cell
    r = rng.standard_normal(lev.N)
    d = rng.standard_normal(lev.N)
    dg = torch.from_numpy(d).cuda()
    h.vanka_sweep(h.finest, torch.from_numpy(r).cuda(), dg)
    dnew = dg.cpu().numpy()
    c0 = int(cells[0])
    m = np.zeros(lev.N)
    np.add.at(m, lev.idx.ravel(), 1.0)
    for dof in lev.idx[c0][:: 17]:
        owners = la.cells_of_dof(int(dof))
        corr = 0.0
        for T in owners:
            idxT = lev.idx[T]
            t = np.array([r[g] - sum(v * d[col] for col, v in la.row(int(g)).items()) for g in idxT])
            y = inv_all[T] @ t
            corr += y[np.nonzero(idxT == dof)[0][0]]
        expect = d[dof] + wl.omega * corr / m[dof]
        assert abs(dnew[dof] - expect) <= 1e-11 * max(abs(expect), 1.0), dof


@pytest.mark.timeout(600)
def test_c3_3d_k1_converged_residual_and_prolongation(c3):
    wl, lev, X_lin, h, la = c3
    b = torch.from_numpy(lev.dofs_from_lattice(synth.random_rhs(wl))).cuda()
    x = torch.zeros_like(b)
    info = h.gmres_solve(b, x, rtol=1e-8)
    assert info["converged"] and info["rel_res_true"] <= 2e-8
    # independent residual through the structured SpMV
    y = torch.empty_like(b)
    h.spmv(h.finest, x, y)
    assert float(torch.linalg.norm(b - y) / torch.linalg.norm(b)) <= 2e-8
    # P reproduces a coarse Q2 polynomial exactly at full size
    from oracle import fem
    g = h.finest
    f = 2 ** (wl.n_levels - 2)
    coarse = fem.Level(wl.dim, wl.k, wl.cells_at(wl.n_levels - 1), wl.length,
                       tuple(xx * f for xx in wl.obstacle_lo), tuple(xx * f for xx in wl.obstacle_hi))

    def nodal(level, fn):
        co = np.stack(np.unravel_index(level.lat_of_node, level.lshape[::-1])[::-1], axis=1) * (level.h / 2)
        v = fn(co)
        out = np.zeros(level.N)
        for a in range(level.k + 1):
            for i in range(level.dim):
                out[a * level.block + i * level.R: a * level.block + (i + 1) * level.R] = v * (i + 1 + a)
        return out
    q = lambda xx: 1.0 + xx[:, 0] ** 2 * xx[:, 1] - 0.5 * xx[:, 2] ** 2 + xx[:, 1] * xx[:, 2]
    fine = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
    h.prolongate_add(g, torch.from_numpy(nodal(coarse, q)).cuda(), fine)
    expect = nodal(lev, q)
    vel = np.zeros(lev.N, dtype=bool)
    for a in range(lev.k + 1):
        vel[a * lev.block: a * lev.block + lev.dim * lev.R] = True
    assert np.abs(fine.cpu().numpy()[vel] - expect[vel]).max() < 1e-12 * np.abs(expect).max()
