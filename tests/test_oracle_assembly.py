"""Pins of the oracle's slab Jacobian and load assembly (CPU only).

The manufactured-solution test fixes every term of the discrete Oseen operator (time derivative
and jump, diffusion, both convection terms, pressure couplings, Nitsche terms, do-nothing
outflow): a dropped term, a wrong sign or a transposed index destroys the O(h^3) / O(h^2) rates.
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fem

sympy = pytest.importorskip("sympy")


def _mms_functions(dim, k, nu):
    x, y, z, t = sympy.symbols("x y z t")
    X = [x, y, z][:dim]
    pi = sympy.pi
    tp = sum(t**j * (j + 1) / 2 for j in range(k + 1))  # polynomial of degree k in time
    if dim == 2:
        psi = sympy.sin(pi * x) * sympy.sin(pi * y) / pi + x**2 * y / 3
        v = [tp * sympy.diff(psi, y), -tp * sympy.diff(psi, x)]
        beta = [1 + y / 2, sympy.sin(pi * x) / 2]
        p = (1 + 2 * t) * sympy.cos(pi * x) * sympy.cos(pi * y / 2)
    else:
        psi = sympy.sin(pi * x) * sympy.sin(pi * y) * sympy.sin(pi * z) / pi
        phi = sympy.cos(pi * x / 2) * sympy.sin(pi * y) * sympy.cos(pi * z) / pi
        # v = curl(psi e_z) + curl(phi e_y)  (divergence free)
        v = [tp * (sympy.diff(psi, y) - sympy.diff(phi, z)), -tp * sympy.diff(psi, x), tp * sympy.diff(phi, x)]
        beta = [1 + y / 2, sympy.sin(pi * x) / 2, z / 3]
        p = (1 + 2 * t) * sympy.cos(pi * x) * sympy.cos(pi * y / 2) * sympy.cos(pi * z / 3)
    f = []
    for l in range(dim):
        e = sympy.diff(v[l], t)
        e += sum(beta[m] * sympy.diff(v[l], X[m]) for m in range(dim))
        e += sum(v[m] * sympy.diff(beta[l], X[m]) for m in range(dim))
        e -= nu * sum(sympy.diff(v[l], X[m], 2) for m in range(dim))
        e += sympy.diff(p, X[l])
        f.append(e)
    # do-nothing traction nu grad v . n - p n on x = L (n = e_x)
    tr = [nu * sympy.diff(v[l], x) - (p if l == 0 else 0) for l in range(dim)]
    lam = lambda exprs: sympy.lambdify((*X, t), exprs, "numpy")
    fv, vv, bv, pv, tv = lam(f), lam(v), lam(beta), lam(p), lam(tr)

    def vec(fn):
        def g(pts, tt=0.0):
            out = fn(*[pts[:, m] for m in range(dim)], tt)
            return np.stack([np.broadcast_to(np.asarray(o, dtype=float), pts.shape[:1]) for o in out], axis=1)
        return g

    def scal(fn):
        return lambda pts, tt=0.0: np.broadcast_to(np.asarray(fn(*[pts[:, m] for m in range(dim)], tt), dtype=float), pts.shape[:1])

    return dict(f=vec(fv), v=vec(vv), beta=vec(bv), p=scal(pv), traction=vec(tv))


def _mms_errors(dim, k, n, nu=0.1, tau=0.1):
    F = _mms_functions(dim, k, nu)
    lev = fem.Level(dim, k, (n,) * dim, (1.0,) * dim, (0,) * dim, (0,) * dim)
    # linearisation point: Q2 interpolant of beta at every time node
    coords = np.stack(np.unravel_index(lev.lat_of_node, lev.lshape[::-1])[::-1], axis=1) * (lev.h / 2)
    bn = F["beta"](coords)
    X_lin = np.zeros(lev.N)
    for l in range(k + 1):
        for i in range(dim):
            X_lin[l * lev.block + i * lev.R: l * lev.block + (i + 1) * lev.R] = bn[:, i]
    J = fem.assemble_jacobian(lev, X_lin, tau, nu)
    b = fem.assemble_load(lev, tau, nu, f=F["f"], g=F["v"], traction=F["traction"],
                          v_prev=lambda pts: F["v"](pts, 0.0))
    X = spla.spsolve(J.tocsc(), b)
    t_nodes = tau * fem.radau_right_nodes(k)
    return fem.l2_errors(lev, X, F["v"], F["p"], t_nodes)


@pytest.mark.parametrize("k", [1, 2])
def test_manufactured_solution_rates_2d(k):
    ns = [4, 8, 16]
    errs = [_mms_errors(2, k, n) for n in ns]
    ev = np.array([e[0].max() for e in errs])
    ep = np.array([e[1].max() for e in errs])
    rv = np.log2(ev[:-1] / ev[1:])
    rp = np.log2(ep[:-1] / ep[1:])
    assert rv[-1] > 2.8, (ev, rv)  # Q2 velocity: O(h^3) in L2
    assert rp[-1] > 1.8, (ep, rp)  # P1disc pressure: O(h^2) in L2


@pytest.mark.slow
def test_manufactured_solution_rates_3d():
    ns = [3, 6]
    errs = [_mms_errors(3, 1, n) for n in ns]
    ev = np.array([e[0].max() for e in errs])
    ep = np.array([e[1].max() for e in errs])
    assert math.log2(ev[0] / ev[1]) > 2.6, ev
    assert math.log2(ep[0] / ep[1]) > 1.6, ep


def _random_level(dim, k, cells, obstacle=True):
    lo = (1, 1) + ((0,) if dim == 3 else ())
    hi = (2, 2) + ((cells[2],) if dim == 3 else ())
    if not obstacle:
        lo = hi = (0,) * dim
    L = (2.2, 0.41) if dim == 2 else (2.5, 0.41, 0.41)
    return fem.Level(dim, k, cells, L, lo, hi)


@pytest.mark.parametrize("dim,k,cells", [(2, 1, (6, 3)), (2, 2, (4, 3)), (3, 1, (4, 3, 2))])
def test_newton_linearisation_is_exact(dim, k, cells):
    """J(w) delta = (c(w+delta) - c(w-delta))/2 for the quadratic convection residual c (Eq. linNewEq)."""
    lev = _random_level(dim, k, cells)
    rng = np.random.default_rng(3)
    w = rng.standard_normal(lev.N)
    delta = rng.standard_normal(lev.N)
    tau, nu = 0.01, 1e-3
    J = fem.assemble_jacobian(lev, w, tau, nu)
    J0 = fem.assemble_jacobian(lev, np.zeros(lev.N), tau, nu)
    lhs = (J - J0) @ delta
    rhs = (fem.convection_residual(lev, w + delta, tau) - fem.convection_residual(lev, w - delta, tau)) / 2
    np.testing.assert_allclose(lhs, rhs, atol=1e-12 * np.abs(rhs).max())


def test_velocity_block_symmetric_for_stokes_dg0():
    """w = 0, k = 0: symmetric Nitsche + diffusion + mass -> symmetric velocity block; B blocks antisymmetric."""
    lev = _random_level(2, 0, (6, 3))
    J = fem.assemble_jacobian(lev, np.zeros(lev.N), 0.01, 1e-3).toarray()
    nv = lev.dim * lev.R
    Avv = J[:nv, :nv]
    np.testing.assert_allclose(Avv, Avv.T, atol=1e-13 * np.abs(Avv).max())
    np.testing.assert_allclose(J[:nv, nv:], -J[nv:, :nv].T, atol=1e-15)
    assert np.abs(J[nv:, nv:]).max() == 0.0


def test_jacobian_affine_in_viscosity():
    lev = _random_level(2, 1, (6, 3))
    w = np.random.default_rng(5).standard_normal(lev.N)
    Js = [fem.assemble_jacobian(lev, w, 0.01, nu).toarray() for nu in (0.0, 1e-3, 2e-3)]
    np.testing.assert_allclose(Js[2] - 2 * Js[1] + Js[0], 0.0, atol=1e-13 * np.abs(Js[1]).max())


def test_element_sum_reproduces_global_matrix_structure():
    """Pressure rows couple only with the velocity of their own cell and time node (Mt diagonal)."""
    lev = _random_level(2, 2, (4, 3))
    w = np.random.default_rng(6).standard_normal(lev.N)
    J = fem.assemble_jacobian(lev, w, 0.01, 1e-3).tocsr()
    for l in range(lev.k + 1):
        for c in (0, lev.C - 1):
            row = l * lev.block + lev.dim * lev.R + c * lev.np_
            cols = J[row].indices[np.abs(J[row].data) > 1e-14]
            allowed = set(lev.idx[c, l * lev.nloc_t: l * lev.nloc_t + lev.nloc_v])
            assert set(cols) <= allowed


def test_workload_sizes():
    """DoF formula N = (k+1)(d R + n_p C) on the synthetic channel levels."""
    import synth
    expect = {
        "c1_2d_k1": [1572, 5956],
        "c2_2d_k2": [2343, 8844, 34320, 135168, 536448],
        "c4_2d_k1": [1562, 5896, 22880, 90112],
        "c3_3d_k1": [18000, 127920],
    }
    for name, ns in expect.items():
        wl = synth.WORKLOADS[name]
        for g, n_exp in enumerate(ns, start=1):
            f = 2 ** (g - 1)
            lev = fem.Level(wl.dim, wl.k, wl.cells_at(g), wl.length,
                            tuple(x * f for x in wl.obstacle_lo), tuple(x * f for x in wl.obstacle_hi))
            assert lev.N == n_exp, (name, g, lev.N)
