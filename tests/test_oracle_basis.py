"""Pins of the oracle's basis functions, quadrature and temporal matrices (CPU only)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import fem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def test_radau_nodes_closed_forms():
    # right Gauss-Radau points of [0,1] (Sec. 2.4: the slab end point is a node)
    np.testing.assert_allclose(fem.radau_right_nodes(0), [1.0], atol=1e-15)
    np.testing.assert_allclose(fem.radau_right_nodes(1), [1 / 3, 1.0], atol=1e-15)
    s6 = math.sqrt(6.0)
    np.testing.assert_allclose(fem.radau_right_nodes(2), [(4 - s6) / 10, (4 + s6) / 10, 1.0], atol=1e-14)


def test_time_matrices_dg1_closed_forms():
    # chi_0 = 3/2 (1 - s), chi_1 = 3/2 s - 1/2, integrated by hand
    Mt, D, T = fem.time_matrices(1, 1.0)
    np.testing.assert_allclose(Mt, [[3 / 4, 0], [0, 1 / 4]], atol=1e-15)
    np.testing.assert_allclose(D, [[9 / 8, 3 / 8], [-9 / 8, 5 / 8]], atol=1e-15)
    np.testing.assert_allclose(T[0, 0, 0], 27 / 32, atol=1e-15)
    np.testing.assert_allclose(T[0, 0, 1], -3 / 32, atol=1e-15)
    np.testing.assert_allclose(T[0, 1, 1], 3 / 32, atol=1e-15)
    np.testing.assert_allclose(T[1, 1, 1], 5 / 32, atol=1e-15)


@pytest.mark.parametrize("k", [0, 1, 2])
@pytest.mark.parametrize("tau", [1.0, 0.01])
def test_time_matrix_identities(k, tau):
    Mt, D, T = fem.time_matrices(k, tau)
    chi = fem.time_basis(k)
    # the (k+1)-point Radau rule is exact to degree 2k, so Mt is diagonal with the Radau weights
    assert np.abs(Mt - np.diag(np.diag(Mt))).max() < 1e-14 * tau
    np.testing.assert_allclose(Mt.sum(), tau, rtol=1e-14)  # sum of weights = slab length
    # D applied to the constant function: derivative vanishes, only the jump term chi_a(0) remains
    np.testing.assert_allclose(D.sum(axis=1), [c(0.0) for c in chi], atol=1e-13)
    # partition of unity in the third index of T
    np.testing.assert_allclose(T.sum(axis=2), Mt, atol=1e-14)
    if k == 2:
        s6 = math.sqrt(6.0)
        np.testing.assert_allclose(np.diag(Mt) / tau, [(16 - s6) / 36, (16 + s6) / 36, 1 / 9], atol=1e-14)
    # D + D^T = chi(1) chi(1)^T + chi(0) chi(0)^T (integration by parts of the time derivative)
    e1 = np.array([c(1.0) for c in chi])
    e0 = np.array([c(0.0) for c in chi])
    np.testing.assert_allclose(D + D.T, np.outer(e1, e1) + np.outer(e0, e0), atol=1e-13)


def test_q2_1d_mass_and_stiffness():
    # textbook 1D P2 element matrices on [0,1]
    M1 = np.array([[4, 2, -1], [2, 16, 2], [-1, 2, 4]]) / 30.0
    K1 = np.array([[7, -8, 1], [-8, 16, -8], [1, -8, 7]]) / 3.0
    lev = fem.Level(2, 0, (1, 1), (1.0, 1.0), (0, 0), (0, 0))
    sm = fem.spatial_matrices(lev, 1.0, 35.0, 35.0)
    # local node i = ix + 3 iy  ->  tensor products in (y, x) order
    np.testing.assert_allclose(sm["M"], np.kron(M1, M1), atol=1e-14)
    np.testing.assert_allclose(sm["K"], np.kron(K1, M1) + np.kron(M1, K1), atol=1e-13)
    lev3 = fem.Level(3, 0, (1, 1, 1), (1.0, 1.0, 1.0), (0, 0, 0), (0, 0, 0))
    sm3 = fem.spatial_matrices(lev3, 1.0, 35.0, 35.0)
    np.testing.assert_allclose(sm3["M"], np.kron(M1, np.kron(M1, M1)), atol=1e-14)


def test_scaled_cell_matrices():
    # affine scaling: mass ~ hx hy, stiffness ~ hy/hx d_x^2 + hx/hy d_y^2
    M1 = np.array([[4, 2, -1], [2, 16, 2], [-1, 2, 4]]) / 30.0
    K1 = np.array([[7, -8, 1], [-8, 16, -8], [1, -8, 7]]) / 3.0
    hx, hy = 0.1375, 0.1025
    lev = fem.Level(2, 0, (1, 1), (hx, hy), (0, 0), (0, 0))
    sm = fem.spatial_matrices(lev, 1.0, 35.0, 35.0)
    np.testing.assert_allclose(sm["M"], hx * hy * np.kron(M1, M1), atol=1e-15)
    np.testing.assert_allclose(sm["K"], hy / hx * np.kron(M1, K1) + hx / hy * np.kron(K1, M1), atol=1e-13)


@pytest.mark.parametrize("dim", [2, 3])
def test_legendre_pressure_mass_is_scaled_identity(dim):
    # Remark 4.1: the P1 Legendre basis is L2-orthonormal on the reference cell
    X, W = fem.volume_rule(dim)
    xi = fem.p1_basis(X)
    np.testing.assert_allclose(np.einsum("q,qa,qb->ab", W, xi, xi), np.eye(dim + 1), atol=1e-14)


def test_gauss_rule_exactness():
    x, w = fem.gauss_01(4)
    for p in range(8):
        np.testing.assert_allclose((w * x**p).sum(), 1.0 / (p + 1), rtol=1e-14)


def test_local_block_sizes_match_paper():
    g = json.load(open(GOLDEN))
    # Sec. 4.3: 3D Q2/P1disc cell block is 85 for dG(0) and 170 for dG(1)  (n_p = 4 in 3D)
    for key, k in (("cell_inverse_3d_dg0", 0), ("cell_inverse_3d_dg1", 1)):
        lev = fem.Level(3, k, (1, 1, 1), (1.0, 1.0, 1.0), (0, 0, 0), (0, 0, 0))
        assert lev.n == g[key]["n"]
        assert lev.n * lev.n * 8 == g[key]["bytes_fp64"]
    assert fem.Level(2, 1, (1, 1), (1.0, 1.0), (0, 0), (0, 0)).n == 42
    assert fem.Level(2, 2, (1, 1), (1.0, 1.0), (0, 0), (0, 0)).n == 63
