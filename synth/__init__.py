"""Seeded synthetic inputs for the channel-flow time-slab solves.

This module holds workload definitions and random-number draws only; it contains none of the
discretisation or solver arithmetic. Both the CPU oracle and the GPU path read their inputs from
here, each mapping the lattice arrays below onto its own degree-of-freedom numbering.

Lattice state layout (one dG(k) time slab, finest level of a workload):
  * the Q2 node lattice of the full box (obstacle included) has (2*nx+1) x (2*ny+1) [x (2*nz+1)]
    points, numbered lexicographically with x fastest: lat = ix + (2nx+1)*(iy + (2ny+1)*iz);
  * the full cell grid has nx*ny[*nz] cells, numbered the same way;
  * a state is a float64 array of shape [k+1, d*P + n_p*Cf] (P lattice points, Cf cells):
    per time node l, d velocity blocks of P values (component-major), then n_p pressure
    coefficients per cell (cell-major).
Entries that belong to removed obstacle nodes or cells are present in the lattice state and are
simply not referenced by either side.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Workload:
    """A seeded channel workload: geometry, discretisation degrees and solver settings."""

    name: str
    dim: int
    k: int
    n_levels: int
    coarse_cells: tuple
    length: tuple
    obstacle_lo: tuple  # half-open range of level-1 cells removed (lo == hi: no obstacle)
    obstacle_hi: tuple
    seed: int
    tau: float = 0.01
    nu: float = 1e-3
    gamma1: float = 35.0
    gamma2: float = 35.0
    omega: float = 0.7
    nu1: int = 2
    nu2: int = 2
    restart: int = 30
    rtol: float = 1e-10
    inflow_u: float = 0.3
    extra: dict = field(default_factory=dict)

    @property
    def fine_cells(self):
        f = 2 ** (self.n_levels - 1)
        return tuple(c * f for c in self.coarse_cells)

    def cells_at(self, level):
        """Cell counts per axis on level 1..n_levels."""
        f = 2 ** (level - 1)
        return tuple(c * f for c in self.coarse_cells)


_H = 0.41

WORKLOADS = {
    # 2D channel, 2 levels (16x4 -> 32x8), dG(1), no obstacle.
    "c1_2d_k1": Workload("c1_2d_k1", 2, 1, 2, (16, 4), (2.2, _H), (0, 0), (0, 0), seed=101),
    # 2D channel with a square obstacle, 5 levels (fine 256x64 minus 16x16), dG(2).
    "c2_2d_k2": Workload("c2_2d_k2", 2, 2, 5, (16, 4), (2.2, _H), (1, 1), (2, 2), seed=102),
    # 3D channel with a square prism obstacle, 3 levels (fine 64x16x16), dG(1).
    "c3_3d_k1": Workload("c3_3d_k1", 3, 1, 3, (16, 4, 4), (2.5, _H, _H), (1, 1, 0), (2, 2, 4),
                         seed=103, rtol=1e-8),
    # 2D adjoint/gradient case, 4 levels (fine 128x32 minus obstacle), dG(1).
    "c4_2d_k1": Workload("c4_2d_k1", 2, 1, 4, (16, 4), (2.2, _H), (1, 1), (2, 2), seed=104),
    # 3D multi-RHS case, 4 levels (fine 128x32x32 minus obstacle), dG(1), 32 right-hand sides.
    "c5_3d_k1": Workload("c5_3d_k1", 3, 1, 4, (16, 4, 4), (2.5, _H, _H), (1, 1, 0), (2, 2, 4),
                         seed=105, rtol=1e-8, extra={"nrhs": 32}),
}


def small_workload(dim, k, coarse_cells, n_levels, obstacle=False, seed=7, **kw):
    """Reduced channel used by the parity tests (same geometry rules, fewer cells)."""
    length = (2.2, _H) if dim == 2 else (2.5, _H, _H)
    if obstacle:
        lo = (1, 1) if dim == 2 else (1, 1, 0)
        hi = (2, 2) if dim == 2 else (2, 2, coarse_cells[2])
    else:
        lo = hi = (0,) * dim
    name = f"small_{dim}d_k{k}_{'x'.join(map(str, coarse_cells))}_L{n_levels}" + ("_obs" if obstacle else "")
    return Workload(name, dim, k, n_levels, tuple(coarse_cells), length, lo, hi, seed=seed, **kw)


def n_pressure(dim):
    """Pressure coefficients per cell of the discontinuous P1 space (3 in 2D, 4 in 3D)."""
    return dim + 1


def lattice_shape(cells):
    return tuple(2 * c + 1 for c in cells)


def state_width(dim, cells):
    P = int(np.prod(lattice_shape(cells)))
    Cf = int(np.prod(cells))
    return dim * P + n_pressure(dim) * Cf


def _lattice_coords(cells, length):
    """Coordinates of the lattice points, each of shape lattice (z, y, x) order flattened x-fastest."""
    axes = [np.linspace(0.0, L, 2 * c + 1) for c, L in zip(cells, length)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")  # (z,) y, x
    return [g.ravel() for g in grids[::-1]]  # x, y, (z) each flattened with x fastest


def linearisation_point(wl: Workload, U: float | None = None, amp: float = 0.1, n_modes: int = 8):
    """Newton linearisation point w on the finest lattice, shape [k+1, state_width].

    Poiseuille inflow profile of amplitude U plus `amp` times a normalised sum of `n_modes`
    divergence-free Fourier modes with N(0,1) amplitudes drawn independently per time node.
    Pressure entries are zero.
    """
    U = wl.inflow_u if U is None else U
    rng = np.random.default_rng(wl.seed)
    cells = wl.fine_cells
    d = wl.dim
    L = wl.length
    xs = _lattice_coords(cells, L)
    P = xs[0].size
    H = L[1]
    base = np.zeros((d, P))
    if d == 2:
        y = xs[1]
        base[0] = 4.0 * U * y * (H - y) / H**2
    else:
        y, z = xs[1], xs[2]
        base[0] = 16.0 * U * y * (H - y) * z * (L[2] - z) / (H**2 * L[2] ** 2)
    p_m = rng.integers(1, 9, size=n_modes)
    q_m = rng.integers(1, 5, size=n_modes)
    s_m = rng.integers(1, 5, size=n_modes)
    out = np.zeros((wl.k + 1, state_width(d, cells)))
    modes = np.zeros((wl.k + 1, d, P))
    for l in range(wl.k + 1):
        a = rng.standard_normal(n_modes)
        b = rng.standard_normal(n_modes)
        for m in range(n_modes):
            ax = math.pi * p_m[m] / L[0]
            ay = math.pi * q_m[m] / L[1]
            sx, cx = np.sin(ax * xs[0]), np.cos(ax * xs[0])
            sy, cy = np.sin(ay * xs[1]), np.cos(ay * xs[1])
            if d == 2:
                # stream function a sin(ax x) sin(ay y); v = (d/dy, -d/dx)
                modes[l, 0] += a[m] * sx * ay * cy
                modes[l, 1] += -a[m] * ax * cx * sy
            else:
                az = math.pi * s_m[m] / L[2]
                sz, cz = np.sin(az * xs[2]), np.cos(az * xs[2])
                # curl(psi e_z) + curl(phi e_y), psi = a sx sy sz, phi = b sx sy sz
                modes[l, 0] += a[m] * sx * ay * cy * sz - b[m] * sx * sy * az * cz
                modes[l, 1] += -a[m] * ax * cx * sy * sz
                modes[l, 2] += b[m] * ax * cx * sy * sz
    scale = amp / max(np.abs(modes).max(), 1e-300)
    for l in range(wl.k + 1):
        out[l, : d * P] = (base + scale * modes[l]).ravel()
    return out


def random_rhs(wl: Workload, seed_offset: int = 0, nrhs: int | None = None):
    """Seeded N(0,1) right-hand side(s) on the finest lattice: [k+1, state_width] or [nrhs, ...]."""
    rng = np.random.default_rng(wl.seed + 1000 + seed_offset)
    shape = (wl.k + 1, state_width(wl.dim, wl.fine_cells))
    if nrhs is None:
        return rng.standard_normal(shape)
    return rng.standard_normal((nrhs,) + shape)


def inflow_sweep(nrhs: int = 32, lo: float = 0.2, hi: float = 0.45):
    """Inflow amplitudes of the multi-right-hand-side workload."""
    return np.linspace(lo, hi, nrhs)
