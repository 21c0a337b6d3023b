"""Shared builders for the parity tests: the same seeded workload on the oracle and on libstm."""
import numpy as np

import synth


def oracle_hierarchy(wl, variant="additive", nu=None):
    from oracle import solvers
    return solvers.Hierarchy(wl, synth.linearisation_point(wl), nu=nu, variant=variant)


def oracle_lattice_index(lev):
    """Lattice-state index of every oracle DoF of `lev` (the documented numbering)."""
    d, K = lev.dim, lev.k + 1
    P = lev.P
    W = d * P + lev.np_ * int(np.prod(lev.cells))
    out = []
    for l in range(K):
        for i in range(d):
            out.append(l * W + i * P + lev.lat_of_node)
        out.append(l * W + d * P + (lev.active_full[:, None] * lev.np_ + np.arange(lev.np_)).ravel())
    return np.concatenate(out)


def gpu_params(wl, prec="f64", smoother="additive", **kw):
    from paper_2107_10561_gb300 import make_params
    args = dict(tau=wl.tau, nu=wl.nu, gamma1=wl.gamma1, gamma2=wl.gamma2, inv_precision=prec,
                smoother=smoother, omega=wl.omega, nu1=wl.nu1, nu2=wl.nu2)
    args.update(kw)
    return make_params(wl.dim, wl.k, wl.n_levels, wl.coarse_cells, wl.length, wl.obstacle_lo, wl.obstacle_hi, **args)


def gpu_hierarchy(wl, prec="f64", smoother="additive", factor=True, **kw):
    import torch
    from paper_2107_10561_gb300 import Hierarchy
    h = Hierarchy(gpu_params(wl, prec, smoother, **kw))
    X = lattice_to_gpu(h, synth.linearisation_point(wl))
    h.assemble_jacobian(X)
    if factor:
        h.factor_cells()
    torch.cuda.synchronize()
    return h


def lattice_to_gpu(h, state, level=None):
    import torch
    idx = h.dof_lattice_index(level)
    return torch.from_numpy(np.ascontiguousarray(state.reshape(-1)[idx])).cuda()


def round_bf16(a):
    """FP64 -> the nearest BF16 value (8 significant bits, ties to even), returned in FP64: one
    rounding straight from FP64. Normal BF16 range only (no BF16 subnormals)."""
    a = np.asarray(a, dtype=np.float64)
    m, e = np.frexp(a)  # a = m 2^e, 0.5 <= |m| < 1; m * 256 is exact and np.rint rounds ties to even
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def round_storage(inv, prec):
    """Cell inverses rounded to their storage precision (FP64 values)."""
    if prec == "f32":
        return inv.astype(np.float32).astype(np.float64)
    if prec == "bf16":
        return round_bf16(inv)
    return inv


def rel_max(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def poiseuille_state(lev, U, nu):
    """Exact steady channel flow on an oracle level (2D): velocity U g_1 e_x at every time node,
    g_1 = 4y(H-y)/H^2 (3D: times 4z(L2-z)/L2^2); pressure (8 nu U / H^2)(L - x) (zero at the do-nothing outflow) as Legendre P1
    coefficients per cell: mean at the centre, x-slope coefficient -(8 nu U / H^2) h_x / (2 sqrt 3)."""
    H, L = lev.length[1], lev.length[0]
    lat = np.stack(np.unravel_index(lev.lat_of_node, lev.lshape[::-1])[::-1], axis=1)
    y = lat[:, 1] * (lev.h[1] / 2.0)
    g = 4.0 * y * (H - y) / H**2
    if lev.dim == 3:  # the inflow profile's z factor (the state is then not a steady solution)
        L2 = lev.length[2]
        z = lat[:, 2] * (lev.h[2] / 2.0)
        g = g * 4.0 * z * (L2 - z) / L2**2
    G = 8.0 * nu * U / H**2
    X = np.zeros(lev.N)
    for a in range(lev.k + 1):
        X[a * lev.block: a * lev.block + lev.R] = U * g
        xc = (lev.cell_xyz[:, 0] + 0.5) * lev.h[0]
        base = a * lev.block + lev.dim * lev.R + np.arange(lev.C) * lev.np_
        X[base] = G * (L - xc)
        X[base + 1] = -G * lev.h[0] / (2.0 * np.sqrt(3.0))
    return X
