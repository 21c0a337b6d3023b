"""Oracle, part 1: discretisation of one dG(k) time slab (TEST INFRASTRUCTURE ONLY).

Spaces (Sec. 2.3, Eq. Def:Vh0): continuous Q2 velocity with equidistant nodes {0, 1/2, 1}^d per
cell; discontinuous P1 pressure with the Legendre basis that is L2-orthonormal on the reference
cell (Remark 4.1): xi_0 = 1, xi_{1+m} = sqrt(3) (2 x_m - 1).  Cells are axis-aligned boxes of a
uniform grid with an optional block of removed cells (the obstacle), so every map is affine.

Time (Sec. 2.4, Eq. time_discrete_ansatz): Lagrange basis at the k+1 right Gauss-Radau points of
the slab; all time integrals are evaluated exactly.

Algebraic layout (Eq. totdofs): per time node l, the d velocity component vectors (R entries each,
Q2 nodes numbered lexicographically with x fastest over the full lattice, unused obstacle nodes
compressed out), then the pressure vector (cell-major: active cell id, then Legendre mode).
Cell-local layout (Eq. locdofs): per time node l, the d velocity components over the 3^d cell
nodes (lexicographic, x fastest), then the n_p pressure modes.
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np
import scipy.sparse as sp

SQRT3 = math.sqrt(3.0)


# ----------------------------------------------------------------------------------------------
# 1D building blocks
# ----------------------------------------------------------------------------------------------
def q2_1d(x):
    """The three quadratic Lagrange polynomials on [0,1] with nodes 0, 1/2, 1; shape [3, ...]."""
    x = np.asarray(x, dtype=float)
    return np.stack([2.0 * (x - 0.5) * (x - 1.0), -4.0 * x * (x - 1.0), 2.0 * x * (x - 0.5)])


def dq2_1d(x):
    """Derivatives of q2_1d; shape [3, ...]."""
    x = np.asarray(x, dtype=float)
    return np.stack([4.0 * x - 3.0, -8.0 * x + 4.0, 4.0 * x - 1.0])


def gauss_01(npts):
    """Gauss-Legendre rule on [0,1]."""
    x, w = np.polynomial.legendre.leggauss(npts)
    return 0.5 * (x + 1.0), 0.5 * w


def local_node_offsets(dim):
    """Offsets (in half-cells) of the 3^d Q2 nodes of a cell, lexicographic with x fastest."""
    return np.array([[(i // 3**m) % 3 for m in range(dim)] for i in range(3**dim)], dtype=np.int64)


def n_pressure(dim):
    """dim P1 = d + 1 pressure modes per cell (3 in 2D, 4 in 3D)."""
    return dim + 1


def q2_basis(X):
    """Tensor Q2 basis at reference points X [np, d]: values [np, 3^d], gradients [np, 3^d, d]."""
    X = np.atleast_2d(X)
    npnt, dim = X.shape
    loc = local_node_offsets(dim)
    v1 = [q2_1d(X[:, m]) for m in range(dim)]  # each [3, np]
    d1 = [dq2_1d(X[:, m]) for m in range(dim)]
    phi = np.ones((npnt, 3**dim))
    dphi = np.ones((npnt, 3**dim, dim))
    for i in range(3**dim):
        for m in range(dim):
            phi[:, i] *= v1[m][loc[i, m]]
            for mm in range(dim):
                dphi[:, i, mm] *= (d1[m] if m == mm else v1[m])[loc[i, m]]
    return phi, dphi


def p1_basis(X):
    """Legendre P1 basis on the reference cell at points X [np, d]; shape [np, d+1]."""
    X = np.atleast_2d(X)
    return np.concatenate([np.ones((X.shape[0], 1)), SQRT3 * (2.0 * X - 1.0)], axis=1)


def volume_rule(dim, npts=4):
    """Tensor Gauss rule with npts^d points on [0,1]^d: points [nq, d], weights [nq]."""
    x, w = gauss_01(npts)
    grids = np.meshgrid(*([x] * dim), indexing="ij")
    wgrids = np.meshgrid(*([w] * dim), indexing="ij")
    X = np.stack([g.ravel() for g in grids[::-1]], axis=1)  # x fastest
    W = np.prod(np.stack([g.ravel() for g in wgrids]), axis=0)
    return X, W


def face_rule(dim, axis, side, npts=4):
    """Gauss rule on the face {x_axis = side} of [0,1]^d: points [nq, d], weights [nq]."""
    if dim == 1:
        return np.array([[float(side)]]), np.array([1.0])
    Xf, Wf = volume_rule(dim - 1, npts)
    X = np.zeros((Xf.shape[0], dim))
    others = [m for m in range(dim) if m != axis]
    for j, m in enumerate(others):
        X[:, m] = Xf[:, j]
    X[:, axis] = float(side)
    return X, Wf


# ----------------------------------------------------------------------------------------------
# Time basis and temporal matrices (Sec. 2.4, Problem 3.1, Eq. time_discrete_ansatz)
# ----------------------------------------------------------------------------------------------
def radau_right_nodes(k):
    """The k+1 right Gauss-Radau points of [0,1] (the end point 1 is a node), ascending.

    They are the roots of P_k - P_{k+1} (Legendre polynomials on [-1,1]) mapped to [0,1].
    """
    from numpy.polynomial import legendre as L

    c = np.zeros(k + 2)
    c[k] = 1.0
    c[k + 1] = -1.0
    r = np.sort(np.real(L.legroots(c)))
    r[-1] = 1.0
    return 0.5 * (r + 1.0)


def lagrange_time(k, s):
    """Values chi_a(s) and derivatives chi_a'(s) of the Radau-Lagrange basis: two arrays [k+1, len(s)].

    Product form chi_a(s) = prod_{b != a} (s - s_b) / (s_a - s_b); the derivative is the sum over
    the omitted factor.
    """
    nodes = radau_right_nodes(k)
    s = np.atleast_1d(np.asarray(s, dtype=float))
    K = k + 1
    val = np.ones((K, s.size))
    der = np.zeros((K, s.size))
    for a in range(K):
        for b in range(K):
            if b == a:
                continue
            val[a] *= (s - nodes[b]) / (nodes[a] - nodes[b])
            term = np.ones(s.size) / (nodes[a] - nodes[b])
            for c in range(K):
                if c != a and c != b:
                    term *= (s - nodes[c]) / (nodes[a] - nodes[c])
            der[a] += term
    return val, der


def time_basis(k):
    """chi_0..chi_k on [0,1] as callables (Lagrange polynomials through the right Radau nodes)."""
    return [(lambda s, a=a: float(lagrange_time(k, s)[0][a][0]) if np.ndim(s) == 0
             else lagrange_time(k, s)[0][a]) for a in range(k + 1)]


def time_matrices(k, tau):
    """Exact temporal matrices of one slab of length tau (test index a = row, trial b = column).

    Mt[a,b]   = tau * int_0^1 chi_a chi_b            (mass in time)
    D[a,b]    = int_0^1 chi_b' chi_a + chi_b(0) chi_a(0)
                (time derivative plus the upwind jump <v(t_{n-1}^+), psi(t_{n-1}^+)>, Problem 3.1)
    T[a,b,c]  = tau * int_0^1 chi_a chi_b chi_c      (convection term in time)
    All integrands are polynomials of degree <= 3k, integrated exactly by (k+3)-point Gauss.
    """
    s, w = gauss_01(k + 3)
    val, der = lagrange_time(k, s)
    v0, _ = lagrange_time(k, np.array([0.0]))
    Mt = tau * np.einsum("q,aq,bq->ab", w, val, val)
    D = np.einsum("q,bq,aq->ab", w, der, val) + np.outer(v0[:, 0], v0[:, 0])
    T = tau * np.einsum("q,aq,bq,cq->abc", w, val, val, val)
    return Mt, D, T


# ----------------------------------------------------------------------------------------------
# Mesh level, numbering and boundary classification
# ----------------------------------------------------------------------------------------------
class Level:
    """One uniform level of the channel mesh with the obstacle cells removed.

    cells: cell counts per axis; length: box size; removed_lo/hi: half-open block of removed
    cells in this level's cell units (lo == hi: nothing removed).
    Boundary classification (Sec. 2.1): x = 0 is the inflow part of Gamma_D, x = L the do-nothing
    outflow Gamma_o, every other box face (walls) and every face shared with a removed cell
    (obstacle surface) belongs to Gamma_D.
    """

    def __init__(self, dim, k, cells, length, removed_lo, removed_hi):
        self.dim, self.k = dim, k
        self.cells = tuple(int(c) for c in cells)
        self.length = tuple(float(x) for x in length)
        self.h = np.array(self.length) / np.array(self.cells)
        self.removed_lo = tuple(removed_lo)
        self.removed_hi = tuple(removed_hi)
        d = dim
        Cf = int(np.prod(self.cells))
        full_xyz = np.stack(np.unravel_index(np.arange(Cf), self.cells[::-1])[::-1], axis=1)
        self.full_xyz = full_xyz
        removed = np.ones(Cf, dtype=bool)
        for m in range(d):
            removed &= (full_xyz[:, m] >= removed_lo[m]) & (full_xyz[:, m] < removed_hi[m])
        self.full_removed = removed
        self.active_full = np.nonzero(~removed)[0]
        self.C = self.active_full.size
        self.cell_xyz = full_xyz[self.active_full]
        # Q2 node lattice
        self.lshape = tuple(2 * c + 1 for c in self.cells)
        self.P = int(np.prod(self.lshape))
        strides = [1]
        for m in range(1, d):
            strides.append(strides[-1] * self.lshape[m - 1])
        self.lstrides = np.array(strides, dtype=np.int64)
        loc = local_node_offsets(d)
        lat_coords = 2 * self.cell_xyz[:, None, :] + loc[None, :, :]
        lat = (lat_coords * self.lstrides).sum(-1)
        used = np.zeros(self.P, dtype=bool)
        used[lat.ravel()] = True
        self.lat_of_node = np.nonzero(used)[0]
        node_of_lat = -np.ones(self.P, dtype=np.int64)
        node_of_lat[self.lat_of_node] = np.arange(self.lat_of_node.size)
        self.node_of_lat = node_of_lat
        self.cell_nodes = node_of_lat[lat]
        self.R = self.lat_of_node.size
        self.np_ = n_pressure(d)
        self.S = self.np_ * self.C
        self.block = d * self.R + self.S
        self.N = (k + 1) * self.block
        self.nloc_v = d * 3**d
        self.nloc_t = self.nloc_v + self.np_
        self.n = (k + 1) * self.nloc_t
        # local -> global DoF map (Eq. locdofs -> Eq. totdofs)
        idx = np.zeros((self.C, self.n), dtype=np.int64)
        for l in range(k + 1):
            for i in range(d):
                o = l * self.nloc_t + i * 3**d
                idx[:, o:o + 3**d] = l * self.block + i * self.R + self.cell_nodes
            o = l * self.nloc_t + self.nloc_v
            for q in range(self.np_):
                idx[:, o + q] = l * self.block + d * self.R + np.arange(self.C) * self.np_ + q
        self.idx = idx
        # Dirichlet faces (face f = 2*axis + side)
        dirich = np.zeros((self.C, 2 * d), dtype=bool)
        for m in range(d):
            for s in (0, 1):
                nb = self.cell_xyz.copy()
                nb[:, m] += 1 if s else -1
                outside = (nb[:, m] < 0) | (nb[:, m] >= self.cells[m])
                if m == 0:
                    on_gd = outside & (s == 0)  # inflow x = 0; x = L is the outflow
                else:
                    on_gd = outside.copy()  # walls
                inside = ~outside
                nb_full = np.zeros(self.C, dtype=np.int64)
                st = 1
                for mm in range(d):
                    nb_full += np.clip(nb[:, mm], 0, self.cells[mm] - 1) * st
                    st *= self.cells[mm]
                on_gd |= inside & removed[nb_full]  # obstacle surface
                dirich[:, 2 * m + s] = on_gd
        self.dirichlet = dirich
        self.outflow = np.zeros((self.C, 2 * d), dtype=bool)
        self.outflow[:, 1] = self.cell_xyz[:, 0] == self.cells[0] - 1
        self.colour = np.zeros(self.C, dtype=np.int64)
        for m in range(d):
            self.colour += (self.cell_xyz[:, m] % 2) << m

    def cell_origin(self):
        return self.cell_xyz * self.h

    # -- lattice state <-> DoF vector --------------------------------------------------------
    def dofs_from_lattice(self, state):
        """Global DoF vector from a lattice state [k+1, d*P + n_p*Cf] given on THIS level."""
        d, K = self.dim, self.k + 1
        out = np.zeros(self.N)
        for l in range(K):
            for i in range(d):
                out[l * self.block + i * self.R: l * self.block + (i + 1) * self.R] = \
                    state[l, i * self.P + self.lat_of_node]
            pcol = d * self.P + (self.active_full[:, None] * self.np_ + np.arange(self.np_)).ravel()
            out[l * self.block + d * self.R:(l + 1) * self.block] = state[l, pcol]
        return out

    def velocity_nodal(self, X):
        """Velocity nodal values of a DoF vector: [k+1, d, R]."""
        K = self.k + 1
        return np.stack([X[l * self.block: l * self.block + self.dim * self.R]
                         .reshape(self.dim, self.R) for l in range(K)])


def fine_lattice_to_level(state_fine, fine_cells, level: Level):
    """Inject a lattice state of the finest level onto `level` (coarse nodes are fine nodes).

    Velocity lattice points are taken at stride 2^(G-g); pressure entries are set to zero
    (the linearisation point only enters through its velocity, Sec. 3 Eq. linNewEq).
    """
    d = level.dim
    f = fine_cells[0] // level.cells[0]
    fshape = tuple(2 * c + 1 for c in fine_cells)
    K = state_fine.shape[0]
    Pf = int(np.prod(fshape))
    out = np.zeros((K, d * level.P + level.np_ * int(np.prod(level.cells))))
    for l in range(K):
        for i in range(d):
            arr = state_fine[l, i * Pf:(i + 1) * Pf].reshape(fshape[::-1])
            sl = tuple(slice(None, None, f) for _ in range(d))
            out[l, i * level.P:(i + 1) * level.P] = arr[sl].ravel()
    return out


# ----------------------------------------------------------------------------------------------
# Element matrices (Sec. 2.3 Eqs. Def:Ah, Def:B_GamD; Sec. 3 Eqs. linNewEq, definition_jacobian_global)
# ----------------------------------------------------------------------------------------------
class RefTables:
    """Basis values on the 4^d volume rule and on the 4^(d-1) rule of every face."""

    def __init__(self, dim):
        self.dim = dim
        self.Xq, self.Wq = volume_rule(dim)
        self.phi, self.dphi = q2_basis(self.Xq)
        self.xi = p1_basis(self.Xq)
        self.faces = []
        for m in range(dim):
            for s in (0, 1):
                X, W = face_rule(dim, m, s)
                phi, dphi = q2_basis(X)
                self.faces.append(dict(axis=m, side=s, normal=(2.0 * s - 1.0), X=X, W=W,
                                       phi=phi, dphi=dphi, xi=p1_basis(X)))


@lru_cache(maxsize=None)
def ref_tables(dim):
    return RefTables(dim)


def spatial_matrices(level: Level, nu, gamma1, gamma2):
    """Cell-geometry matrices of a uniform level (identical for all cells of the level).

    M[i,j]      = (phi_j, phi_i)_T                          velocity mass
    K[i,j]      = (grad phi_j, grad phi_i)_T                velocity stiffness
    Div[m][q,j] = (d_m phi_j, xi_q)_T                       divergence coupling
    per face f with outer normal n = +-e_axis:
      S[f][i,j] = <phi_j, phi_i>_f,  G[f][i,j] = <grad phi_j . n, phi_i>_f,  Pf[f][q,i] = <phi_i, xi_q>_f
    """
    rt = ref_tables(level.dim)
    d, h = level.dim, level.h
    vol = float(np.prod(h))
    gphys = rt.dphi / h[None, None, :]
    M = vol * np.einsum("q,qi,qj->ij", rt.Wq, rt.phi, rt.phi)
    K = vol * np.einsum("q,qim,qjm->ij", rt.Wq, gphys, gphys)
    Div = np.stack([vol * np.einsum("q,qa,qj->aj", rt.Wq, rt.xi, gphys[:, :, m]) for m in range(d)])
    faces = []
    for f in rt.faces:
        m = f["axis"]
        area = float(np.prod([h[mm] for mm in range(d) if mm != m]))
        gn = f["normal"] * f["dphi"][:, :, m] / h[m]
        faces.append(dict(
            axis=m, normal=f["normal"],
            S=area * np.einsum("q,qi,qj->ij", f["W"], f["phi"], f["phi"]),
            G=area * np.einsum("q,qi,qj->ij", f["W"], f["phi"], gn),
            Pf=area * np.einsum("q,qa,qi->ai", f["W"], f["xi"], f["phi"]),
        ))
    return dict(M=M, K=K, Div=Div, faces=faces, hT=float(np.sqrt((h**2).sum())))


def linear_blocks(level: Level, sm, nu, gamma1, gamma2, dirichlet_row):
    """Linear spatial blocks of one cell with Dirichlet-face mask `dirichlet_row` [2d].

    Velocity-velocity (test component l, trial m):
      A[l][m] = delta_lm (nu K - nu G - nu G^T + gamma1 nu/h S) + gamma2/h n_l n_m S, summed over
      the Gamma_D faces, from nu(grad v, grad psi), -<nu grad v . n, psi>, the Nitsche form B_GamD.
    Pressure column (test velocity (l,i), trial xi_q): Bc[l][i,q] = -(xi_q, d_l phi_i) + <xi_q n_l, phi_i>
    Pressure row (test xi_q, trial velocity (m,j)):   Br[m][q,j] = (d_m phi_j, xi_q) - <phi_j n_m, xi_q>
    """
    d = level.dim
    hT = sm["hT"]
    nv = 3**d
    A = np.zeros((d, d, nv, nv))
    Bc = np.zeros((d, nv, d + 1))
    Br = np.zeros((d, d + 1, nv))
    for l in range(d):
        A[l, l] += nu * sm["K"]
        Bc[l] -= sm["Div"][l].T
        Br[l] += sm["Div"][l]
    for f_id, f in enumerate(sm["faces"]):
        if not dirichlet_row[f_id]:
            continue
        m = f["axis"]
        n = f["normal"]
        for l in range(d):
            A[l, l] += -nu * f["G"] - nu * f["G"].T + gamma1 * nu / hT * f["S"]
        A[m, m] += gamma2 / hT * n * n * f["S"]
        Bc[m] += n * f["Pf"].T
        Br[m] -= n * f["Pf"]
    return A, Bc, Br


def convection_blocks(level: Level, wcell):
    """Newton linearisation of the convection term for a batch of cells (Sec. 3, Eq. linNewEq).

    wcell: [nc, d, 3^d] nodal velocity of the linearisation point on each cell.
    Returns N [nc, d, d, 3^d, 3^d] with
      N[l][m][i,j] = ((w . grad) phi_j delta_lm + phi_j d_m w_l, phi_i)_T,
    the derivative of <(v . grad) v, psi> at v = w in the direction phi_j e_m, tested with phi_i e_l.
    """
    rt = ref_tables(level.dim)
    d, h = level.dim, level.h
    vol = float(np.prod(h))
    gphys = rt.dphi / h[None, None, :]
    wq = np.einsum("qs,cls->cql", rt.phi, wcell)  # w at quad points
    gw = np.einsum("qsm,cls->cqlm", gphys, wcell)  # d_m w_l at quad points
    Wphi = vol * rt.Wq[:, None] * rt.phi  # [q, i]
    adv = np.einsum("cqm,qjm->cqj", wq, gphys)  # (w . grad) phi_j
    T1 = np.einsum("qi,cqj->cij", Wphi, adv)
    T2 = np.einsum("qi,qj,cqlm->clmij", Wphi, rt.phi, gw)
    N = T2.copy()
    for l in range(d):
        N[:, l, l] += T1
    return N


def element_matrices(level: Level, cells, X_lin, tau, nu, gamma1, gamma2):
    """Element Jacobians of the slab system for the given cells, [nc, n, n] in Eq. locdofs order.

    Block (a,b) in time (Problem 3.1 with the Newton linearisation of Eq. linNewEq):
      velocity-velocity  D_ab M delta_lm + Mt_ab A_lm + sum_c T_abc N(w^c)_lm
      velocity-pressure  Mt_ab Bc_l        pressure-velocity  Mt_ab Br_m      pressure-pressure 0
    X_lin is the linearisation point as a DoF vector of this level (only velocities are used).
    """
    d, k = level.dim, level.k
    K = k + 1
    nv = 3**d
    Mt, D, T = time_matrices(k, tau)
    sm = spatial_matrices(level, nu, gamma1, gamma2)
    wn = level.velocity_nodal(X_lin)  # [K, d, R]
    cells = np.asarray(cells)
    nc = cells.size
    Ncv = np.stack([convection_blocks(level, wn[c][:, level.cell_nodes[cells]].transpose(1, 0, 2))
                    for c in range(K)], axis=1)  # [nc, K, d, d, nv, nv]
    E = np.zeros((nc, level.n, level.n))
    # the linear blocks depend only on the Dirichlet-face mask: group cells by it
    masks = level.dirichlet[cells]
    keys = {}
    for ci in range(nc):
        keys.setdefault(tuple(masks[ci]), []).append(ci)
    for key, members in keys.items():
        A, Bc, Br = linear_blocks(level, sm, nu, gamma1, gamma2, np.array(key))
        mem = np.array(members)
        for a in range(K):
            for b in range(K):
                for l in range(d):
                    ra = a * level.nloc_t + l * nv
                    for m in range(d):
                        cb = b * level.nloc_t + m * nv
                        blk = Mt[a, b] * A[l, m] + np.einsum("c,xcij->xij", T[a, b], Ncv[mem][:, :, l, m])
                        if l == m:
                            blk = blk + D[a, b] * sm["M"]
                        E[mem, ra:ra + nv, cb:cb + nv] = blk
                    pb = b * level.nloc_t + level.nloc_v
                    E[mem, ra:ra + nv, pb:pb + d + 1] = Mt[a, b] * Bc[l]
                pa = a * level.nloc_t + level.nloc_v
                for m in range(d):
                    cb = b * level.nloc_t + m * nv
                    E[mem, pa:pa + d + 1, cb:cb + nv] = Mt[a, b] * Br[m]
    return E


def assemble_jacobian(level: Level, X_lin, tau, nu, gamma1=35.0, gamma2=35.0, chunk=512):
    """Global Jacobian J = sum_T R_T^T E_T R_T as a scipy CSR matrix (Sec. 3, Eq. linNewEq)."""
    N = level.N
    J = sp.csr_matrix((N, N))
    for s in range(0, level.C, chunk):
        cells = np.arange(s, min(level.C, s + chunk))
        E = element_matrices(level, cells, X_lin, tau, nu, gamma1, gamma2)
        rows = np.broadcast_to(level.idx[cells][:, :, None], E.shape)
        cols = np.broadcast_to(level.idx[cells][:, None, :], E.shape)
        J = J + sp.coo_matrix((E.ravel(), (rows.ravel(), cols.ravel())), shape=(N, N)).tocsr()
    J.eliminate_zeros()
    J.sort_indices()
    return J


def convection_residual(level: Level, X, tau):
    """Nonlinear convection term int_{I_n} <(v . grad) v, psi> dt tested with every velocity DoF.

    Evaluated directly from v = sum_b v^b chi_b (quadratic in X); used to pin the Newton
    linearisation (central differences of a quadratic are exact).
    """
    d, k = level.dim, level.k
    K = k + 1
    rt = ref_tables(d)
    h = level.h
    vol = float(np.prod(h))
    gphys = rt.dphi / h[None, None, :]
    _, _, T = time_matrices(k, tau)
    vn = level.velocity_nodal(X)
    out = np.zeros(level.N)
    vc = vn[:, :, level.cell_nodes]  # [K, d, C, nv]
    vq = np.einsum("qs,bdcs->bcqd", rt.phi, vc)
    gq = np.einsum("qsm,bdcs->bcqdm", gphys, vc)
    for a in range(K):
        for l in range(d):
            acc = np.zeros((level.C, 3**d))
            for b in range(K):
                for c in range(K):
                    # (v^c . grad) v^b_l at quad points, tested with phi_i
                    adv = np.einsum("cqm,cqm->cq", vq[c], gq[b][:, :, l, :])
                    acc += T[a, b, c] * vol * np.einsum("q,qi,cq->ci", rt.Wq, rt.phi, adv)
            rows = a * level.block + l * level.R + level.cell_nodes
            np.add.at(out, rows.ravel(), acc.ravel())
    return out


# ----------------------------------------------------------------------------------------------
# Right-hand side (Problem 3.1 right-hand side with Eq. Def:Lh), used by the manufactured-solution
# pins and by the adjoint workload
# ----------------------------------------------------------------------------------------------
def assemble_load(level: Level, tau, nu, gamma1=35.0, gamma2=35.0, f=None, g=None, traction=None,
                  v_prev=None, nt=None):
    """b = int_{I_n} L_h(psi; f, g) dt + <v_prev, psi(t_{n-1}^+)> (+ <traction, psi>_{Gamma_o}).

    f(x, t), g(x, t), traction(x, t) return arrays [npts, d]; x is [npts, d] and t the time
    relative to the slab start (0 <= t <= tau). v_prev(x) returns [npts, d].
    L_h = (f, psi) + B_GamD(g, (psi, xi)) with
    B_GamD(g, (psi, xi)) = -<g, nu grad psi . n + xi n> + gamma1 nu <h^-1 g, psi> + gamma2 <h^-1 g.n, psi.n>.
    """
    d, k = level.dim, level.k
    K = k + 1
    rt = ref_tables(d)
    h = level.h
    vol = float(np.prod(h))
    hT = float(np.sqrt((h**2).sum()))
    nv = 3**d
    chi = time_basis(k)
    st, sw = gauss_01(k + 3 if nt is None else nt)
    x0 = level.cell_origin()  # [C, d]
    bl = np.zeros((level.C, level.n))
    gphys = rt.dphi / h[None, None, :]
    for a in range(K):
        for ts, tw in zip(st, sw):
            t = tau * ts
            wt = tau * tw * chi[a](ts)
            if f is not None:
                xq = x0[:, None, :] + rt.Xq[None, :, :] * h
                fv = f(xq.reshape(-1, d), t).reshape(level.C, -1, d)
                for l in range(d):
                    bl[:, a * level.nloc_t + l * nv: a * level.nloc_t + (l + 1) * nv] += \
                        wt * vol * np.einsum("q,qi,cq->ci", rt.Wq, rt.phi, fv[:, :, l])
            for f_id, fc in enumerate(rt.faces):
                m, n = fc["axis"], fc["normal"]
                area = float(np.prod([h[mm] for mm in range(d) if mm != m]))
                gn = n * fc["dphi"][:, :, m] / h[m]
                xq = x0[:, None, :] + fc["X"][None, :, :] * h
                mask_d = level.dirichlet[:, f_id]
                if g is not None and mask_d.any():
                    cs = np.nonzero(mask_d)[0]
                    gv = g(xq[cs].reshape(-1, d), t).reshape(cs.size, -1, d)
                    for l in range(d):
                        ro = a * level.nloc_t + l * nv
                        val = (-nu * np.einsum("q,qi,cq->ci", fc["W"], gn, gv[:, :, l])
                               + gamma1 * nu / hT * np.einsum("q,qi,cq->ci", fc["W"], fc["phi"], gv[:, :, l]))
                        if l == m:
                            val += gamma2 / hT * np.einsum("q,qi,cq->ci", fc["W"], fc["phi"], gv[:, :, m])
                        bl[cs, ro:ro + nv] += wt * area * val
                    po = a * level.nloc_t + level.nloc_v
                    bl[cs, po:po + d + 1] += wt * area * (-n) * np.einsum("q,qa,cq->ca", fc["W"], fc["xi"], gv[:, :, m])
                mask_o = level.outflow[:, f_id]
                if traction is not None and mask_o.any():
                    cs = np.nonzero(mask_o)[0]
                    tv = traction(xq[cs].reshape(-1, d), t).reshape(cs.size, -1, d)
                    for l in range(d):
                        ro = a * level.nloc_t + l * nv
                        bl[cs, ro:ro + nv] += wt * area * np.einsum("q,qi,cq->ci", fc["W"], fc["phi"], tv[:, :, l])
        if v_prev is not None:
            xq = x0[:, None, :] + rt.Xq[None, :, :] * h
            pv = v_prev(xq.reshape(-1, d)).reshape(level.C, -1, d)
            for l in range(d):
                bl[:, a * level.nloc_t + l * nv: a * level.nloc_t + (l + 1) * nv] += \
                    chi[a](0.0) * vol * np.einsum("q,qi,cq->ci", rt.Wq, rt.phi, pv[:, :, l])
    b = np.zeros(level.N)
    np.add.at(b, level.idx.ravel(), bl.ravel())
    return b


def l2_errors(level: Level, X, v_exact, p_exact, t_nodes):
    """L2(Omega) errors of velocity and pressure at each time node: arrays [k+1]."""
    d, K = level.dim, level.k + 1
    rt = ref_tables(d)
    vol = float(np.prod(level.h))
    x0 = level.cell_origin()
    xq = (x0[:, None, :] + rt.Xq[None, :, :] * level.h).reshape(-1, d)
    ev, ep = np.zeros(K), np.zeros(K)
    for l in range(K):
        vn = X[l * level.block: l * level.block + d * level.R].reshape(d, level.R)
        ve = v_exact(xq, t_nodes[l]).reshape(level.C, -1, d)
        err = 0.0
        for i in range(d):
            vh = np.einsum("qs,cs->cq", rt.phi, vn[i][level.cell_nodes])
            err += (vol * rt.Wq[None, :] * (vh - ve[:, :, i]) ** 2).sum()
        ev[l] = math.sqrt(err)
        pc = X[l * level.block + d * level.R:(l + 1) * level.block].reshape(level.C, d + 1)
        ph = np.einsum("qa,ca->cq", rt.xi, pc)
        pe = p_exact(xq, t_nodes[l]).reshape(level.C, -1)
        ep[l] = math.sqrt((vol * rt.Wq[None, :] * (ph - pe) ** 2).sum())
    return ev, ep


# ----------------------------------------------------------------------------------------------
# Intergrid transfer (Sec. 4.1): prolongation by interpolation, restriction by its transpose
# ----------------------------------------------------------------------------------------------
def prolongation(coarse: Level, fine: Level):
    """P: coarse DoF vector -> fine DoF vector, as a scipy CSR matrix [N_fine, N_coarse].

    Velocity: each fine Q2 node takes the value of the coarse Q2 function at its position
    (evaluated in an active coarse cell that contains it). Pressure: each fine cell takes the
    L2 projection of the coarse P1 function of its parent cell onto its own Legendre basis
    (exact, the spaces are nested). The same map acts on every component and time node.
    """
    d, K = fine.dim, fine.k + 1
    rows, cols, vals = [], [], []
    # velocity node map: fine lattice coords -> coarse cell + reference point
    fcoord = np.stack(np.unravel_index(fine.lat_of_node, fine.lshape[::-1])[::-1], axis=1)  # half-fine-cell units
    # position in coarse-cell units = fcoord / 4
    active_c = np.zeros(int(np.prod(coarse.cells)), dtype=np.int64) - 1
    active_c[coarse.active_full] = np.arange(coarse.C)
    vrows, vcols, vvals = [], [], []
    for nf in range(fine.R):
        pos = fcoord[nf] / 4.0
        cand = None
        # candidate coarse cells containing the point (lowest active index)
        base = np.floor(pos).astype(int)
        options = []
        for off in range(2**d):
            c = base - np.array([(off >> m) & 1 for m in range(d)])
            if np.any(c < 0) or np.any(c >= np.array(coarse.cells)):
                continue
            if np.any(pos < c) or np.any(pos > c + 1):
                continue
            cf = int(sum(c[m] * int(np.prod(coarse.cells[:m])) for m in range(d)))
            if active_c[cf] >= 0:
                options.append(active_c[cf])
        cand = min(options)
        ref = pos - coarse.cell_xyz[cand]
        phi, _ = q2_basis(ref[None, :])
        for s in range(3**d):
            if abs(phi[0, s]) > 0.0:
                vrows.append(nf)
                vcols.append(coarse.cell_nodes[cand, s])
                vvals.append(phi[0, s])
    Pv = sp.csr_matrix((vvals, (vrows, vcols)), shape=(fine.R, coarse.R))
    # pressure: projection onto the child's orthonormal Legendre basis
    Xq, Wq = volume_rule(d)
    xi_child = p1_basis(Xq)
    prow, pcol, pval = [], [], []
    for cf in range(fine.C):
        parent_xyz = fine.cell_xyz[cf] // 2
        o = fine.cell_xyz[cf] - 2 * parent_xyz
        cfull = int(sum(parent_xyz[m] * int(np.prod(coarse.cells[:m])) for m in range(d)))
        cp = active_c[cfull]
        xi_parent = p1_basis((Xq + o) / 2.0)
        Mproj = np.einsum("q,qa,qb->ab", Wq, xi_child, xi_parent)
        for a in range(d + 1):
            for b in range(d + 1):
                if Mproj[a, b] != 0.0:
                    prow.append(cf * (d + 1) + a)
                    pcol.append(cp * (d + 1) + b)
                    pval.append(Mproj[a, b])
    Pp = sp.csr_matrix((pval, (prow, pcol)), shape=(fine.S, coarse.S))
    blk = sp.block_diag([Pv] * d + [Pp])
    P = sp.block_diag([blk] * K, format="csr")
    P.eliminate_zeros()
    return P
