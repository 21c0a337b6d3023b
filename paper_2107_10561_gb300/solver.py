"""Python binding of libstm: the C-ABI calls with torch tensors as device buffers.

Every method forwards to the entry point of the same name in include/stm.h; the binding only
checks shapes/dtypes/devices and converts pointers. All arithmetic runs in libstm's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib


def make_params(dim, k, n_levels, coarse_cells, length, obstacle_lo=(0, 0, 0), obstacle_hi=(0, 0, 0),
                tau=0.01, nu=1e-3, gamma1=35.0, gamma2=35.0, inv_precision="f64", smoother="additive",
                omega=0.7, nu1=2, nu2=2, defect_precision="f64"):
    p = _lib.StmParams()
    p.dim, p.k, p.n_levels = dim, k, n_levels
    pad = lambda t, v: list(t) + [v] * (3 - len(t))
    p.coarse_cells[:] = pad(coarse_cells, 1)
    p.length[:] = pad(length, 1.0)
    p.obstacle_lo[:] = pad(obstacle_lo, 0)
    p.obstacle_hi[:] = pad(obstacle_hi, 0)
    p.tau, p.nu, p.gamma1, p.gamma2 = tau, nu, gamma1, gamma2
    p.inv_precision = _lib.PRECISION[inv_precision] if isinstance(inv_precision, str) else inv_precision
    p.smoother = _lib.SMOOTHER[smoother] if isinstance(smoother, str) else smoother
    p.omega, p.nu1, p.nu2 = omega, nu1, nu2
    p.defect_precision = (_lib.PRECISION[defect_precision] if isinstance(defect_precision, str)
                          else defect_precision)
    return p


def _ptr(t, n=None, name="tensor"):
    import torch

    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA float64 tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} has {t.numel()} entries, expected {n}")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch

    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


class Hierarchy:
    """Owner of one libstm hierarchy (all levels' matrices, inverses and work vectors)."""

    def __init__(self, params: _lib.StmParams):
        self.lib = _lib.load()
        self.params = params
        h = C.c_void_p()
        _lib.check(self.lib.stm_build_hierarchy(C.byref(params), C.byref(h)), "stm_build_hierarchy")
        self.h = h
        self.n_levels = params.n_levels

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.lib.stm_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def finest(self):
        return self.n_levels - 1

    def sizes(self, level):
        n, c, nl, nnz = C.c_longlong(), C.c_longlong(), C.c_int(), C.c_longlong()
        _lib.check(self.lib.stm_sizes(self.h, level, C.byref(n), C.byref(c), C.byref(nl), C.byref(nnz)), "stm_sizes")
        return dict(n_dofs=n.value, n_cells=c.value, n_local=nl.value, nnz=nnz.value)

    def n_dofs(self, level=None):
        return self.sizes(self.finest if level is None else level)["n_dofs"]

    def dof_lattice_index(self, level=None):
        level = self.finest if level is None else level
        out = np.zeros(self.n_dofs(level), dtype=np.int64)
        _lib.check(self.lib.stm_dof_lattice_index(self.h, level, out.ctypes.data_as(_lib._LP)), "stm_dof_lattice_index")
        return out

    def assemble_jacobian(self, X, nu=None, stream=None):
        nu = self.params.nu if nu is None else nu
        _lib.check(self.lib.stm_assemble_jacobian(self.h, _ptr(X, self.n_dofs(), "X"), nu, _stream(stream)),
                   "stm_assemble_jacobian")

    def factor_cells(self, stream=None):
        bl, bc = C.c_int(), C.c_longlong()
        st = self.lib.stm_factor_cells(self.h, _stream(stream), C.byref(bl), C.byref(bc))
        if st != _lib.STM_OK:
            err = _lib.StmError(st, "stm_factor_cells", (self.lib.stm_last_error() or b"").decode())
            err.bad_level, err.bad_cell = bl.value, bc.value
            raise err

    def spmv(self, level, x, y, transpose=False, stream=None):
        n = self.n_dofs(level)
        _lib.check(self.lib.stm_spmv(self.h, level, _ptr(x, n, "x"), _ptr(y, n, "y"), int(transpose), _stream(stream)),
                   "stm_spmv")

    def defect(self, level, r, d, t, transpose=False, stream=None):
        """t = r - J_g d (or J_g^T d) as the V-cycle computes it (params.defect_precision)."""
        n = self.n_dofs(level)
        _lib.check(self.lib.stm_defect(self.h, level, _ptr(r, n, "r"), _ptr(d, n, "d"), _ptr(t, n, "t"),
                                       int(transpose), _stream(stream)), "stm_defect")

    def vanka_sweep(self, level, r, d, transpose=False, stream=None):
        n = self.n_dofs(level)
        _lib.check(self.lib.stm_vanka_sweep(self.h, level, _ptr(r, n, "r"), _ptr(d, n, "d"), int(transpose),
                                            _stream(stream)), "stm_vanka_sweep")

    def restrict(self, level, fine, coarse, stream=None):
        _lib.check(self.lib.stm_restrict(self.h, level, _ptr(fine, self.n_dofs(level), "fine"),
                                         _ptr(coarse, self.n_dofs(level - 1), "coarse"), _stream(stream)), "stm_restrict")

    def prolongate_add(self, level, coarse, fine, stream=None):
        _lib.check(self.lib.stm_prolongate_add(self.h, level, _ptr(coarse, self.n_dofs(level - 1), "coarse"),
                                               _ptr(fine, self.n_dofs(level), "fine"), _stream(stream)),
                   "stm_prolongate_add")

    def coarse_solve(self, r, d, transpose=False, stream=None):
        n = self.n_dofs(0)
        _lib.check(self.lib.stm_coarse_solve(self.h, _ptr(r, n, "r"), _ptr(d, n, "d"), int(transpose), _stream(stream)),
                   "stm_coarse_solve")

    def vcycle(self, r, d, transpose=False, stream=None):
        n = self.n_dofs()
        _lib.check(self.lib.stm_vcycle(self.h, _ptr(r, n, "r"), _ptr(d, n, "d"), int(transpose), _stream(stream)),
                   "stm_vcycle")

    @staticmethod
    def _opts(restart, max_iter, rtol, transpose, use_x0):
        o = _lib.GmresOpts()
        o.restart, o.max_iter, o.transpose, o.use_x0, o.rtol = restart, max_iter, int(transpose), int(use_x0), rtol
        return o

    @staticmethod
    def _info(inf):
        hist = [inf.history[i] for i in range(inf.n_history)] if inf.history and inf.n_history > 0 else []
        return dict(iters=inf.iters, restarts=inf.restarts, converged=bool(inf.converged),
                    rel_res_true=inf.rel_res_true, rel_res_est=inf.rel_res_est, history=hist,
                    ms_total=inf.ms_total, graphs=bool(inf.graphs))

    def gmres_solve(self, b, x, rtol=1e-10, restart=30, max_iter=1000, transpose=False, use_x0=False,
                    stream=None, raise_on_fail=True):
        n = self.n_dofs()
        o = self._opts(restart, max_iter, rtol, transpose, use_x0)
        inf = _lib.SolveInfo()
        st = self.lib.stm_gmres_solve(self.h, _ptr(b, n, "b"), _ptr(x, n, "x"), C.byref(o), C.byref(inf),
                                      _stream(stream))
        info = self._info(inf)
        info["status"] = _lib.STATUS_NAMES.get(st, st)
        if st != _lib.STM_OK and raise_on_fail:
            _lib.check(st, "stm_gmres_solve")
        return info

    def gmres_solve_host(self, b, x, rtol=1e-10, restart=30, max_iter=1000, transpose=False, use_x0=False,
                         stream=None, raise_on_fail=True):
        """b, x: host float64 arrays (numpy or CPU torch, ideally pinned) of n_dofs entries."""
        n = self.n_dofs()
        bp, xp = _host_ptr(b, n, "b"), _host_ptr(x, n, "x")
        o = self._opts(restart, max_iter, rtol, transpose, use_x0)
        inf = _lib.SolveInfo()
        st = self.lib.stm_gmres_solve_host(self.h, bp, xp, C.byref(o), C.byref(inf), _stream(stream))
        info = self._info(inf)
        info["status"] = _lib.STATUS_NAMES.get(st, st)
        if st != _lib.STM_OK and raise_on_fail:
            _lib.check(st, "stm_gmres_solve_host")
        return info

    def assemble_rhs(self, U, nu, b, which=0, stream=None):
        """b = b(U, nu) + c(w, w) (which=0), db/dU (1) or db/dnu (2) on the finest level."""
        _lib.check(self.lib.stm_assemble_rhs(self.h, float(U), float(nu), int(which), _ptr(b, self.n_dofs(), "b"),
                                             _stream(stream)), "stm_assemble_rhs")

    def assemble_load(self, U, nu, b, w=None, stream=None):
        """b = b(U, nu) + c(w, w) on the finest level for the linearisation point w (device DoF vector;
        None: the point of the last assemble_jacobian)."""
        n = self.n_dofs()
        _lib.check(self.lib.stm_assemble_load(self.h, float(U), float(nu), None if w is None else _ptr(w, n, "w"),
                                              _ptr(b, n, "b"), _stream(stream)), "stm_assemble_load")

    def adjoint_gradient(self, U, nu, j, X, lam=None, rtol=1e-12, restart=30, max_iter=1000, stream=None):
        """(dJ/dU, dJ/dnu, info) of J = j . X for the Newton step J(w; nu) X = b(U, nu) + c(w, w): the
        library solves J^T lambda = j and forms lambda . db/dU and lambda . (db/dnu - (dJ/dnu) X)."""
        n = self.n_dofs()
        o = self._opts(restart, max_iter, rtol, True, False)
        inf = _lib.SolveInfo()
        gU, gnu = C.c_double(), C.c_double()
        st = self.lib.stm_adjoint_gradient(self.h, float(U), float(nu), _ptr(j, n, "j"), _ptr(X, n, "X"), C.byref(o),
                                           C.byref(inf), None if lam is None else _ptr(lam, n, "lambda"),
                                           C.byref(gU), C.byref(gnu), _stream(stream))
        info = self._info(inf)
        info["status"] = _lib.STATUS_NAMES.get(st, st)
        _lib.check(st, "stm_adjoint_gradient")
        return gU.value, gnu.value, info

    def newton_solve(self, X, U, nu=None, max_newton=20, max_halvings=8, abs_tol=1e-10, reduction=1e4,
                     rtol=1e-10, restart=30, max_iter=1000, prev=None, stream=None, raise_on_fail=True):
        """Damped Newton for the slab problem F(X) = A X + c(X, X) - b(U, nu) = 0 (stm_newton_solve).

        X: device float64 [n_dofs], initial iterate, overwritten with the last iterate.
        prev: None (initial value U g_1 e_x) or the previous slab's device DoF vector (time marching)."""
        nu = self.params.nu if nu is None else nu
        no = _lib.NewtonOpts(int(max_newton), int(max_halvings), float(abs_tol), float(reduction))
        go = self._opts(restart, max_iter, rtol, False, False)
        inf = _lib.NewtonInfo()
        pp = None if prev is None else _ptr(prev, self.n_dofs(), "prev")
        st = self.lib.stm_newton_solve(self.h, float(U), float(nu), _ptr(X, self.n_dofs(), "X"), pp, C.byref(no),
                                       C.byref(go), C.byref(inf), _stream(stream))
        info = {"newton_iters": inf.newton_iters, "gmres_iters": inf.gmres_iters, "converged": bool(inf.converged),
                "res": [inf.res[i] for i in range(inf.n_res)], "lam": [inf.lam[i] for i in range(inf.newton_iters)],
                "gmres_step": [inf.gmres_step[i] for i in range(inf.newton_iters)],
                "status": _lib.STATUS_NAMES.get(st, st)}
        if st != _lib.STM_OK and raise_on_fail:
            _lib.check(st, "stm_newton_solve")
        return info

    def time_march(self, X_init, U, n_slabs, j=None, **newton_kw):
        """Slabs 1..n_slabs in sequence (Problem 3.1): slab n starts from the previous slab's state and
        takes its last time node as initial value. Returns the slab states (device tensors), the Newton
        infos and, with functional weights j (device), the history j . X_n."""
        import torch
        states, infos, values = [], [], []
        prev = X_init
        for _ in range(n_slabs):
            X = prev.clone()
            infos.append(self.newton_solve(X, U, prev=prev, **newton_kw))
            states.append(X)
            if j is not None:
                values.append(self.dot(j, X))
            prev = X
        return states, infos, values

    def functional_weights(self, wake_lo, wake_hi, j, stream=None):
        lo = (C.c_int * 3)(*(list(wake_lo) + [0] * (3 - len(wake_lo))))
        hi = (C.c_int * 3)(*(list(wake_hi) + [1] * (3 - len(wake_hi))))
        _lib.check(self.lib.stm_functional_weights(self.h, lo, hi, _ptr(j, self.n_dofs(), "j"), _stream(stream)),
                   "stm_functional_weights")

    def jacobian_dnu_apply(self, x, y, stream=None):
        n = self.n_dofs()
        _lib.check(self.lib.stm_jacobian_dnu_apply(self.h, _ptr(x, n, "x"), _ptr(y, n, "y"), _stream(stream)),
                   "stm_jacobian_dnu_apply")

    def dot(self, x, y, stream=None):
        out = C.c_double()
        n = x.numel()
        _lib.check(self.lib.stm_dot(self.h, _ptr(x, n, "x"), _ptr(y, n, "y"), n, C.byref(out), _stream(stream)),
                   "stm_dot")
        return out.value

    def vanka_sweep_multi(self, level, R, D, stream=None):
        """One additive smoothing step for every column of R, D: CUDA float64 [nrhs, n_dofs]."""
        nrhs, n = R.shape
        if tuple(D.shape) != (nrhs, n) or n != self.n_dofs(level):
            raise ValueError("R and D must be [nrhs, n_dofs(level)]")
        _lib.check(self.lib.stm_vanka_sweep_multi(self.h, level, nrhs, _ptr(R, nrhs * n, "R"), _ptr(D, nrhs * n, "D"),
                                                  _stream(stream)), "stm_vanka_sweep_multi")

    def vanka_sweep_fused(self, level, Rf, Df, Ra, Da, stream=None):
        """One additive smoothing step for forward columns (Rf, Df: CUDA float64 [n_fwd <= 16, n_dofs]) and
        adjoint columns (Ra, Da: [n_adj <= 16, n_dofs]) from one pass over the cell inverses."""
        n = self.n_dofs(level)
        nf = 0 if Rf is None else Rf.shape[0]
        na = 0 if Ra is None else Ra.shape[0]
        for A, B, k in ((Rf, Df, nf), (Ra, Da, na)):
            if k and (tuple(A.shape) != (k, n) or tuple(B.shape) != (k, n)):
                raise ValueError("R and D must be [ncols, n_dofs(level)]")
        _lib.check(self.lib.stm_vanka_sweep_fused(self.h, level, nf, _ptr(Rf, nf * n, "Rf") if nf else None,
                                                  _ptr(Df, nf * n, "Df") if nf else None, na,
                                                  _ptr(Ra, na * n, "Ra") if na else None,
                                                  _ptr(Da, na * n, "Da") if na else None, _stream(stream)),
                   "stm_vanka_sweep_fused")

    def gmres_solve_multi(self, B, X, rtol=1e-8, restart=30, max_iter=1000, use_x0=False, stream=None,
                          raise_on_fail=True):
        """Lock-stepped FGMRES for every column of B: CUDA float64 [nrhs <= 32, n_dofs]; returns per-column infos."""
        nrhs, n = B.shape
        if tuple(X.shape) != (nrhs, n) or n != self.n_dofs():
            raise ValueError("B and X must be [nrhs, n_dofs]")
        o = self._opts(restart, max_iter, rtol, False, use_x0)
        infos = (_lib.SolveInfo * nrhs)()
        st = self.lib.stm_gmres_solve_multi(self.h, nrhs, _ptr(B, nrhs * n, "B"), _ptr(X, nrhs * n, "X"), C.byref(o),
                                            infos, _stream(stream))
        out = [self._info(i) for i in infos]
        if st != _lib.STM_OK and raise_on_fail:
            _lib.check(st, "stm_gmres_solve_multi")
        return out

    def profile_enable(self, enable=True):
        _lib.check(self.lib.stm_profile_enable(self.h, int(enable)), "stm_profile_enable")

    def profile_read(self, kernel_class, level=-1):
        """(total event ms, launches, algorithmic bytes) of one kernel class (one level, -1: all)."""
        ms, n, by = C.c_double(), C.c_longlong(), C.c_double()
        cls = _lib.KCLASS[kernel_class] if isinstance(kernel_class, str) else kernel_class
        _lib.check(self.lib.stm_profile_read(self.h, cls, int(level), C.byref(ms), C.byref(n), C.byref(by)),
                   "stm_profile_read")
        return dict(ms=ms.value, launches=n.value, bytes=by.value)

    @staticmethod
    def measure_fp64_peak(stream=None):
        out = C.c_double()
        lib = _lib.load()
        _lib.check(lib.stm_measure_fp64_peak(C.byref(out), _stream(stream)), "stm_measure_fp64_peak")
        return out.value

    @staticmethod
    def selftest_bounded_wait(stream=None):
        """(timed_out, ms) of the bounded-wait self-test (stm_selftest_bounded_wait)."""
        t, ms = C.c_int(), C.c_double()
        lib = _lib.load()
        _lib.check(lib.stm_selftest_bounded_wait(C.byref(t), C.byref(ms), _stream(stream)),
                   "stm_selftest_bounded_wait")
        return bool(t.value), ms.value

    @staticmethod
    def kernel_launches():
        return int(_lib.load().stm_kernel_launches())

    def copy_jacobian(self, level):
        import scipy.sparse as sp

        s = self.sizes(level)
        rowptr = np.zeros(s["n_dofs"] + 1, dtype=np.int64)
        col = np.zeros(s["nnz"], dtype=np.int32)
        val = np.zeros(s["nnz"], dtype=np.float64)
        _lib.check(self.lib.stm_copy_jacobian(self.h, level, rowptr.ctypes.data_as(_lib._LP),
                                              col.ctypes.data_as(_lib._IP), val.ctypes.data_as(_lib._DP)),
                   "stm_copy_jacobian")
        return sp.csr_matrix((val, col, rowptr), shape=(s["n_dofs"], s["n_dofs"]))

    def copy_cell_inverses(self, level):
        s = self.sizes(level)
        out = np.zeros((s["n_cells"], s["n_local"], s["n_local"]))
        _lib.check(self.lib.stm_copy_cell_inverses(self.h, level, out.ctypes.data_as(_lib._DP)), "stm_copy_cell_inverses")
        return out


def vanka_apply_noalloc(inv_colmajor, idx, t, d, omega, stream=None):
    """Allocation-free additive Vanka correction (stm_vanka_apply_noalloc): d += omega W sum_T R_T^T J_T^{-1} t_T.

    inv_colmajor: CUDA float64 [C, n, n] with inv_colmajor[c, j, i] = (J_T^{-1})_{ij};
    idx: CUDA int32 [C, n]; t, d: CUDA float64 [N]. No device memory is allocated by the library.
    """
    import torch

    lib = _lib.load()
    C_, n, n2 = inv_colmajor.shape
    if n != n2 or tuple(idx.shape) != (C_, n) or idx.dtype != torch.int32 or not idx.is_cuda or not idx.is_contiguous():
        raise ValueError("inv must be [C, n, n] and idx a contiguous CUDA int32 [C, n]")
    N = t.numel()
    _lib.check(lib.stm_vanka_apply_noalloc(C_, n, N, _ptr(inv_colmajor, C_ * n * n, "inv"), C.c_void_p(idx.data_ptr()),
                                           _ptr(t, N, "t"), _ptr(d, N, "d"), float(omega), _stream(stream)),
               "stm_vanka_apply_noalloc")


def _host_ptr(a, n, name):
    import torch

    if isinstance(a, torch.Tensor):
        if a.is_cuda or a.dtype != torch.float64 or not a.is_contiguous() or a.numel() != n:
            raise ValueError(f"{name}: host contiguous float64 tensor of {n} entries expected")
        return C.cast(C.c_void_p(a.data_ptr()), _lib._DP)
    a = np.ascontiguousarray(a)
    if a.dtype != np.float64 or a.size != n:
        raise ValueError(f"{name}: float64 array of {n} entries expected")
    return a.ctypes.data_as(_lib._DP)
