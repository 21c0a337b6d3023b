/*
 * libstm — space-time multigrid for one dG(k) time slab of the incompressible Navier–Stokes
 * equations, discretised with the inf-sup stable Q2/P1^disc pair, on one GPU.
 *
 * The library solves the Newton system J d = r of one time slab (Eq. linNewEq, Eq. LinSysMG of
 * Anselmann & Bause, arXiv 2107.10561) by flexible GMRES right-preconditioned with one geometric
 * multigrid V-cycle (Algorithm 1) whose smoother is the cell-based space-time Vanka smoother
 * (Sec. 4.2, Eq. LocVanka, with the damping factor of Sec. 5.3) built from precomputed dense
 * cell inverses on every level (Sec. 4.3).
 *
 * Conventions shared by every entry point:
 *  - Pointers named *_dev are device pointers (e.g. torch CUDA tensors), FP64, contiguous, owned
 *    by the caller; *_host pointers are host memory owned by the caller. The library never keeps
 *    a caller pointer after a call returns. Everything else (matrices, inverses, work vectors) is
 *    allocated by stm_build_hierarchy and freed by stm_destroy.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream). Calls enqueue
 *    work on it and return without synchronising, except where a comment says otherwise.
 *  - Vector layout (Eq. totdofs): for each time node l = 0..k: velocity component 1 (R entries),
 *    ..., component d (R entries), then the pressure (n_p entries per active cell, cell-major).
 *    Q2 nodes are numbered lexicographically (x fastest) over the level's full node lattice with
 *    the nodes of removed obstacle cells compressed out; active cells likewise.
 *  - Cell-local layout (Eq. locdofs): per time node l, velocity component 1..d over the 3^d
 *    cell nodes (x fastest), then the n_p Legendre pressure modes; n = (k+1)(d 3^d + n_p).
 *  - Levels are numbered 0 (coarsest) .. n_levels-1 (finest).
 *  - Errors are reported by return code only (never abort, never throw); stm_last_error()
 *    returns a thread-local message for the last failing call on the calling thread.
 */
#ifndef STM_H
#define STM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stm_hierarchy stm_hierarchy;

typedef enum {
  STM_OK = 0,
  STM_ERR_INVALID_ARG = 1,   /* bad parameter, level index, size or NULL pointer            */
  STM_ERR_CUDA = 2,          /* a CUDA runtime call failed (message names it)               */
  STM_ERR_OOM = 3,           /* device or host allocation failed                            */
  STM_ERR_SINGULAR_CELL = 4, /* a cell matrix (or the coarse matrix) had a zero/non-finite pivot */
  STM_ERR_NOT_CONVERGED = 5, /* FGMRES hit max_iter before reaching rtol; x holds last iterate */
  STM_ERR_NONFINITE = 6,     /* NaN/Inf met in a residual norm                              */
  STM_ERR_STATE = 7          /* call order violated (e.g. vcycle before factor_cells)       */
} stm_status;

typedef enum { STM_F64 = 0, STM_F32 = 1, STM_BF16 = 2 } stm_precision;

typedef enum {
  STM_VANKA_ADDITIVE = 0,       /* d += omega W sum_T R_T^T J_T^{-1} R_T (r - J d), W = diag(1/m_i) */
  STM_VANKA_COLOURED = 1,       /* 2^d colours; per colour: t = r - J d, d_T += omega J_T^{-1} t_T  */
  STM_VANKA_PAPER_OVERWRITE = 2 /* Sec. 4.2 literal: one residual, each DoF keeps the update of
                                   its highest-index cell ("last update in the loop wins")         */
} stm_smoother;

/* Problem and method parameters (r = 2 fixed: Q2/P1disc, Eq. Def:Vh0).
 * Geometry: box [0,length[0]] x [0,length[1]] (x [0,length[2]]), uniform level-1 grid of
 * coarse_cells cells, refined n_levels-1 times by bisection; the level-1 cells with
 * obstacle_lo[m] <= index[m] < obstacle_hi[m] for all m are removed (lo == hi: no obstacle).
 * x = 0 is the inflow part of Gamma_D, x = length[0] the do-nothing outflow Gamma_o, every other
 * boundary face (channel walls, obstacle surface) belongs to Gamma_D (Sec. 2.1). */
typedef struct {
  int dim;               /* 2 or 3                                                        */
  int k;                 /* dG(k) time degree, 0..2 (Sec. 2.4)                            */
  int n_levels;          /* G >= 2                                                        */
  int coarse_cells[3];   /* level-1 grid                                                  */
  double length[3];      /* box size                                                      */
  int obstacle_lo[3], obstacle_hi[3];
  double tau, nu;        /* slab length and viscosity                                     */
  double gamma1, gamma2; /* Nitsche penalties (Eq. Def:B_GamD; the paper uses 35, 35)     */
  int inv_precision;     /* stm_precision of the stored cell inverses                     */
  int smoother;          /* stm_smoother                                                  */
  double omega;          /* damping omega_d of the local update (Sec. 5.3)                */
  int nu1, nu2;          /* pre-/post-smoothing steps of the V-cycle                      */
  int defect_precision;  /* stm_precision of the V-cycle's defects r - J_g d (smoothing steps
                            and the defect before restriction): STM_F64, or STM_F32 = FP32 copies
                            of J_g's values (kept in step with every assembly), FP32 products
                            and sums, FP64 vectors. STM_BF16 is rejected. The FGMRES products
                            and true residuals are FP64 in every case; flexible GMRES (Sec. 3)
                            keeps each preconditioned vector, so an inexact V-cycle only changes
                            the iteration count. The multi-RHS V-cycle keeps FP64 defects.
                            Zero-initialised structs get STM_F64.                              */
} stm_params;

/* Host setup of all levels (numbering, cell->DoF maps, colours, multiplicities, CSR patterns of
 * J_g, transfer matrices) and upload to the current CUDA device. Synchronous.
 * Cites: mesh hierarchy V^1 c ... c V^G of Sec. 4.1; local DoF sets of Eq. locdofs. */
stm_status stm_build_hierarchy(const stm_params* params, stm_hierarchy** out);

/* Sizes of one level: n_dofs = (k+1)(d R + n_p C), n_cells = C, n_local = n, nnz of J_g. */
stm_status stm_sizes(const stm_hierarchy* h, int level, long long* n_dofs, long long* n_cells,
                     int* n_local, long long* nnz);

/* For every global DoF of `level`, its index into the flattened lattice state of that level:
 * shape [k+1][d*P + n_p*Cf] with P = prod(2 c_m + 1) lattice points and Cf = prod(c_m) cells,
 * velocity entry l*W + comp*P + lattice_index, pressure entry l*W + d*P + full_cell*n_p + mode.
 * out_host: n_dofs int64 values, caller-owned. Synchronous. */
stm_status stm_dof_lattice_index(const stm_hierarchy* h, int level, long long* out_host);

/* Assemble the slab Jacobian J_g on every level (Problem 3.1 linearised as in Eq. linNewEq,
 * forms of Eqs. Def:Ah and Def:B_GamD, time blocks of Eq. newton_system_matrix_dG_1) at the
 * linearisation point whose finest-level DoF vector is X_dev (only its velocity is used; coarse
 * levels take its values at their own nodes, which are fine nodes). nu overrides params.nu.
 * Invalidates previous cell factors. */
stm_status stm_assemble_jacobian(stm_hierarchy* h, const double* X_dev, double nu, void* stream);

/* For every level g >= 1 and every cell T: J_T = J_g[idx_T, idx_T] (the rows and columns of the
 * assembled matrix, Sec. 4.4), explicit inverse by Gauss-Jordan elimination with partial pivoting
 * in FP64, stored in params.inv_precision (Sec. 4.3). Level 0: explicit FP64 inverse of J_0 for
 * the direct coarse solve (Algorithm 1). Synchronises once to read the pivot flags; on
 * STM_ERR_SINGULAR_CELL, *bad_level / *bad_cell name the first failing cell (cell -1: coarse). */
stm_status stm_factor_cells(stm_hierarchy* h, void* stream, int* bad_level, long long* bad_cell);

/* y = J_g x (transpose = 0) or y = J_g^T x (transpose = 1); x, y: n_dofs of `level`. */
stm_status stm_spmv(stm_hierarchy* h, int level, const double* x_dev, double* y_dev, int transpose,
                    void* stream);

/* The V-cycle's defect t = r - J_g d (transpose = 1: r - J_g^T d) on `level`, computed as inside
 * Algorithm 1 (before each smoothing step with d != 0 and before the restriction): in FP64, or
 * with params.defect_precision = STM_F32 over FP32 copies of J_g's values (d rounded to FP32 to
 * nearest, FP32 products and sums, r and t in FP64). r, d, t: n_dofs of `level`, device; t must not
 * alias r or d. STM_ERR_STATE before stm_assemble_jacobian. */
stm_status stm_defect(stm_hierarchy* h, int level, const double* r_dev, const double* d_dev, double* t_dev,
                      int transpose, void* stream);

/* One smoothing step d <- S(d, r) on level g >= 1 with params.smoother and params.omega
 * (Eq. LocVanka with damping; residual r - J_g d recomputed inside, as stm_defect computes it, in
 * params.defect_precision). transpose = 1 smooths for J_g^T with the transposed cell inverses. */
stm_status stm_vanka_sweep(stm_hierarchy* h, int level, const double* r_dev, double* d_dev,
                           int transpose, void* stream);

/* Restriction coarse = P^T fine (level g -> g-1) and prolongation fine += P coarse
 * (g-1 -> g); P interpolates the coarse Q2/P1disc function (Sec. 4.1, MGTransferPrebuilt). */
stm_status stm_restrict(stm_hierarchy* h, int level, const double* fine_dev, double* coarse_dev,
                        void* stream);
stm_status stm_prolongate_add(stm_hierarchy* h, int level, const double* coarse_dev,
                              double* fine_dev, void* stream);

/* Direct coarse solve d = J_0^{-1} r (or J_0^{-T} r). */
stm_status stm_coarse_solve(stm_hierarchy* h, const double* r_dev, double* d_dev, int transpose,
                            void* stream);

/* One V(nu1,nu2)-cycle (Algorithm 1) on the finest level with zero initial guess: d = M^{-1} r.
 * Equal, bit for bit, to its steps composed through stm_vanka_sweep, stm_defect, stm_restrict,
 * stm_coarse_solve and stm_prolongate_add. */
stm_status stm_vcycle(stm_hierarchy* h, const double* r_dev, double* d_dev, int transpose,
                      void* stream);

typedef struct {
  int restart;   /* Krylov dimension m of FGMRES(m), e.g. 30                         */
  int max_iter;  /* total iteration limit (the paper treats 1000 as divergence)      */
  int transpose; /* 1: solve J^T x = b (adjoint) with the transposed preconditioner  */
  int use_x0;    /* 1: x_dev holds the initial guess on entry; 0: start from x = 0   */
  double rtol;   /* a cycle ends when the recurrence estimate of ||b - J x||_2 drops to
                    rtol ||b||_2; the solve ends when the recomputed true residual does (else
                    it restarts from x)                                                  */
} stm_gmres_opts;

typedef struct {
  int iters;           /* FGMRES iterations (preconditioner applications)             */
  int restarts;        /* completed restart cycles                                    */
  int converged;       /* 1 if the true residual ||b - J x||_2 <= rtol ||b||_2 at exit  */
  double rel_res_true; /* ||b - J x||_2 / ||b||_2 recomputed at exit                  */
  double rel_res_est;  /* last recurrence estimate                                    */
  const double* history; /* relative residual history: entry 0 the initial true residual,
                            then the recurrence estimate after every iteration and the true
                            residual at every restart; library-owned host memory, valid
                            until the next solve on the same hierarchy                  */
  int n_history;       /* entries of history                                          */
  double ms_total;     /* host wall time of the call in ms (the call synchronises)    */
  int graphs;          /* 1 if the V-cycles of this call were replayed from CUDA graphs
                          (0 with profiling on, for the 32-column solve, or if capture
                          was refused and the V-cycles were launched directly)          */
} stm_solve_info;

/* Right-preconditioned flexible GMRES (Sec. 3) on the finest level, preconditioned by one
 * V-cycle per iteration, classical Gram-Schmidt with re-orthogonalisation. Synchronises once
 * per iteration to read the new Hessenberg column for the stopping test. Returns
 * STM_ERR_NOT_CONVERGED (x = last iterate, info filled) if max_iter is reached before the true
 * residual meets rtol, or on a breakdown (a zero column of the rotated Hessenberg matrix, possible
 * in flexible GMRES when a preconditioned direction adds nothing). */
stm_status stm_gmres_solve(stm_hierarchy* h, const double* b_dev, double* x_dev,
                           const stm_gmres_opts* opts, stm_solve_info* info, void* stream);

/* Same solve with HOST buffers: b_host is copied to the device, the solution is copied back
 * into x_host (use_x0: x_host holds the initial guess). Synchronous on return. */
stm_status stm_gmres_solve_host(stm_hierarchy* h, const double* b_host, double* x_host,
                                const stm_gmres_opts* opts, stm_solve_info* info, void* stream);

/* Right-hand side of one Newton step from the linearisation point w of the last
 * stm_assemble_jacobian, on the finest level (Problem 3.1 with f = 0, Eqs. Def:Lh, Def:B_GamD):
 *   which = 0: b(U, nu) + c(w, w), where b(U, nu) = int_{I_n} B_GamD(g, (psi, xi)) dt
 *              + <v(t_{n-1}^-), psi(t_{n-1}^+)> with inflow data g = U g_1 on x = 0 (g = 0 on walls and
 *              obstacle), previous-slab state U g_1 e_x, g_1 the Poiseuille profile 4y(H-y)/H^2
 *              (3D: 16 y(H-y) z(L-z)/(H^2 L^2)), and c(w, w) = sum_bc T_abc <(w^c . grad) w^b, psi>;
 *              then J(w) X = b + c is exactly one Newton step from w;
 *   which = 1: db/dU (b is linear in U);   which = 2: db/dnu (b is affine in nu).
 * b_dev: FP64 [n_dofs of the finest level], overwritten. */
stm_status stm_assemble_rhs(stm_hierarchy* h, double U, double nu, int which, double* b_dev, void* stream);

/* Load vector of one Newton step on the finest level (Problem 3.1 with f = 0, Eqs. Def:Lh, Def:B_GamD,
 * linearised as in Eq. linNewEq): b_dev = b(U, nu) + c(w, w) for the linearisation point w whose
 * finest-level DoF vector is w_dev (only its velocity is used), with b and c as for stm_assemble_rhs
 * (which = 0). w_dev = NULL takes the point of the last stm_assemble_jacobian. The assembled matrices
 * and the stored linearisation point are left unchanged. b_dev: FP64 [n_dofs], overwritten.
 * STM_ERR_STATE for w_dev = NULL before any assembly. */
stm_status stm_assemble_load(stm_hierarchy* h, double U, double nu, const double* w_dev, double* b_dev,
                             void* stream);

/* Gradient of the drag-like functional J(X) = j . X of one Newton step J(w; nu) X = b(U, nu) + c(w, w)
 * with respect to the inflow amplitude U and the viscosity nu (adjoint method; the paper has no
 * gradient, the formulas follow from differentiating Eq. linNewEq with w fixed):
 *   solve J^T lambda = j with the transposed GMG-preconditioned FGMRES of stm_gmres_solve
 *   (opts->transpose and opts->use_x0 are ignored; lambda starts from zero), then
 *   *dJdU  = lambda . db/dU,
 *   *dJdnu = lambda . (db/dnu - (dJ/dnu) X),
 * J assembled at w with this nu and factored (stm_factor_cells) beforehand; X_dev the forward solution
 * (FP64 [n_dofs]); j_dev the functional weights (stm_functional_weights). lambda_dev: NULL, or an FP64
 * [n_dofs] buffer that receives lambda. info (may be NULL) describes the adjoint solve. Synchronous.
 * Errors: the FGMRES errors (STM_ERR_NOT_CONVERGED leaves the gradient outputs untouched). */
stm_status stm_adjoint_gradient(stm_hierarchy* h, double U, double nu, const double* j_dev, const double* X_dev,
                                const stm_gmres_opts* opts, stm_solve_info* info, double* lambda_dev,
                                double* dJdU, double* dJdnu, void* stream);

/* Nonlinear slab problem F(X) = 0 (Sec. 3, Eq. nonlineq) with the data of stm_assemble_rhs:
 *   F(X) = A X + c(X, X) - b(U, nu),  A the linear part of the slab operator, c the convection term,
 * solved by damped Newton (Eqs. linNewEq, linNewEqU): step m assembles J(X^m) on every level (coarse
 * levels take X^m at their nodes), factors the cells, solves J(X^m) D = -F(X^m) with the
 * GMG-preconditioned FGMRES of stm_gmres_solve (gopts; transpose and use_x0 ignored), and sets
 * X^{m+1} = X^m + lambda D with the first lambda in 1, 1/2, 1/4, ... (at most max_halvings halvings)
 * that lowers ||F||_2. Stops when ||F|| <= max(abs_tol, ||F(X^0)|| / reduction) (Sec. 5.1 uses 1e-10
 * and 1e4). F is evaluated as (b + c(X, X)) - J(X) X, which equals -F since J(X) X = A X + 2 c(X, X).
 * prev_dev: NULL, or the previous slab's FP64 finest-level DoF vector (time marching, Problem 3.1): the
 * initial value v(t_{n-1}^-) is then the velocity of its last time node (right Radau: the slab end), and
 * b holds <v_h(t_{n-1}^-), psi(t_{n-1}^+)> for that discrete field instead of the Poiseuille state.
 * X_dev: FP64 [n_dofs of the finest level], the initial iterate on entry and the last iterate on
 * return (also on STM_ERR_NOT_CONVERGED). On return J is assembled at the last iterate and the cell
 * factors are stale (call stm_factor_cells before another linear solve). Synchronises once per
 * residual evaluation. Errors: STM_ERR_INVALID_ARG, STM_ERR_NONFINITE, STM_ERR_SINGULAR_CELL, the
 * FGMRES errors, STM_ERR_NOT_CONVERGED after max_newton steps. */
#define STM_NEWTON_MAX_STEPS 32
typedef struct {
  int max_newton;    /* Newton steps at most, <= STM_NEWTON_MAX_STEPS */
  int max_halvings;  /* line-search halvings per step at most (0: undamped) */
  double abs_tol;    /* stop when ||F|| <= abs_tol ... */
  double reduction;  /* ... or when ||F|| <= ||F(X^0)|| / reduction (>= 1) */
} stm_newton_opts;
typedef struct {
  int newton_iters;  /* steps taken */
  int gmres_iters;   /* FGMRES iterations over all steps */
  int converged;
  int n_res;         /* valid entries of res (newton_iters + 1) */
  double res[STM_NEWTON_MAX_STEPS + 1]; /* ||F(X^m)||_2, m = 0 .. newton_iters */
  double lam[STM_NEWTON_MAX_STEPS];     /* accepted step lengths */
  int gmres_step[STM_NEWTON_MAX_STEPS]; /* FGMRES iterations of each step */
} stm_newton_info;
stm_status stm_newton_solve(stm_hierarchy* h, double U, double nu, double* X_dev, const double* prev_dev,
                            const stm_newton_opts* nopts, const stm_gmres_opts* gopts, stm_newton_info* info,
                            void* stream);

/* Weights j of the drag-like functional J(X) = int_{I_n} int_wake v_1 dx dt = j . X, where the wake
 * is the union of finest cells inside the level-1 cell box [wake_lo, wake_hi) (all z in 3D).
 * j_dev: FP64 [n_dofs of the finest level], overwritten. */
stm_status stm_functional_weights(stm_hierarchy* h, const int* wake_lo, const int* wake_hi, double* j_dev,
                                  void* stream);

/* y = (dJ/dnu) x on the finest level. J is affine in nu; its nu-part is the diffusion and the
 * gamma1 / symmetric Nitsche terms of Eqs. Def:Ah and Def:B_GamD, diagonal in time (Mt). */
stm_status stm_jacobian_dnu_apply(stm_hierarchy* h, const double* x_dev, double* y_dev, void* stream);

/* *out = x . y over n entries (FP64, deterministic reduction). Synchronous. */
stm_status stm_dot(stm_hierarchy* h, const double* x_dev, const double* y_dev, long long n, double* out,
                   void* stream);

/* Multi-right-hand-side path: nrhs <= 32 columns share the hierarchy (one J, one set of cell
 * inverses). Vectors are column-major [nrhs][n_dofs] (leading dimension n_dofs), FP64, on the device.
 *  - stm_vanka_sweep_multi: one additive smoothing step D <- S(D, R) on level g >= 1 for every column
 *    (Eq. LocVanka with damping). The local products Y_T = J_T^{-1} T_T run on the 32-column blocks:
 *    with BF16 inverses on the tensor cores (FP32 accumulation; T split into two BF16 parts so that the
 *    only rounding is the stored inverse's), with FP32 / FP64 inverses on CUDA cores.
 *  - stm_gmres_solve_multi: right-preconditioned FGMRES per column, lock-stepped so that every
 *    iteration applies one 32-column V-cycle (Algorithm 1) and one 32-column product with J; each
 *    column keeps its own Arnoldi basis, Hessenberg matrix and stopping test. infos: nrhs entries.
 *    Additive smoother and J x = b only (transpose must be 0); restart <= 60. Synchronises once per
 *    iteration. Returns STM_ERR_NOT_CONVERGED if some column hits max_iter. */
stm_status stm_vanka_sweep_multi(stm_hierarchy* h, int level, int nrhs, const double* R_dev, double* D_dev,
                                 void* stream);
stm_status stm_gmres_solve_multi(stm_hierarchy* h, int nrhs, const double* B_dev, double* X_dev,
                                 const stm_gmres_opts* opts, stm_solve_info* infos, void* stream);

/* One additive smoothing step (Eq. LocVanka, damped, multiplicity-weighted) on level g >= 1 for n_fwd
 * right-hand sides of J d = r and n_adj of the adjoint system J^T d = r at once, with one pass over the
 * stored cell inverses: forward columns get d += omega W sum_T R_T^T J_T^{-1} R_T (r - J d), adjoint
 * columns d += omega W sum_T R_T^T J_T^{-T} R_T (r - J^T d). With BF16 inverses both local products run
 * on the tensor cores from the same shared-memory copy of each inverse (read as J_T^{-1} and as J_T^{-T}).
 * Rf/Df: [n_fwd][n_dofs], Ra/Da: [n_adj][n_dofs], column-major FP64 on the device (D updated in place),
 * 0 <= n_fwd, n_adj <= 16. Synchronises once at the end (reports a timed-out tensor-core pipeline as
 * STM_ERR_CUDA). The paper smooths one system at a time; pairing forward and adjoint columns over one read
 * of the inverses (which dominate the bytes of a sweep, Sec. 4.3) is this library's addition, for a
 * forward solve and its adjoint that share J. */
stm_status stm_vanka_sweep_fused(stm_hierarchy* h, int level, int n_fwd, const double* Rf_dev, double* Df_dev,
                                 int n_adj, const double* Ra_dev, double* Da_dev, void* stream);

/* Copies of internal data for verification (synchronous, caller-owned host buffers):
 * the CSR of J_g (rowptr: n_dofs+1, colidx/val: nnz) and the cell inverses of level g >= 1 as
 * FP64, row-major per cell ([n_cells][n][n], converted from the stored precision). */
stm_status stm_copy_jacobian(const stm_hierarchy* h, int level, long long* rowptr_host,
                             int* colidx_host, double* val_host);
stm_status stm_copy_cell_inverses(const stm_hierarchy* h, int level, double* inv_host);

/* Additive Vanka correction that allocates nothing. The paper has no counterpart: this entry point
 * exists for integration only.
 *
 * For callers that must not allocate device memory once they are running -- for example code
 * whose device memory is owned by another component's pool allocator, or latency-critical loops
 * that cannot afford the implicit device synchronisation of cudaMalloc/cudaFree. It needs no
 * hierarchy: the caller passes every input and output, and the library allocates nothing.
 *
 * Computes, for all cells T at once,
 *   d_i += omega * (1/m_i) * sum over the cells T containing i of (J_T^{-1} t_T)_i,
 * with m_i the number of cells whose DoF list contains i (DoFs in no cell are left unchanged).
 *   inv_dev : n_cells cell inverses, FP64, each n_local x n_local COLUMN-major, back to back
 *   idx_dev : int32 [n_cells][n_local] global DoF of each local DoF (entries outside
 *             [0, n_dofs) are ignored)
 *   t_dev   : FP64 [n_dofs] residual r - J d;  d_dev: FP64 [n_dofs], updated in place
 * Limits: n_dofs <= 1048576 (else STM_ERR_INVALID_ARG, nothing launched), 1 <= n_local <= 1024.
 * Scratch: a fixed 16 MiB file-scope device array, present on every device that loads the library
 * until the process exits. Every call looks up that array's device address on the current device
 * (so calls after cudaDeviceReset, or on another device, get the address valid there); the first
 * call on a device, and the first after a reset, also loads the library's device code there, so make
 * it before any stream capture. Every call reuses the same array and clears the part it needs, so
 * calls that overlap on the GPU (other streams, other host threads) race with each other and must be
 * serialised by the caller. The shared-DoF sum uses FP64 atomics, so the result matches
 * stm_vanka_sweep(additive) up to summation order. */
stm_status stm_vanka_apply_noalloc(long long n_cells, int n_local, long long n_dofs, const double* inv_dev,
                                   const int* idx_dev, const double* t_dev, double* d_dev, double omega,
                                   void* stream);

/* Measurement support (not part of the method). Kernel classes whose launches can be timed with
 * CUDA events recorded on the launching stream, and the algorithmic bytes each launch moves:
 *   VANKA_LOCAL   y_T = J_T^{-1} t_T over the cells of one launch: C (n^2 s + 20 n) bytes
 *                 (inverse in storage width s, int32 index map, gathered t, written y);
 *   JACOBIAN_SPMV residual / product with J_g: 8 nnz + 24 N bytes (values, x, y, b; column
 *                 indices are representation overhead and not counted);
 *   VANKA_COMBINE second pass of the additive/overwrite smoother; TRANSFER P and P^T products;
 *   COARSE        dense coarse solve; KRYLOV Gram-Schmidt, norms and updates of FGMRES;
 *   DEFECT_F32    the V-cycle's defect r - J_g d over the FP32 copies (defect_precision =
 *                 STM_F32): 4 nnz + 20 N bytes (values, d in FP32, r, t);
 *   ROUND_F32     the rounding of d to FP32 that precedes each FP32 defect: 12 N bytes. */
typedef enum {
  STM_KCLASS_VANKA_LOCAL = 0,
  STM_KCLASS_JACOBIAN_SPMV = 1,
  STM_KCLASS_VANKA_COMBINE = 2,
  STM_KCLASS_TRANSFER = 3,
  STM_KCLASS_COARSE = 4,
  STM_KCLASS_KRYLOV = 5,
  STM_KCLASS_DEFECT_F32 = 6,
  STM_KCLASS_ROUND_F32 = 7
} stm_kernel_class;

/* Turn event timing of kernel launches on (1) or off (0); turning it on clears the records. */
stm_status stm_profile_enable(stm_hierarchy* h, int enable);
/* Synchronises the device and returns, for one kernel class on one level (-1: all levels), the
 * summed event time (ms), the number of timed launches and the summed algorithmic bytes since
 * profiling was enabled. Per-level figures exist for VANKA_LOCAL, VANKA_COMBINE, JACOBIAN_SPMV,
 * DEFECT_F32. */
stm_status stm_profile_read(stm_hierarchy* h, int kernel_class, int level, double* total_ms, long long* launches,
                            double* bytes);
/* Measured FP64 FMA throughput of the current device in TFLOP/s (8 independent FMA chains per thread,
 * best of two timed runs). The FP64 products with J are bound by this rate on GB300. Synchronous. */
stm_status stm_measure_fp64_peak(double* tflops, void* stream);
/* Verification of the bounded waits of the pipelined kernels (the tensor-core smoother): one thread
 * waits on an mbarrier phase that nothing completes, with the same helper the pipelines use. The wait
 * gives up after one second of wall time and sets bit 128 of a device error word; the kernel then
 * returns normally and the context stays usable. *timed_out = 1 when the bit was set, *ms = the
 * kernel's CUDA-event time. Synchronous; allocates and frees 4 bytes of device memory. */
stm_status stm_selftest_bounded_wait(int* timed_out, double* ms, void* stream);

/* Number of kernel launches issued by this library in this process so far. */
long long stm_kernel_launches(void);

void stm_destroy(stm_hierarchy* h);
const char* stm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* STM_H */
