// C-ABI entry points of libstm (declared in include/stm.h).
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"

struct stm_hierarchy {
  stm::Hierarchy H;
};

namespace stm {
const char* last_error_cstr();
}

using namespace stm;


static stm_status bad_arg(const char* msg) {
  set_error(msg);
  return STM_ERR_INVALID_ARG;
}

static cudaStream_t S(void* p) { return reinterpret_cast<cudaStream_t>(p); }

namespace stm {
stm_status check_kernel_error(Hierarchy& H, cudaStream_t s) {
  int e = 0;
  STM_CUDA(cudaMemcpyAsync(&e, H.dkerr, sizeof(int), cudaMemcpyDeviceToHost, s));
  STM_CUDA(cudaStreamSynchronize(s));
  if (e) {
    STM_CUDA(cudaMemsetAsync(H.dkerr, 0, sizeof(int), s));
    set_error("a tensor-core pipeline wait timed out (error word " + std::to_string(e) + ")");
    return STM_ERR_CUDA;
  }
  return STM_OK;
}
}  // namespace stm

extern "C" {

const char* stm_last_error(void) { return last_error_cstr(); }

stm_status stm_build_hierarchy(const stm_params* params, stm_hierarchy** out) {
  if (!params || !out) return bad_arg("stm_build_hierarchy: NULL argument");
  *out = nullptr;
  const stm_params& p = *params;
  if (p.dim != 2 && p.dim != 3) return bad_arg("dim must be 2 or 3");
  if (p.k < 0 || p.k > 2) return bad_arg("k must be 0, 1 or 2");
  if (p.n_levels < 2 || p.n_levels > 12) return bad_arg("n_levels must be in [2, 12]");
  for (int m = 0; m < p.dim; ++m) {
    if (p.coarse_cells[m] < 1) return bad_arg("coarse_cells must be >= 1");
    if (!(p.length[m] > 0.0)) return bad_arg("length must be > 0");
    if (p.obstacle_lo[m] < 0 || p.obstacle_hi[m] > p.coarse_cells[m] || p.obstacle_lo[m] > p.obstacle_hi[m])
      return bad_arg("obstacle range outside the coarse grid");
  }
  if (p.inv_precision < STM_F64 || p.inv_precision > STM_BF16) return bad_arg("inv_precision");
  if (p.defect_precision != STM_F64 && p.defect_precision != STM_F32) return bad_arg("defect_precision must be F64 or F32");
  if (p.smoother < STM_VANKA_ADDITIVE || p.smoother > STM_VANKA_PAPER_OVERWRITE) return bad_arg("smoother");
  if (!(p.tau > 0.0) || !(p.nu >= 0.0) || p.nu1 < 0 || p.nu2 < 0) return bad_arg("tau, nu, nu1, nu2");
  stm_hierarchy* h = new (std::nothrow) stm_hierarchy();
  if (!h) {
    set_error("host allocation failed");
    return STM_ERR_OOM;
  }
  h->H.p = p;
  stm_status st = build_levels(h->H);
  if (st != STM_OK) {
    free_hierarchy(h->H);
    delete h;
    return st;
  }
  *out = h;
  return STM_OK;
}

void stm_destroy(stm_hierarchy* h) {
  if (!h) return;
  free_hierarchy(h->H);
  delete h;
}

stm_status stm_sizes(const stm_hierarchy* h, int level, long long* n_dofs, long long* n_cells, int* n_local,
                     long long* nnz) {
  if (!h) return bad_arg("NULL hierarchy");
  if (level < 0 || level >= (int)h->H.L.size()) return bad_arg("level out of range");
  const Level& L = h->H.L[level];
  if (n_dofs) *n_dofs = L.N;
  if (n_cells) *n_cells = L.C;
  if (n_local) *n_local = L.n;
  if (nnz) *nnz = L.nnz;
  return STM_OK;
}

stm_status stm_dof_lattice_index(const stm_hierarchy* h, int level, long long* out) {
  if (!h || !out) return bad_arg("NULL argument");
  if (level < 0 || level >= (int)h->H.L.size()) return bad_arg("level out of range");
  const Level& L = h->H.L[level];
  const long long W = L.dim * L.P_lat + (long long)L.np * L.Cfull;
  long long e = 0;
  for (int a = 0; a < L.K; ++a) {
    for (int l = 0; l < L.dim; ++l)
      for (int nd = 0; nd < L.R; ++nd) out[e++] = a * W + l * L.P_lat + L.h_node_lat[nd];
    for (int c = 0; c < L.C; ++c)
      for (int q = 0; q < L.np; ++q) out[e++] = a * W + L.dim * L.P_lat + (long long)L.h_cell_full[c] * L.np + q;
  }
  return STM_OK;
}

stm_status stm_assemble_jacobian(stm_hierarchy* h, const double* X, double nu, void* stream) {
  if (!h || !X) return bad_arg("NULL argument");
  Hierarchy& H = h->H;
  clear_graphs(H);
  STM_TRY(inject_linearisation(H, X, S(stream)));
  for (int g = 0; g < (int)H.L.size(); ++g) STM_TRY(assemble_level(H, g, nu, S(stream)));
  H.assembled = true;
  H.factored = false;
  return STM_OK;
}

stm_status stm_factor_cells(stm_hierarchy* h, void* stream, int* bad_level, long long* bad_cell) {
  if (!h) return bad_arg("NULL hierarchy");
  Hierarchy& H = h->H;
  if (!H.assembled) {
    set_error("factor_cells before assemble_jacobian");
    return STM_ERR_STATE;
  }
  if (bad_level) *bad_level = -1;
  if (bad_cell) *bad_cell = -1;
  clear_graphs(H);
  cudaStream_t s = S(stream);
  for (int g = 1; g < (int)H.L.size(); ++g) {
    STM_CUDA(cudaMemsetAsync(H.dflag, 0, sizeof(int) * 2, s));
    STM_CUDA(cudaMemsetAsync(H.dbad, 0xff, sizeof(long long), s));
    STM_TRY(factor_level(H, g, s));
    int flag = 0;
    long long bad = -1;
    STM_CUDA(cudaMemcpyAsync(&flag, H.dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
    STM_CUDA(cudaMemcpyAsync(&bad, H.dbad, sizeof(long long), cudaMemcpyDeviceToHost, s));
    STM_CUDA(cudaStreamSynchronize(s));
    if (flag) {
      if (bad_level) *bad_level = g;
      if (bad_cell) *bad_cell = bad;
      set_error("singular cell matrix (zero or non-finite pivot)");
      return STM_ERR_SINGULAR_CELL;
    }
  }
  STM_CUDA(cudaMemsetAsync(H.dflag + 1, 0, sizeof(int), s));
  STM_TRY(factor_coarse(H, s));
  int cflag = 0;
  STM_CUDA(cudaMemcpyAsync(&cflag, H.dflag + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  STM_CUDA(cudaStreamSynchronize(s));
  if (cflag) {
    if (bad_level) *bad_level = 0;
    set_error("singular coarse matrix");
    return STM_ERR_SINGULAR_CELL;
  }
  H.factored = true;
  return STM_OK;
}

static stm_status need_level(const Hierarchy& H, int level, int lo) {
  if (level < lo || level >= (int)H.L.size()) return bad_arg("level out of range");
  return STM_OK;
}

stm_status stm_spmv(stm_hierarchy* h, int level, const double* x, double* y, int transpose, void* stream) {
  if (!h || !x || !y) return bad_arg("NULL argument");
  STM_TRY(need_level(h->H, level, 0));
  if (!h->H.assembled) {
    set_error("spmv before assemble_jacobian");
    return STM_ERR_STATE;
  }
  return jacobian_apply(h->H, level, x, nullptr, y, 0, transpose, S(stream));
}

stm_status stm_defect(stm_hierarchy* h, int level, const double* r, const double* d, double* t, int transpose,
                      void* stream) {
  if (!h || !r || !d || !t) return bad_arg("NULL argument");
  if (t == r || t == d) return bad_arg("t must not alias r or d");
  STM_TRY(need_level(h->H, level, 0));
  if (!h->H.assembled) {
    set_error("defect before assemble_jacobian");
    return STM_ERR_STATE;
  }
  return smoother_defect(h->H, level, d, r, t, transpose, S(stream));
}

stm_status stm_vanka_sweep(stm_hierarchy* h, int level, const double* r, double* d, int transpose, void* stream) {
  if (!h || !r || !d) return bad_arg("NULL argument");
  STM_TRY(need_level(h->H, level, 1));
  if (!h->H.factored) {
    set_error("vanka_sweep before factor_cells");
    return STM_ERR_STATE;
  }
  return vanka_step(h->H, level, r, d, transpose, false, S(stream));
}

stm_status stm_restrict(stm_hierarchy* h, int level, const double* fine, double* coarse, void* stream) {
  if (!h || !fine || !coarse) return bad_arg("NULL argument");
  STM_TRY(need_level(h->H, level, 1));
  Level& L = h->H.L[level];
  return transfer_restrict(L, h->H.L[level - 1], fine, coarse, S(stream));
}

stm_status stm_prolongate_add(stm_hierarchy* h, int level, const double* coarse, double* fine, void* stream) {
  if (!h || !fine || !coarse) return bad_arg("NULL argument");
  STM_TRY(need_level(h->H, level, 1));
  Level& L = h->H.L[level];
  return transfer_prolong_add(L, h->H.L[level - 1], coarse, fine, S(stream));
}

stm_status stm_coarse_solve(stm_hierarchy* h, const double* r, double* d, int transpose, void* stream) {
  if (!h || !r || !d) return bad_arg("NULL argument");
  if (!h->H.factored) {
    set_error("coarse_solve before factor_cells");
    return STM_ERR_STATE;
  }
  return coarse_apply(h->H, r, d, transpose, S(stream));
}

stm_status stm_vcycle(stm_hierarchy* h, const double* r, double* d, int transpose, void* stream) {
  if (!h || !r || !d) return bad_arg("NULL argument");
  if (!h->H.factored) {
    set_error("vcycle before factor_cells");
    return STM_ERR_STATE;
  }
  return vcycle(h->H, r, d, transpose, S(stream));
}

// ---------------------------------------------------------------------------------------------
// Flexible GMRES (Sec. 3), right preconditioned, CGS with one re-orthogonalisation
// ---------------------------------------------------------------------------------------------
__global__ void k_scale_host(double* y, const double* x, double f, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = x[i] * f;
}

static stm_status ensure_krylov(Hierarchy& H, int m) {
  const long long N = H.L.back().N;
  if (H.restart_cap >= m && H.V) return STM_OK;
  void* ptrs[] = {H.V, H.Z, H.w, H.hcol, H.part, H.yvec};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  H.nblk_dot = 304;
  STM_CUDA(cudaMalloc(&H.V, sizeof(double) * (size_t)(m + 1) * N));
  STM_CUDA(cudaMalloc(&H.Z, sizeof(double) * (size_t)m * N));
  STM_CUDA(cudaMalloc(&H.w, sizeof(double) * (size_t)N));
  STM_CUDA(cudaMalloc(&H.hcol, sizeof(double) * (size_t)(2 * m + 8)));
  STM_CUDA(cudaMalloc(&H.part, sizeof(double) * (size_t)(m + 2) * H.nblk_dot));
  STM_CUDA(cudaMalloc(&H.yvec, sizeof(double) * (size_t)(m + 2)));
  H.restart_cap = m;
  return STM_OK;
}

static stm_status gmres_core(Hierarchy& H, const double* b, double* x, const stm_gmres_opts& o, stm_solve_info* info,
                             cudaStream_t s) {
  const int m = o.restart;
  const long long N = H.L.back().N;
  const int tr = o.transpose ? 1 : 0;
  const int G = (int)H.L.size();
  STM_TRY(ensure_krylov(H, m));
  const int nb = H.nblk_dot;
  const int sblocks = (int)std::min<long long>((N + 255) / 256, sm_count() * 8LL);
  stm_solve_info inf{};
  H.hist.clear();
  auto host_norm = [&](const double* v, double* out) -> stm_status {
    STM_TRY(vec_norm_sq(v, N, H.hcol, H.part, nb, s));
    double t = 0.0;
    STM_CUDA(cudaMemcpyAsync(&t, H.hcol, sizeof(double), cudaMemcpyDeviceToHost, s));
    STM_CUDA(cudaStreamSynchronize(s));
    *out = std::sqrt(t);
    return STM_OK;
  };
  double bnorm = 0.0;
  STM_TRY(host_norm(b, &bnorm));
  if (!std::isfinite(bnorm)) {
    set_error("non-finite right-hand side");
    return STM_ERR_NONFINITE;
  }
  if (!o.use_x0 || bnorm == 0.0) STM_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * N, s));
  if (bnorm == 0.0) {
    inf.converged = 1;
    inf.history = H.hist.data();
    if (info) *info = inf;
    return STM_OK;
  }
  const double tol = o.rtol * bnorm;
  std::vector<double> Hm((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), hc(m + 2), y(m);
  int it = 0, cycles = 0;
  bool converged = false, breakdown = false;
  double est = 1.0;
  for (;;) {
    // r = b - J x  -> V[0]. The stopping decision is taken on this true residual: a cycle that ends
    // because the recurrence estimate met rtol comes back here, and restarts if b - J x does not.
    // From x = 0 the first residual is b itself (exactly), so no product is needed.
    if (cycles == 0 && !o.use_x0) {
      STM_CUDA(cudaMemcpyAsync(H.V, b, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    } else {
      STM_TRY(jacobian_apply(H, G - 1, x, b, H.V, 1, tr, s));
    }
    double beta = 0.0;
    STM_TRY(host_norm(H.V, &beta));
    if (!std::isfinite(beta)) {
      set_error("non-finite residual norm");
      return STM_ERR_NONFINITE;
    }
    if (cycles == 0) est = beta / bnorm;
    inf.rel_res_true = beta / bnorm;
    H.hist.push_back(beta / bnorm);
    if (beta <= tol || it >= o.max_iter || breakdown) {
      converged = beta <= tol;
      break;
    }
    ++cycles;
    k_scale_host<<<sblocks, 256, 0, s>>>(H.V, H.V, 1.0 / beta, N); note_launch();
    std::fill(Hm.begin(), Hm.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int jd = 0;
    for (int j = 0; j < m; ++j) {
      double* vj = H.V + (size_t)j * N;
      double* zj = H.Z + (size_t)j * N;
      STM_TRY(vcycle_graph(H, vj, zj, tr, s));
      STM_TRY(jacobian_apply(H, G - 1, zj, nullptr, H.w, 0, tr, s));
      // classical Gram-Schmidt, twice
      ProfScope ps(&H, STM_KCLASS_KRYLOV, s, 8.0 * N * (4.0 * (j + 1) + 4.0));
      STM_TRY(batched_dots(H.V, j + 1, H.w, N, H.hcol, H.part, nb, s));
      STM_TRY(batched_update(H.V, j + 1, H.hcol, H.w, N, s));
      STM_TRY(batched_dots(H.V, j + 1, H.w, N, H.hcol + m + 2, H.part, nb, s));
      STM_TRY(batched_update(H.V, j + 1, H.hcol + m + 2, H.w, N, s));
      STM_TRY(vec_axpby_dev(H.hcol, H.hcol + m + 2, j + 1, s));
      STM_TRY(vec_norm_sq(H.w, N, H.hcol + j + 1, H.part, nb, s));
      STM_CUDA(cudaMemcpyAsync(hc.data(), H.hcol, sizeof(double) * (j + 2), cudaMemcpyDeviceToHost, s));
      STM_CUDA(cudaStreamSynchronize(s));
      const double hn = std::sqrt(hc[j + 1]);
      if (!std::isfinite(hn)) {
        set_error("non-finite Arnoldi norm");
        return STM_ERR_NONFINITE;
      }
      for (int i = 0; i <= j; ++i) Hm[(size_t)i * m + j] = hc[i];
      Hm[(size_t)(j + 1) * m + j] = hn;
      if (hn > 0.0) {
        k_scale_host<<<sblocks, 256, 0, s>>>(H.V + (size_t)(j + 1) * N, H.w, 1.0 / hn, N);
        note_launch();
      }
      for (int i = 0; i < j; ++i) {
        const double a = Hm[(size_t)i * m + j], bb = Hm[(size_t)(i + 1) * m + j];
        Hm[(size_t)i * m + j] = cs[i] * a + sn[i] * bb;
        Hm[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
      }
      const double a = Hm[(size_t)j * m + j], bb = Hm[(size_t)(j + 1) * m + j];
      const double rho = std::hypot(a, bb);
      if (!(rho > 0.0)) {
        // zero Hessenberg column: in flexible GMRES (Sec. 3) the new direction may add nothing even
        // though the least-squares problem is not solved; keep the columns before it and stop
        breakdown = true;
        break;
      }
      cs[j] = a / rho;
      sn[j] = bb / rho;
      Hm[(size_t)j * m + j] = rho;
      Hm[(size_t)(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++it;
      jd = j + 1;
      est = std::fabs(g[j + 1]) / bnorm;
      H.hist.push_back(est);
      // hn == 0 with rho > 0: the Krylov space is invariant and the least-squares solution exact
      if (std::fabs(g[j + 1]) <= tol || it >= o.max_iter || hn == 0.0) break;
    }
    // y = H^{-1} g (upper triangular), x += Z y
    for (int i = jd - 1; i >= 0; --i) {
      double t = g[i];
      for (int k2 = i + 1; k2 < jd; ++k2) t -= Hm[(size_t)i * m + k2] * y[k2];
      y[i] = t / Hm[(size_t)i * m + i];
    }
    if (jd > 0) {
      STM_CUDA(cudaMemcpyAsync(H.yvec, y.data(), sizeof(double) * jd, cudaMemcpyHostToDevice, s));
      STM_TRY(gemv_accumulate(H.Z, jd, H.yvec, x, N, s));
    }
  }
  inf.iters = it;
  inf.restarts = cycles > 0 ? cycles - 1 : 0;
  inf.converged = converged ? 1 : 0;
  inf.rel_res_est = est;
  inf.history = H.hist.data();
  inf.n_history = (int)H.hist.size();
  inf.graphs = (H.use_graphs && !H.prof.on) ? 1 : 0;
  if (info) *info = inf;
  if (!converged) {
    set_error(breakdown ? "FGMRES breakdown: zero column in the Hessenberg matrix before rtol was met"
                        : "FGMRES reached max_iter");
    return STM_ERR_NOT_CONVERGED;
  }
  return STM_OK;
}

stm_status stm_gmres_solve(stm_hierarchy* h, const double* b, double* x, const stm_gmres_opts* opts,
                           stm_solve_info* info, void* stream) {
  if (!h || !b || !x || !opts) return bad_arg("NULL argument");
  if (opts->restart < 1 || opts->restart > 200 || opts->max_iter < 0 || !(opts->rtol >= 0.0))
    return bad_arg("restart in [1,200], max_iter >= 0, rtol >= 0");
  if (!h->H.factored) {
    set_error("gmres_solve before factor_cells");
    return STM_ERR_STATE;
  }
  const auto t0 = std::chrono::steady_clock::now();
  const stm_status st = gmres_core(h->H, b, x, *opts, info, S(stream));
  if (info) info->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return st;
}

stm_status stm_gmres_solve_host(stm_hierarchy* h, const double* b_host, double* x_host, const stm_gmres_opts* opts,
                                stm_solve_info* info, void* stream) {
  if (!h || !b_host || !x_host || !opts) return bad_arg("NULL argument");
  if (!h->H.factored) {
    set_error("gmres_solve before factor_cells");
    return STM_ERR_STATE;
  }
  Hierarchy& H = h->H;
  const long long N = H.L.back().N;
  cudaStream_t s = S(stream);
  if (!H.bbuf) STM_CUDA(cudaMalloc(&H.bbuf, sizeof(double) * N));
  if (!H.xbuf) STM_CUDA(cudaMalloc(&H.xbuf, sizeof(double) * N));
  STM_CUDA(cudaMemcpyAsync(H.bbuf, b_host, sizeof(double) * N, cudaMemcpyHostToDevice, s));
  if (opts->use_x0) STM_CUDA(cudaMemcpyAsync(H.xbuf, x_host, sizeof(double) * N, cudaMemcpyHostToDevice, s));
  stm_status st = stm_gmres_solve(h, H.bbuf, H.xbuf, opts, info, stream);
  if (st != STM_OK && st != STM_ERR_NOT_CONVERGED) return st;
  STM_CUDA(cudaMemcpyAsync(x_host, H.xbuf, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
  STM_CUDA(cudaStreamSynchronize(s));
  return st;
}

// ---------------------------------------------------------------------------------------------
// Damped Newton for the nonlinear slab problem (Sec. 3, Eqs. nonlineq, linNewEq, linNewEqU)
// ---------------------------------------------------------------------------------------------
static stm_status assemble_all(Hierarchy& H, const double* X, double nu, cudaStream_t s) {
  clear_graphs(H);
  STM_TRY(inject_linearisation(H, X, s));
  for (int g = 0; g < (int)H.L.size(); ++g) STM_TRY(assemble_level(H, g, nu, s));
  H.assembled = true;
  H.factored = false;
  return STM_OK;
}

// With J = J(X) assembled at X: negF = (b + c(X, X)) - J(X) X = -F(X) (F = A X + c(X, X) - b, and
// J(X) X = A X + 2 c(X, X)); *norm = ||F(X)||_2.
static stm_status newton_residual(Hierarchy& H, const double* X, double U, double nu, const double* vprev,
                                  double* negF, double* norm, cudaStream_t s) {
  const long long N = H.L.back().N;
  STM_TRY(assemble_cellvec(H, 0, U, nu, nullptr, nullptr, H.nw_B, s, vprev));
  STM_TRY(jacobian_apply(H, (int)H.L.size() - 1, X, H.nw_B, negF, 1, 0, s));
  STM_TRY(vec_norm_sq(negF, N, H.hcol, H.part, H.nblk_dot, s));
  double t = 0.0;
  STM_CUDA(cudaMemcpyAsync(&t, H.hcol, sizeof(double), cudaMemcpyDeviceToHost, s));
  STM_CUDA(cudaStreamSynchronize(s));
  *norm = std::sqrt(t);
  if (!std::isfinite(*norm)) {
    set_error("non-finite nonlinear residual");
    return STM_ERR_NONFINITE;
  }
  return STM_OK;
}

stm_status stm_newton_solve(stm_hierarchy* h, double U, double nu, double* X, const double* prev,
                            const stm_newton_opts* nopts, const stm_gmres_opts* gopts, stm_newton_info* info,
                            void* stream) {
  if (!h || !X || !nopts || !gopts) return bad_arg("NULL argument");
  if (nopts->max_newton < 0 || nopts->max_newton > STM_NEWTON_MAX_STEPS || nopts->max_halvings < 0 ||
      nopts->max_halvings > 60 || !(nopts->abs_tol >= 0.0) || !(nopts->reduction >= 1.0))
    return bad_arg("max_newton in [0, STM_NEWTON_MAX_STEPS], max_halvings in [0, 60], abs_tol >= 0, reduction >= 1");
  if (gopts->restart < 1 || gopts->restart > 200 || gopts->max_iter < 0 || !(gopts->rtol >= 0.0))
    return bad_arg("restart in [1,200], max_iter >= 0, rtol >= 0");
  Hierarchy& H = h->H;
  cudaStream_t s = S(stream);
  const long long N = H.L.back().N;
  STM_TRY(ensure_krylov(H, gopts->restart));
  double** bufs[] = {&H.nw_negF, &H.nw_D, &H.nw_Xt, &H.nw_B, &H.nw_Ft};
  for (double** b : bufs)
    if (!*b) STM_CUDA(cudaMalloc((void**)b, sizeof(double) * N));
  // the previous slab's last time node (right Radau: the slab end) carries v(t_{n-1}^-)
  const double* vprev = prev ? prev + (long long)(H.L.back().K - 1) * H.L.back().block : nullptr;
  stm_newton_info inf{};
  stm_gmres_opts go = *gopts;
  go.transpose = 0;
  go.use_x0 = 0;
  double res = 0.0;
  STM_TRY(assemble_all(H, X, nu, s));
  STM_TRY(newton_residual(H, X, U, nu, vprev, H.nw_negF, &res, s));
  inf.res[0] = res;
  inf.n_res = 1;
  const double target = std::max(nopts->abs_tol, res / nopts->reduction);
  bool converged = res <= target;
  for (int m = 0; m < nopts->max_newton && !converged; ++m) {
    int bl = -1;
    long long bc = -1;
    STM_TRY(stm_factor_cells(h, stream, &bl, &bc));
    stm_solve_info si{};
    const stm_status st = gmres_core(H, H.nw_negF, H.nw_D, go, &si, s);
    inf.gmres_iters += si.iters;
    inf.gmres_step[m] = si.iters;
    if (st != STM_OK) {
      if (info) *info = inf;  // the steps taken so far
      return st;
    }
    double lam = 1.0, rt = 0.0;
    for (int hv = 0;; ++hv) {
      STM_TRY(vec_copy(H.nw_Xt, X, N, s));
      STM_TRY(vec_axpy(H.nw_Xt, lam, H.nw_D, N, s));
      STM_TRY(assemble_all(H, H.nw_Xt, nu, s));
      STM_TRY(newton_residual(H, H.nw_Xt, U, nu, vprev, H.nw_Ft, &rt, s));
      if (rt < res || hv == nopts->max_halvings) break;
      lam *= 0.5;
    }
    // accept: X <- X + lam D, -F(X) <- the trial's
    STM_TRY(vec_copy(X, H.nw_Xt, N, s));
    std::swap(H.nw_negF, H.nw_Ft);
    res = rt;
    inf.lam[m] = lam;
    inf.res[m + 1] = res;
    inf.n_res = m + 2;
    inf.newton_iters = m + 1;
    converged = res <= target;
  }
  inf.converged = converged ? 1 : 0;
  if (info) *info = inf;
  if (!converged) {
    set_error("Newton reached max_newton");
    return STM_ERR_NOT_CONVERGED;
  }
  return STM_OK;
}

stm_status stm_assemble_rhs(stm_hierarchy* h, double U, double nu, int which, double* b_dev, void* stream) {
  if (!h || !b_dev) return bad_arg("NULL argument");
  if (which < 0 || which > 2) return bad_arg("which must be 0 (b + c), 1 (db/dU) or 2 (db/dnu)");
  if (which == 0 && !h->H.assembled) {
    set_error("assemble_rhs(which=0) needs the linearisation point of assemble_jacobian");
    return STM_ERR_STATE;
  }
  return assemble_cellvec(h->H, which, U, nu, nullptr, nullptr, b_dev, S(stream));
}

stm_status stm_assemble_load(stm_hierarchy* h, double U, double nu, const double* w_dev, double* b_dev,
                             void* stream) {
  if (!h || !b_dev) return bad_arg("NULL argument");
  Hierarchy& H = h->H;
  cudaStream_t s = S(stream);
  if (!w_dev) {
    if (!H.assembled) {
      set_error("assemble_load without w needs the linearisation point of assemble_jacobian");
      return STM_ERR_STATE;
    }
    return assemble_cellvec(H, 0, U, nu, nullptr, nullptr, b_dev, s);
  }
  const Level& F = H.L.back();
  if (!H.ag_wnod) STM_CUDA(cudaMalloc(&H.ag_wnod, sizeof(double) * (size_t)F.K * F.dim * F.R));
  STM_TRY(inject_level(H, (int)H.L.size() - 1, w_dev, H.ag_wnod, s));
  return assemble_cellvec(H, 0, U, nu, nullptr, nullptr, b_dev, s, nullptr, H.ag_wnod);
}

stm_status stm_adjoint_gradient(stm_hierarchy* h, double U, double nu, const double* j_dev, const double* X_dev,
                                const stm_gmres_opts* opts, stm_solve_info* info, double* lambda_dev,
                                double* dJdU, double* dJdnu, void* stream) {
  if (!h || !j_dev || !X_dev || !opts || !dJdU || !dJdnu) return bad_arg("NULL argument");
  if (opts->restart < 1 || opts->restart > 200 || opts->max_iter < 0 || !(opts->rtol >= 0.0))
    return bad_arg("restart in [1,200], max_iter >= 0, rtol >= 0");
  Hierarchy& H = h->H;
  if (!H.factored) {
    set_error("adjoint_gradient before factor_cells");
    return STM_ERR_STATE;
  }
  const long long N = H.L.back().N;
  cudaStream_t s = S(stream);
  if (!H.ag_buf) STM_CUDA(cudaMalloc(&H.ag_buf, sizeof(double) * 4 * (size_t)N));
  double* dbdU = H.ag_buf;  // db/dU, db/dnu and (dJ/dnu) X back to back: one batched dot with lambda
  double* dbdnu = dbdU + N;
  double* dJX = dbdnu + N;
  double* lam = lambda_dev ? lambda_dev : dJX + N;
  stm_gmres_opts o = *opts;
  o.transpose = 1;
  o.use_x0 = 0;
  const auto t0 = std::chrono::steady_clock::now();
  const stm_status st = gmres_core(H, j_dev, lam, o, info, s);  // J^T lambda = j
  if (info) info->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (st != STM_OK) return st;
  STM_TRY(assemble_cellvec(H, 1, U, nu, nullptr, nullptr, dbdU, s));
  STM_TRY(assemble_cellvec(H, 2, U, nu, nullptr, nullptr, dbdnu, s));
  STM_TRY(dnu_apply(H, X_dev, dJX, s));
  STM_TRY(batched_dots(dbdU, 3, lam, N, H.hcol, H.part, H.nblk_dot, s));
  double dots[3] = {0.0, 0.0, 0.0};
  STM_CUDA(cudaMemcpyAsync(dots, H.hcol, sizeof(double) * 3, cudaMemcpyDeviceToHost, s));
  STM_CUDA(cudaStreamSynchronize(s));
  *dJdU = dots[0];
  *dJdnu = dots[1] - dots[2];
  return STM_OK;
}

stm_status stm_functional_weights(stm_hierarchy* h, const int* wake_lo, const int* wake_hi, double* j_dev,
                                  void* stream) {
  if (!h || !wake_lo || !wake_hi || !j_dev) return bad_arg("NULL argument");
  for (int m = 0; m < h->H.p.dim; ++m)
    if (wake_lo[m] < 0 || wake_hi[m] > h->H.p.coarse_cells[m] || wake_lo[m] > wake_hi[m])
      return bad_arg("wake box outside the level-1 grid");
  return assemble_cellvec(h->H, 3, 0.0, h->H.p.nu, wake_lo, wake_hi, j_dev, S(stream));
}

stm_status stm_jacobian_dnu_apply(stm_hierarchy* h, const double* x_dev, double* y_dev, void* stream) {
  if (!h || !x_dev || !y_dev) return bad_arg("NULL argument");
  return dnu_apply(h->H, x_dev, y_dev, S(stream));
}

stm_status stm_dot(stm_hierarchy* h, const double* x_dev, const double* y_dev, long long n, double* out,
                   void* stream) {
  if (!h || !x_dev || !y_dev || !out || n < 0) return bad_arg("NULL argument or negative size");
  Hierarchy& H = h->H;
  STM_TRY(ensure_krylov(H, std::max(H.restart_cap, 30)));
  cudaStream_t s = S(stream);
  STM_TRY(batched_dots(x_dev, 1, y_dev, n, H.hcol, H.part, H.nblk_dot, s));
  STM_CUDA(cudaMemcpyAsync(out, H.hcol, sizeof(double), cudaMemcpyDeviceToHost, s));
  STM_CUDA(cudaStreamSynchronize(s));
  return STM_OK;
}

// ---------------------------------------------------------------------------------------------
// Multi-right-hand-side smoothing step and FGMRES (up to 32 columns sharing one hierarchy)
// ---------------------------------------------------------------------------------------------
stm_status stm_vanka_sweep_multi(stm_hierarchy* h, int level, int nrhs, const double* R_dev, double* D_dev,
                                 void* stream) {
  if (!h || !R_dev || !D_dev) return bad_arg("NULL argument");
  if (nrhs < 1 || nrhs > 32) return bad_arg("nrhs must be in [1, 32]");
  STM_TRY(need_level(h->H, level, 1));
  if (!h->H.factored) {
    set_error("vanka_sweep_multi before factor_cells");
    return STM_ERR_STATE;
  }
  Hierarchy& H = h->H;
  if (H.p.smoother != STM_VANKA_ADDITIVE) return bad_arg("multi-RHS smoothing implements the additive smoother");
  STM_TRY(ensure_multi(H));
  Level& L = H.L[level];
  cudaStream_t s = S(stream);
  STM_TRY(multi_to_interleaved(R_dev, L.mr, L.N, nrhs, s));
  STM_TRY(multi_to_interleaved(D_dev, L.md, L.N, nrhs, s));
  STM_TRY(vanka_step_multi(H, level, L.mr, L.md, false, s));
  STM_TRY(multi_from_interleaved(L.md, D_dev, L.N, nrhs, s));
  return check_kernel_error(H, s);
}

stm_status stm_vanka_sweep_fused(stm_hierarchy* h, int level, int n_fwd, const double* Rf_dev, double* Df_dev,
                                 int n_adj, const double* Ra_dev, double* Da_dev, void* stream) {
  if (!h) return bad_arg("NULL argument");
  if (n_fwd < 0 || n_fwd > 16 || n_adj < 0 || n_adj > 16 || n_fwd + n_adj < 1)
    return bad_arg("n_fwd and n_adj must be in [0, 16], at least one column");
  if ((n_fwd && (!Rf_dev || !Df_dev)) || (n_adj && (!Ra_dev || !Da_dev))) return bad_arg("NULL argument");
  STM_TRY(need_level(h->H, level, 1));
  if (!h->H.factored) {
    set_error("vanka_sweep_fused before factor_cells");
    return STM_ERR_STATE;
  }
  Hierarchy& H = h->H;
  if (H.p.smoother != STM_VANKA_ADDITIVE) return bad_arg("the fused smoothing step implements the additive smoother");
  STM_TRY(ensure_multi(H));
  Level& L = H.L[level];
  cudaStream_t s = S(stream);
  // interleaved block: columns 0-15 forward, 16-31 adjoint (unused columns zero)
  STM_CUDA(cudaMemsetAsync(L.mr, 0, sizeof(double) * (size_t)L.N * 32, s));
  STM_CUDA(cudaMemsetAsync(L.md, 0, sizeof(double) * (size_t)L.N * 32, s));
  STM_TRY(multi_columns_in(Rf_dev, L.mr, L.N, n_fwd, 0, s));
  STM_TRY(multi_columns_in(Df_dev, L.md, L.N, n_fwd, 0, s));
  STM_TRY(multi_columns_in(Ra_dev, L.mr, L.N, n_adj, 16, s));
  STM_TRY(multi_columns_in(Da_dev, L.md, L.N, n_adj, 16, s));
  STM_TRY(vanka_step_multi(H, level, L.mr, L.md, false, s, 16));
  STM_TRY(multi_columns_out(L.md, Df_dev, L.N, n_fwd, 0, s));
  STM_TRY(multi_columns_out(L.md, Da_dev, L.N, n_adj, 16, s));
  return check_kernel_error(H, s);
}

static stm_status ensure_krylov_multi(Hierarchy& H, int m) {
  const size_t N = (size_t)H.L.back().N, NRs = 32;
  if (H.mrestart_cap >= m && H.mV) return STM_OK;
  void* ptrs[] = {H.mV, H.mZ, H.mW, H.mB, H.mX, H.mh, H.mpart, H.mf, H.my};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  STM_CUDA(cudaMalloc(&H.mV, sizeof(double) * (m + 1) * N * NRs));
  STM_CUDA(cudaMalloc(&H.mZ, sizeof(double) * m * N * NRs));
  STM_CUDA(cudaMalloc(&H.mW, sizeof(double) * N * NRs));
  STM_CUDA(cudaMalloc(&H.mB, sizeof(double) * N * NRs));
  STM_CUDA(cudaMalloc(&H.mX, sizeof(double) * N * NRs));
  STM_CUDA(cudaMalloc(&H.mh, sizeof(double) * (2 * m + 8) * NRs));
  STM_CUDA(cudaMalloc(&H.mpart, sizeof(double) * (m + 2) * 304 * NRs));
  STM_CUDA(cudaMalloc(&H.mf, sizeof(double) * NRs));
  STM_CUDA(cudaMalloc(&H.my, sizeof(double) * (m + 1) * NRs));
  H.mrestart_cap = m;
  return STM_OK;
}

stm_status stm_gmres_solve_multi(stm_hierarchy* h, int nrhs, const double* B_dev, double* X_dev,
                                 const stm_gmres_opts* opts, stm_solve_info* infos, void* stream) {
  if (!h || !B_dev || !X_dev || !opts) return bad_arg("NULL argument");
  if (nrhs < 1 || nrhs > 32) return bad_arg("nrhs must be in [1, 32]");
  if (opts->restart < 1 || opts->restart > 60 || opts->max_iter < 0 || !(opts->rtol >= 0.0))
    return bad_arg("restart in [1,60], max_iter >= 0, rtol >= 0");
  if (opts->transpose) return bad_arg("the multi-RHS solve implements J x = b only");
  Hierarchy& H = h->H;
  if (!H.factored) {
    set_error("gmres_solve_multi before factor_cells");
    return STM_ERR_STATE;
  }
  if (H.p.smoother != STM_VANKA_ADDITIVE) return bad_arg("multi-RHS solve implements the additive smoother");
  const int m = opts->restart;
  const int nb = 304;
  Level& F = H.L.back();
  const long long N = F.N;
  cudaStream_t s = S(stream);
  STM_TRY(ensure_multi(H));
  STM_TRY(ensure_krylov_multi(H, m));
  const size_t VS = (size_t)N * 32;  // doubles per multi-vector
  STM_TRY(multi_to_interleaved(B_dev, H.mB, N, nrhs, s));
  if (opts->use_x0) {
    STM_TRY(multi_to_interleaved(X_dev, H.mX, N, nrhs, s));
  } else {
    STM_CUDA(cudaMemsetAsync(H.mX, 0, sizeof(double) * VS, s));
  }
  std::vector<double> hbuf((2 * m + 8) * 32), fvec(32), yv((m + 1) * 32, 0.0);
  auto col_norms = [&](const double* V, double* out) -> stm_status {
    STM_TRY(mdots(V, 1, V, N, H.mh, H.mpart, nb, s));
    STM_CUDA(cudaMemcpyAsync(hbuf.data(), H.mh, sizeof(double) * 32, cudaMemcpyDeviceToHost, s));
    STM_CUDA(cudaStreamSynchronize(s));
    for (int c = 0; c < 32; ++c) out[c] = std::sqrt(hbuf[c]);
    return STM_OK;
  };
  double bnorm[32], beta[32];
  STM_TRY(col_norms(H.mB, bnorm));
  for (int c = 0; c < nrhs; ++c)
    if (!std::isfinite(bnorm[c])) {
      set_error("non-finite right-hand side");
      return STM_ERR_NONFINITE;
    }
  std::vector<int> iters(32, 0), conv(32, 0), cycles(32, 0), broke(32, 0);
  for (auto& v : H.mhist) v.clear();
  std::vector<double> est(32, 1.0), relres(32, 0.0);
  for (int c = 0; c < 32; ++c)
    if (c >= nrhs || bnorm[c] == 0.0) conv[c] = 1;
  std::vector<double> Hm((size_t)(m + 1) * m * 32), cs(m * 32), sn(m * 32), g((m + 1) * 32);
  int it = 0;
  for (;;) {
    // true residuals B - J X; a column counts as converged only when its true residual meets rtol
    // (a cycle that stopped on the recurrence estimate is checked here and restarted if needed)
    if (it == 0 && !opts->use_x0) {
      // from X = 0 the first residuals are the right-hand sides themselves (exactly)
      STM_CUDA(cudaMemcpyAsync(H.mV, H.mB, sizeof(double) * VS, cudaMemcpyDeviceToDevice, s));
    } else {
      ProfScope ps(&H, STM_KCLASS_JACOBIAN_SPMV, s, 8.0 * (double)F.nnz + 24.0 * 32 * (double)F.N,
                   (int)H.L.size() - 1);
      STM_TRY(spmm_structured(F, H.mX, H.mB, H.mV, 1, s));
    }
    STM_TRY(col_norms(H.mV, beta));
    bool any = false;
    std::vector<int> active(32, 0), jd(32, 0);
    for (int c = 0; c < 32; ++c) {
      if (c < nrhs && bnorm[c] > 0.0) {
        if (!std::isfinite(beta[c])) {
          set_error("non-finite residual norm");
          return STM_ERR_NONFINITE;
        }
        if (cycles[c] == 0) est[c] = beta[c] / bnorm[c];
        relres[c] = beta[c] / bnorm[c];
        H.mhist[c].push_back(relres[c]);
        conv[c] = beta[c] <= opts->rtol * bnorm[c];
      }
      active[c] = !conv[c] && !broke[c] && it < opts->max_iter;
      if (active[c]) cycles[c] += 1;
      any = any || active[c];
      fvec[c] = active[c] ? 1.0 / beta[c] : 0.0;
    }
    if (!any) break;
    STM_CUDA(cudaMemcpyAsync(H.mf, fvec.data(), sizeof(double) * 32, cudaMemcpyHostToDevice, s));
    STM_TRY(mscale(H.mV, H.mV, H.mf, N, s));
    std::fill(Hm.begin(), Hm.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    for (int c = 0; c < 32; ++c) g[c] = active[c] ? beta[c] : 0.0;  // g[j][c] at j * 32 + c
    int jmax = 0;
    for (int j = 0; j < m; ++j) {
      double* vj = H.mV + j * VS;
      double* zj = H.mZ + j * VS;
      STM_TRY(vcycle_multi(H, vj, zj, s));
      {
        ProfScope ps(&H, STM_KCLASS_JACOBIAN_SPMV, s, 8.0 * (double)F.nnz + 16.0 * 32 * (double)F.N,
                     (int)H.L.size() - 1);
        STM_TRY(spmm_structured(F, zj, nullptr, H.mW, 0, s));
      }
      {
        ProfScope ps(&H, STM_KCLASS_KRYLOV, s, 8.0 * VS * (4.0 * (j + 1) + 4.0));
        STM_TRY(mdots(H.mV, j + 1, H.mW, N, H.mh, H.mpart, nb, s));
        STM_TRY(mupdate(H.mV, j + 1, H.mh, H.mW, N, -1.0, s));
        STM_TRY(mdots(H.mV, j + 1, H.mW, N, H.mh + (m + 2) * 32, H.mpart, nb, s));
        STM_TRY(mupdate(H.mV, j + 1, H.mh + (m + 2) * 32, H.mW, N, -1.0, s));
        STM_TRY(madd_small(H.mh, H.mh + (m + 2) * 32, (j + 1) * 32, s));
        STM_TRY(mdots(H.mW, 1, H.mW, N, H.mh + (j + 1) * 32, H.mpart, nb, s));
      }
      STM_CUDA(cudaMemcpyAsync(hbuf.data(), H.mh, sizeof(double) * (j + 2) * 32, cudaMemcpyDeviceToHost, s));
      STM_TRY(check_kernel_error(H, s));
      ++it;
      jmax = j + 1;
      bool still = false;
      for (int c = 0; c < 32; ++c) {
        fvec[c] = 0.0;
        if (!active[c]) continue;
        auto Hc = [&](int r, int k) -> double& { return Hm[((size_t)r * m + k) * 32 + c]; };
        const double hn = std::sqrt(hbuf[(j + 1) * 32 + c]);
        if (!std::isfinite(hn)) {
          set_error("non-finite Arnoldi norm");
          return STM_ERR_NONFINITE;
        }
        for (int i = 0; i <= j; ++i) Hc(i, j) = hbuf[i * 32 + c];
        Hc(j + 1, j) = hn;
        for (int i = 0; i < j; ++i) {
          const double a = Hc(i, j), b = Hc(i + 1, j);
          Hc(i, j) = cs[i * 32 + c] * a + sn[i * 32 + c] * b;
          Hc(i + 1, j) = -sn[i * 32 + c] * a + cs[i * 32 + c] * b;
        }
        const double a = Hc(j, j), b = Hc(j + 1, j);
        const double rho = std::hypot(a, b);
        if (!(rho > 0.0)) {  // zero Hessenberg column (flexible GMRES breakdown): keep the earlier columns
          active[c] = 0;
          broke[c] = 1;
          continue;
        }
        cs[j * 32 + c] = a / rho;
        sn[j * 32 + c] = b / rho;
        Hc(j, j) = rho;
        Hc(j + 1, j) = 0.0;
        g[(j + 1) * 32 + c] = -sn[j * 32 + c] * g[j * 32 + c];
        g[j * 32 + c] = cs[j * 32 + c] * g[j * 32 + c];
        iters[c] += 1;
        jd[c] = j + 1;
        est[c] = std::fabs(g[(j + 1) * 32 + c]) / bnorm[c];
        H.mhist[c].push_back(est[c]);
        if (std::fabs(g[(j + 1) * 32 + c]) <= opts->rtol * bnorm[c] || hn == 0.0) {
          active[c] = 0;  // estimate met rtol (or an invariant Krylov space): checked at the next top
        } else if (it >= opts->max_iter) {
          active[c] = 0;
        } else {
          fvec[c] = 1.0 / hn;
          still = true;
        }
      }
      // next basis vector (columns that stopped get zeros)
      STM_CUDA(cudaMemcpyAsync(H.mf, fvec.data(), sizeof(double) * 32, cudaMemcpyHostToDevice, s));
      STM_TRY(mscale(H.mV + (j + 1) * VS, H.mW, H.mf, N, s));
      if (!still) break;
    }
    // per column: y = H^{-1} g over its own jd columns, x += Z y
    std::fill(yv.begin(), yv.end(), 0.0);
    for (int c = 0; c < 32; ++c) {
      for (int i = jd[c] - 1; i >= 0; --i) {
        double t = g[i * 32 + c];
        for (int k2 = i + 1; k2 < jd[c]; ++k2) t -= Hm[((size_t)i * m + k2) * 32 + c] * yv[k2 * 32 + c];
        yv[i * 32 + c] = t / Hm[((size_t)i * m + i) * 32 + c];
      }
    }
    STM_CUDA(cudaMemcpyAsync(H.my, yv.data(), sizeof(double) * jmax * 32, cudaMemcpyHostToDevice, s));
    STM_TRY(mupdate(H.mZ, jmax, H.my, H.mX, N, 1.0, s));
  }
  // the last loop top computed the true residuals of the returned X
  STM_TRY(multi_from_interleaved(H.mX, X_dev, N, nrhs, s));
  STM_CUDA(cudaStreamSynchronize(s));
  bool all = true, broken = false;
  for (int c = 0; c < nrhs; ++c) {
    all = all && conv[c];
    broken = broken || (broke[c] && !conv[c]);
    if (infos) {
      infos[c].iters = iters[c];
      infos[c].restarts = cycles[c] > 0 ? cycles[c] - 1 : 0;
      infos[c].converged = conv[c];
      infos[c].rel_res_true = relres[c];
      infos[c].rel_res_est = est[c];
      infos[c].history = H.mhist[c].data();
      infos[c].n_history = (int)H.mhist[c].size();
      infos[c].graphs = 0;
    }
  }
  if (!all) {
    set_error(broken ? "multi-RHS FGMRES breakdown (zero Hessenberg column) in some column"
                     : "multi-RHS FGMRES reached max_iter for some columns");
    return STM_ERR_NOT_CONVERGED;
  }
  return STM_OK;
}

stm_status stm_copy_jacobian(const stm_hierarchy* h, int level, long long* rowptr, int* colidx, double* val) {
  if (!h || !rowptr || !colidx || !val) return bad_arg("NULL argument");
  STM_TRY(need_level(h->H, level, 0));
  const Level& L = h->H.L[level];
  STM_CUDA(cudaDeviceSynchronize());
  STM_CUDA(cudaMemcpy(rowptr, L.rowptr, sizeof(long long) * (L.N + 1), cudaMemcpyDeviceToHost));
  STM_CUDA(cudaMemcpy(colidx, L.colidx, sizeof(int) * L.nnz, cudaMemcpyDeviceToHost));
  STM_CUDA(cudaMemcpy(val, L.val, sizeof(double) * L.nnz, cudaMemcpyDeviceToHost));
  return STM_OK;
}

stm_status stm_copy_cell_inverses(const stm_hierarchy* h, int level, double* out) {
  if (!h || !out) return bad_arg("NULL argument");
  STM_TRY(need_level(h->H, level, 1));
  const Hierarchy& H = h->H;
  if (!H.factored) {
    set_error("copy_cell_inverses before factor_cells");
    return STM_ERR_STATE;
  }
  const Level& L = H.L[level];
  const InvLayout lay = inv_layout(L.n, H.p.inv_precision);
  const size_t nn2 = (size_t)L.n * L.n, cs = (size_t)L.n * lay.ld, tot = cs * L.C;
  const int prec = H.p.inv_precision;
  const size_t es = prec == STM_F64 ? 8 : prec == STM_F32 ? 4 : 2;
  std::vector<unsigned char> raw(tot * es);
  STM_CUDA(cudaDeviceSynchronize());
  STM_CUDA(cudaMemcpy(raw.data(), L.inv, tot * es, cudaMemcpyDeviceToHost));
  for (size_t c = 0; c < (size_t)L.C; ++c)
    for (int j = 0; j < L.n; ++j)
      for (int i = 0; i < L.n; ++i) {
        const size_t e = c * cs + (size_t)j * lay.ld + i;  // stored column-major, leading dimension ld
        double v;
        if (prec == STM_F64) {
          std::memcpy(&v, &raw[e * 8], 8);
        } else if (prec == STM_F32) {
          float f;
          std::memcpy(&f, &raw[e * 4], 4);
          v = f;
        } else {
          uint16_t b16;
          std::memcpy(&b16, &raw[e * 2], 2);
          uint32_t u = (uint32_t)b16 << 16;
          float f;
          std::memcpy(&f, &u, 4);
          v = f;
        }
        out[c * nn2 + (size_t)i * L.n + j] = v;
      }
  return STM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Measurement support: launch counter and per-class event timing
// ---------------------------------------------------------------------------------------------
namespace stm {
std::atomic<long long> g_launches{0};

static cudaEvent_t pool_get(Profiler& P) {
  if (!P.pool.empty()) {
    cudaEvent_t e = P.pool.back();
    P.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

ProfScope::ProfScope(Hierarchy* H_, int cls_, cudaStream_t s_, double bytes_, int level_)
    : H(H_), cls(cls_), level(level_), s(s_), bytes(bytes_) {
  if (H && H->prof.on) {
    a = pool_get(H->prof);
    cudaEventRecord(a, s);
  }
}

ProfScope::~ProfScope() {
  if (a) {
    cudaEvent_t b = pool_get(H->prof);
    cudaEventRecord(b, s);
    H->prof.recs.push_back(ProfRec{a, b, cls, level, bytes});
  }
}

static void profile_drain(Profiler& P) {
  for (ProfRec& r : P.recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      const int slots[2] = {0, (r.level >= 0 && r.level + 1 < kProfLevels) ? r.level + 1 : -1};
      for (int k = 0; k < 2; ++k) {
        if (slots[k] < 0) continue;
        P.total_ms[r.cls][slots[k]] += ms;
        P.count[r.cls][slots[k]] += 1;
        P.bytes[r.cls][slots[k]] += r.bytes;
      }
    }
    P.pool.push_back(r.a);
    P.pool.push_back(r.b);
  }
  P.recs.clear();
}
}  // namespace stm

extern "C" {

stm_status stm_profile_enable(stm_hierarchy* h, int enable) {
  if (!h) return bad_arg("NULL hierarchy");
  Profiler& P = h->H.prof;
  STM_CUDA(cudaDeviceSynchronize());
  profile_drain(P);
  if (enable) {
    for (int c = 0; c < STM_KCLASS_COUNT; ++c)
      for (int l = 0; l < kProfLevels; ++l) P.total_ms[c][l] = 0.0, P.count[c][l] = 0, P.bytes[c][l] = 0.0;
  }
  P.on = enable != 0;
  return STM_OK;
}

stm_status stm_profile_read(stm_hierarchy* h, int kernel_class, int level, double* total_ms, long long* launches,
                            double* bytes) {
  if (!h) return bad_arg("NULL hierarchy");
  if (kernel_class < 0 || kernel_class >= STM_KCLASS_COUNT) return bad_arg("kernel_class out of range");
  if (level < -1 || level + 1 >= kProfLevels) return bad_arg("level out of range");
  Profiler& P = h->H.prof;
  STM_CUDA(cudaDeviceSynchronize());
  profile_drain(P);
  const int slot = level + 1;
  if (total_ms) *total_ms = P.total_ms[kernel_class][slot];
  if (launches) *launches = P.count[kernel_class][slot];
  if (bytes) *bytes = P.bytes[kernel_class][slot];
  return STM_OK;
}

long long stm_kernel_launches(void) { return g_launches.load(); }

}  // extern "C"
