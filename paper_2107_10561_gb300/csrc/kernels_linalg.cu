// Sparse and dense FP64 linear algebra of the V-cycle and of FGMRES:
//  * CSR products with J_g (residual t = r - J d, Alg. 1 and Eq. LocVanka), with P and P^T (Sec. 4.1);
//  * J_g^T on the same, structurally symmetric pattern (values permuted once per assembly);
//  * the coarse solve d = J_0^{-1} r as a dense matrix-vector product with the explicit inverse;
//  * Gram-Schmidt building blocks of flexible GMRES (batched dots / updates, norms).
#include "internal.h"

namespace stm {

static int sms() { return sm_count(); }

// VL lanes per row (VL = 1, 2, 4, 8, 16 or 32, chosen from the mean row length); values and column
// indices are streamed once (cache-streaming loads), x stays cached. mode 0: y = A x;
// 1: y = b - A x; 2: y += A x.
template <int VL>
__global__ void __launch_bounds__(256) k_csr(const long long* __restrict__ rowptr, const int* __restrict__ col,
                                             const double* __restrict__ val, long long nrows,
                                             const double* __restrict__ x, const double* __restrict__ b,
                                             double* __restrict__ y, int mode) {
  // The row loop is uniform across each warp (a warp owns 32/VL consecutive rows per step), so the
  // full-mask shuffles below always see all 32 lanes.
  constexpr int GPW = 32 / VL;
  const int lane = threadIdx.x & (VL - 1);
  const int gw = (threadIdx.x & 31) / VL;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long wb = warp * GPW; wb < nrows; wb += nwarps * GPW) {
    const long long row = wb + gw;
    const bool ok = row < nrows;
    const long long e0 = ok ? rowptr[row] : 0, e1 = ok ? rowptr[row + 1] : 0;
    double s0 = 0.0, s1 = 0.0;
    long long e = e0 + lane;
    for (; e + VL < e1; e += 2 * VL) {
      const double v0 = __ldcs(val + e), v1 = __ldcs(val + e + VL);
      const int c0 = __ldcs(col + e), c1 = __ldcs(col + e + VL);
      s0 += v0 * __ldg(x + c0);
      s1 += v1 * __ldg(x + c1);
    }
    if (e < e1) s0 += __ldcs(val + e) * __ldg(x + __ldcs(col + e));
    double s = s0 + s1;
#pragma unroll
    for (int off = VL / 2; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off, VL);
    if (ok && lane == 0) {
      if (mode == 0) y[row] = s;
      else if (mode == 1) y[row] = b[row] - s;
      else y[row] += s;
    }
  }
}

stm_status csr_apply(const long long* rowptr, const int* col, const double* val, long long nrows, long long nnz,
                     const double* x, const double* b, double* y, int mode, cudaStream_t s) {
  if (nrows <= 0) return STM_OK;
  const double mean = (double)nnz / (double)nrows;
  int VL = 1;
  while (VL < 32 && VL < mean * 0.75) VL *= 2;
  const long long threads_needed = nrows * VL;
  const int blocks = (int)std::min<long long>((threads_needed + 255) / 256, (long long)sms() * 8);
  switch (VL) {
    case 1: k_csr<1><<<blocks, 256, 0, s>>>(rowptr, col, val, nrows, x, b, y, mode); break;
    case 2: k_csr<2><<<blocks, 256, 0, s>>>(rowptr, col, val, nrows, x, b, y, mode); break;
    case 4: k_csr<4><<<blocks, 256, 0, s>>>(rowptr, col, val, nrows, x, b, y, mode); break;
    case 8: k_csr<8><<<blocks, 256, 0, s>>>(rowptr, col, val, nrows, x, b, y, mode); break;
    case 16: k_csr<16><<<blocks, 256, 0, s>>>(rowptr, col, val, nrows, x, b, y, mode); break;
    default: k_csr<32><<<blocks, 256, 0, s>>>(rowptr, col, val, nrows, x, b, y, mode); break;
  }
  note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}

// valT[p] = value of the mirrored entry (col, row) of entry p = (row, col) (binary search in row col).
__global__ void k_transpose_values(const long long* __restrict__ rowptr, const int* __restrict__ col,
                                   const double* __restrict__ val, double* __restrict__ valT, long long nrows,
                                   int* flag) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long row = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < nrows; row += warps) {
    for (long long e = rowptr[row] + lane; e < rowptr[row + 1]; e += 32) {
      const int j = col[e];
      long long lo = rowptr[j], hi = rowptr[j + 1] - 1;
      double v = 0.0;
      bool found = false;
      while (lo <= hi) {
        const long long mid = (lo + hi) >> 1;
        const int cm = col[mid];
        if (cm == (int)row) { v = val[mid]; found = true; break; }
        if (cm < (int)row) lo = mid + 1; else hi = mid - 1;
      }
      if (!found) atomicExch(flag, 1);
      valT[e] = v;
    }
  }
}

stm_status ensure_transpose(Hierarchy& H, int g, cudaStream_t s) {
  Level& L = H.L[g];
  if (L.valT) return STM_OK;
  STM_CUDA(cudaMalloc(&L.valT, sizeof(double) * L.nnz));
  STM_CUDA(cudaMemsetAsync(H.dflag + 2, 0, sizeof(int), s));
  const int blocks = (int)std::min<long long>((L.N + 7) / 8, (long long)sms() * 16);
  k_transpose_values<<<blocks, 256, 0, s>>>(L.rowptr, L.colidx, L.val, L.valT, L.N, H.dflag + 2); note_launch();
  STM_CUDA(cudaGetLastError());
  int flag = 0;
  STM_CUDA(cudaMemcpyAsync(&flag, H.dflag + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
  STM_CUDA(cudaStreamSynchronize(s));
  if (flag) {
    set_error("J pattern is not structurally symmetric");
    return STM_ERR_STATE;
  }
  // node-block and pressure-row copies of J^T for the transposed SpMV
  STM_CUDA(cudaMalloc(&L.nvalJT, sizeof(double) * L.nval_len));
  STM_CUDA(cudaMalloc(&L.pvalJT, sizeof(double) * L.pval_len));
  STM_CUDA(cudaMemsetAsync(L.pvalJT, 0, sizeof(double) * L.pval_len, s));
  STM_TRY(build_nodeblock_from(L, L.valT, L.nvalJT, L.pvalJT, s));
  if (H.p.defect_precision == STM_F32) STM_TRY(build_values_f32(L, 1, s));
  return STM_OK;
}

stm_status jacobian_apply(Hierarchy& H, int g, const double* x, const double* b, double* y, int mode,
                          int transpose, cudaStream_t s) {
  Level& L = H.L[g];
  if (transpose) STM_TRY(ensure_transpose(H, g, s));
  ProfScope ps(&H, STM_KCLASS_JACOBIAN_SPMV, s, 8.0 * (double)L.nnz + 24.0 * (double)L.N, g);
  if (!transpose) return spmv_nodeblock(L, L.nval, L.pvalT, x, b, y, mode, s);
  return spmv_nodeblock(L, L.nvalJT, L.pvalJT, x, b, y, mode, s);
}

stm_status jacobian_defect_colour(Hierarchy& H, int g, int colour, const double* x, const double* b, double* y,
                                  int transpose, cudaStream_t s) {
  Level& L = H.L[g];
  if (transpose) STM_TRY(ensure_transpose(H, g, s));
  const int j0 = L.colour_job_off[colour], nj = L.colour_job_off[colour + 1] - j0;
  ProfScope ps(&H, STM_KCLASS_JACOBIAN_SPMV, s, 8.0 * (double)L.nnz * nj / std::max(L.R, 1) + 24.0 * (double)L.N, g);
  return spmv_nodeblock(L, transpose ? L.nvalJT : L.nval, transpose ? L.pvalJT : L.pvalT, x, b, y, 1, s,
                        L.colour_jobs + j0, nj);
}

// The outer solver is flexible GMRES (Sec. 3): it keeps every preconditioned vector z_j = V(v_j), so
// the V-cycle need not be an exact fixed linear map. With defect_precision = STM_F32 the V-cycle's
// defects run over FP32 copies of J_g: half the bytes and no FP64 arithmetic, with rounding (about
// 1e-7 of |J_g||d|) below that of FP32 or BF16 cell inverses. The Arnoldi products and the true
// residual stay FP64.
stm_status smoother_defect(Hierarchy& H, int g, const double* x, const double* b, double* y, int transpose,
                           cudaStream_t s, bool x32_current) {
  if (H.p.defect_precision != STM_F32) return jacobian_apply(H, g, x, b, y, 1, transpose, s);
  if (transpose) STM_TRY(ensure_transpose(H, g, s));
  return defect_f32(H, g, transpose, x, b, y, s, x32_current);
}

// Dense coarse solve: d = Cinv r (row-major) or d = Cinv^T r.
__global__ void k_dense_gemv(const double* __restrict__ A, long long n, const double* __restrict__ x,
                             double* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long row = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < n; row += warps) {
    const double* a = A + row * n;
    double s = 0.0;
    for (long long j = lane; j < n; j += 32) s += a[j] * x[j];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) y[row] = s;
  }
}
stm_status coarse_apply(Hierarchy& H, const double* r, double* d, int transpose, cudaStream_t s) {
  const long long n = H.N0;
  if (H.coarse_slab) {
    ProfScope ps(&H, STM_KCLASS_COARSE, s, 0.0);
    return coarse_slab_apply(H, r, d, transpose, s);
  }
  ProfScope ps(&H, STM_KCLASS_COARSE, s, 8.0 * (double)n * (double)n + 16.0 * (double)n);
  const int blocks = (int)std::min<long long>((n + 7) / 8, (long long)sms() * 16);
  k_dense_gemv<<<blocks, 256, 0, s>>>(transpose ? H.cinvT : H.cinv, n, r, d);
  note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}

// Algorithm 1 (V-cycle), iterative form of the recursion, zero initial guess on every level.
stm_status vcycle(Hierarchy& H, const double* r_fine, double* d_fine, int transpose, cudaStream_t s) {
  const int G = (int)H.L.size();
  const int nu1 = H.p.nu1, nu2 = H.p.nu2;
  // with FP32 defects, every d a defect reads here was last written by the combine of the additive /
  // overwrite smoother or by the prolongation, which store it rounded to FP32 as well (the coloured
  // smoother's local solves write d directly, so its defects round d themselves)
  const bool f32 = H.p.defect_precision == STM_F32;
  const bool mirrored = f32 && H.p.smoother != STM_VANKA_COLOURED;
  // descend
  const double* r = r_fine;
  for (int g = G - 1; g >= 1; --g) {
    Level& L = H.L[g];
    double* d = (g == G - 1) ? d_fine : L.d;
    STM_CUDA(cudaMemsetAsync(d, 0, sizeof(double) * L.N, s));
    for (int it = 0; it < nu1; ++it) {
      stm_status st = vanka_step(H, g, r, d, transpose, it == 0, s, mirrored && it > 0);
      if (st != STM_OK) return st;
    }
    // t = r - J d, restrict to the next coarser level
    stm_status st = (nu1 > 0) ? smoother_defect(H, g, d, r, L.t, transpose, s, mirrored)
                              : vec_copy(L.t, r, L.N, s);
    if (st != STM_OK) return st;
    Level& Lc = H.L[g - 1];
    {
      ProfScope ps(&H, STM_KCLASS_TRANSFER, s, 0.0, g);
      st = transfer_restrict(L, Lc, L.t, Lc.r, s);
    }
    if (st != STM_OK) return st;
    r = Lc.r;
  }
  // coarse solve
  {
    Level& L0 = H.L[0];
    double* d0 = (G == 1) ? d_fine : L0.d;
    stm_status st = coarse_apply(H, r, d0, transpose, s);
    if (st != STM_OK) return st;
  }
  // ascend
  for (int g = 1; g < G; ++g) {
    Level& L = H.L[g];
    double* d = (g == G - 1) ? d_fine : L.d;
    const double* rg = (g == G - 1) ? r_fine : L.r;
    stm_status st;
    {
      ProfScope ps(&H, STM_KCLASS_TRANSFER, s, 0.0, g);
      st = transfer_prolong_add(L, H.L[g - 1], H.L[g - 1].d, d, s, f32 ? L.x32 : nullptr);
    }
    if (st != STM_OK) return st;
    for (int it = 0; it < nu2; ++it) {
      st = vanka_step(H, g, rg, d, transpose, false, s, mirrored);
      if (st != STM_OK) return st;
    }
  }
  return STM_OK;
}

void clear_graphs(Hierarchy& H) {
  for (auto& kv : H.vgraphs) cudaGraphExecDestroy(kv.second.first);
  H.vgraphs.clear();
}

stm_status vcycle_graph(Hierarchy& H, const double* r, double* d, int transpose, cudaStream_t s) {
  if (H.prof.on || !H.use_graphs) return vcycle(H, r, d, transpose, s);
  const auto key = std::make_tuple(r, d, transpose);
  auto it = H.vgraphs.find(key);
  if (it == H.vgraphs.end()) {
    if (transpose)
      for (int g = 0; g < (int)H.L.size(); ++g) STM_TRY(ensure_transpose(H, g, s));
    if (!H.cap_stream) STM_CUDA(cudaStreamCreateWithFlags(&H.cap_stream, cudaStreamNonBlocking));
    const long long before = g_launches.load();
    STM_CUDA(cudaStreamBeginCapture(H.cap_stream, cudaStreamCaptureModeThreadLocal));
    const stm_status st = vcycle(H, r, d, transpose, H.cap_stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(H.cap_stream, &graph);
    const long long kernels = g_launches.load() - before;
    g_launches.fetch_sub(kernels);  // counted again on every graph launch
    if (st != STM_OK || ce != cudaSuccess || !graph) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      H.use_graphs = false;  // capture not possible here: launch directly from now on
      return vcycle(H, r, d, transpose, s);
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      cudaGetLastError();
      H.use_graphs = false;
      return vcycle(H, r, d, transpose, s);
    }
    it = H.vgraphs.emplace(key, std::make_pair(exec, kernels)).first;
  }
  STM_CUDA(cudaGraphLaunch(it->second.first, s));
  note_launch(it->second.second);
  return STM_OK;
}

// ---------------------------------------------------------------------------------------------
// Krylov helpers
// ---------------------------------------------------------------------------------------------
__global__ void k_fill(double* x, double v, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) x[i] = v;
}
stm_status vec_fill(double* x, double v, long long n, cudaStream_t s) {
  k_fill<<<(int)std::min<long long>((n + 255) / 256, sms() * 8LL), 256, 0, s>>>(x, v, n); note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}
__global__ void k_axpy(double* __restrict__ y, double a, const double* __restrict__ x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] += a * x[i];
}
stm_status vec_axpy(double* y, double a, const double* x, long long n, cudaStream_t s) {
  k_axpy<<<(int)std::max<long long>(1, std::min<long long>((n + 255) / 256, sms() * 8LL)), 256, 0, s>>>(y, a, x, n);
  note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}
stm_status vec_copy(double* y, const double* x, long long n, cudaStream_t s) {
  STM_CUDA(cudaMemcpyAsync(y, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  return STM_OK;
}
// y = x * scale[0] (inv = 0) or y = x / scale[0] (inv = 1)
__global__ void k_scale_to(double* y, const double* x, const double* sc, int inv, long long n) {
  const double f = inv ? 1.0 / sc[0] : sc[0];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) y[i] = x[i] * f;
}
stm_status vec_scale_to(double* y, const double* x, const double* sc, int inv, long long n, cudaStream_t s) {
  k_scale_to<<<(int)std::min<long long>((n + 255) / 256, sms() * 8LL), 256, 0, s>>>(y, x, sc, inv, n); note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}

// part[v][blk] = partial sum of V[v] . w over the block's chunk; then out[v] = sum_blk part (fixed order)
// Four dot products per pass over w (w read once for each group of four); per product the same
// reduction tree as a single one: warp shuffles, then the warp sums in warp order.
__global__ void k_dots_partial(const double* __restrict__ V, int nv, const double* __restrict__ w, long long n,
                               double* __restrict__ part) {
  constexpr int CH = 4;
  __shared__ double red[CH][32];
  for (int v0 = 0; v0 < nv; v0 += CH) {
    const int nc = min(CH, nv - v0);
    double s[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) s[u] = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
      const double wi = w[i];
#pragma unroll
      for (int u = 0; u < CH; ++u)
        if (u < nc) s[u] += V[(long long)(v0 + u) * n + i] * wi;
    }
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      for (int off = 16; off > 0; off >>= 1) s[u] += __shfl_down_sync(0xffffffffu, s[u], off);
      if ((threadIdx.x & 31) == 0) red[u][threadIdx.x >> 5] = s[u];
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      for (int u = 0; u < nc; ++u) {
        double t = threadIdx.x < (blockDim.x >> 5) ? red[u][threadIdx.x] : 0.0;
        for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
        if (threadIdx.x == 0) part[(long long)(v0 + u) * gridDim.x + blockIdx.x] = t;
      }
    }
    __syncthreads();
  }
}
__global__ void k_dots_final(const double* __restrict__ part, int nv, int nblk, double* __restrict__ out) {
  const int v = blockIdx.x;
  if (v >= nv) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[(long long)v * nblk + b];
  __shared__ double red[32];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (threadIdx.x == 0) out[v] = s;
  }
}
stm_status batched_dots(const double* V, int nv, const double* w, long long n, double* out, double* part,
                        int nblk, cudaStream_t s) {
  k_dots_partial<<<nblk, 256, 0, s>>>(V, nv, w, n, part); note_launch();
  k_dots_final<<<nv, 256, 0, s>>>(part, nv, nblk, out); note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}
stm_status vec_norm_sq(const double* x, long long n, double* out, double* part, int nblk, cudaStream_t s) {
  return batched_dots(x, 1, x, n, out, part, nblk, s);
}
// w -= sum_v h[v] V[v]
__global__ void k_batched_update(const double* __restrict__ V, int nv, const double* __restrict__ h,
                                 double* __restrict__ w, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double s = w[i];
    for (int v = 0; v < nv; ++v) s -= h[v] * V[(long long)v * n + i];
    w[i] = s;
  }
}
stm_status batched_update(const double* V, int nv, const double* h, double* w, long long n, cudaStream_t s) {
  k_batched_update<<<(int)std::min<long long>((n + 255) / 256, sms() * 8LL), 256, 0, s>>>(V, nv, h, w, n); note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}
// x += sum_v y[v] Z[v]
__global__ void k_gemv_acc(const double* __restrict__ Z, int nz, const double* __restrict__ y, double* __restrict__ x,
                           long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double s = x[i];
    for (int v = 0; v < nz; ++v) s += y[v] * Z[(long long)v * n + i];
    x[i] = s;
  }
}
stm_status gemv_accumulate(const double* Z, int nz, const double* y, double* x, long long n, cudaStream_t s) {
  k_gemv_acc<<<(int)std::min<long long>((n + 255) / 256, sms() * 8LL), 256, 0, s>>>(Z, nz, y, x, n); note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}
__global__ void k_axpy_small(double* a, const double* b, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) a[i] += b[i];
}
stm_status vec_axpby_dev(double* hacc, const double* h2, int n, cudaStream_t s) {
  k_axpy_small<<<1, 256, 0, s>>>(hacc, h2, n); note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}

}  // namespace stm
