// Multi-right-hand-side path: up to 32 right-hand sides share one hierarchy (one J, one set of
// cell inverses). Multi-vectors are stored interleaved, [N][32] FP64 (column c of DoF i at
// i * 32 + c), so every gather of a DoF fetches its 32 values in one 256-byte line.
//  * SpMM with J_g: the structured pattern of k_spmv_struct, one warp per node (cell) with the
//    32 lanes on the 32 right-hand sides: each value of J is read once for all columns (broadcast).
//  * Vanka local solves Y_T = J_T^{-1} T_T for a 32-column block (a6'' of the hot path): with BF16
//    inverses on the tcgen05 tensor cores (kernels_mrhs_tc.cu: TMA-staged inverses, FP32 accumulators
//    in tensor memory, the gathered block split into T_hi + T_lo BF16 parts so that the only rounding
//    is that of the stored inverse), Y in FP32; FP32 / FP64 inverses (and BF16 ones whose stored
//    columns are not whole 16-byte units) on CUDA cores, Y in FP32 / FP64.
//  * additive combine, transfers, coarse solve and the V-cycle (Algorithm 1) on 32 columns.
#include <cstdint>
#include <type_traits>

#include "internal.h"

namespace stm {

constexpr int NR = 32;  // columns of a multi-vector

static int msms() { return sm_count(); }

// ---------------------------------------------------------------------------------------------
// layout conversion: column-major [nrhs][N] (ld N) <-> interleaved [N][32]
// ---------------------------------------------------------------------------------------------
__global__ void k_to_interleaved(const double* __restrict__ src, double* __restrict__ dst, long long N, int nrhs) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N * NR; e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / NR;
    const int c = (int)(e - i * NR);
    dst[e] = c < nrhs ? src[(long long)c * N + i] : 0.0;
  }
}
__global__ void k_from_interleaved(const double* __restrict__ src, double* __restrict__ dst, long long N, int nrhs) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N * nrhs; e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e / N);
    const long long i = e - (long long)c * N;
    dst[e] = src[i * NR + c];
  }
}
// columns [col0, col0 + ncols) of the interleaved block from a column-major source (others untouched)
__global__ void k_to_interleaved_at(const double* __restrict__ src, double* __restrict__ dst, long long N, int ncols,
                                    int col0) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N * ncols; e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e / N);
    const long long i = e - (long long)c * N;
    dst[i * NR + col0 + c] = src[e];
  }
}
__global__ void k_from_interleaved_at(const double* __restrict__ src, double* __restrict__ dst, long long N, int ncols,
                                      int col0) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N * ncols; e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e / N);
    const long long i = e - (long long)c * N;
    dst[e] = src[i * NR + col0 + c];
  }
}
stm_status multi_columns_in(const double* src, double* dst, long long N, int ncols, int col0, cudaStream_t s) {
  if (ncols <= 0) return STM_OK;
  k_to_interleaved_at<<<(int)std::min<long long>((N * ncols + 255) / 256, msms() * 16LL), 256, 0, s>>>(src, dst, N, ncols,
                                                                                                      col0);
  note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}
stm_status multi_columns_out(const double* src, double* dst, long long N, int ncols, int col0, cudaStream_t s) {
  if (ncols <= 0) return STM_OK;
  k_from_interleaved_at<<<(int)std::min<long long>((N * ncols + 255) / 256, msms() * 16LL), 256, 0, s>>>(src, dst, N,
                                                                                                        ncols, col0);
  note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}

stm_status multi_to_interleaved(const double* src, double* dst, long long N, int nrhs, cudaStream_t s) {
  k_to_interleaved<<<(int)std::min<long long>((N * NR + 255) / 256, msms() * 16LL), 256, 0, s>>>(src, dst, N, nrhs);
  note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}
stm_status multi_from_interleaved(const double* src, double* dst, long long N, int nrhs, cudaStream_t s) {
  k_from_interleaved<<<(int)std::min<long long>((N * nrhs + 255) / 256, msms() * 16LL), 256, 0, s>>>(src, dst, N, nrhs);
  note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}

// ---------------------------------------------------------------------------------------------
// SpMM with J_g (FP64): mode 0: Y = J X; 1: Y = B - J X
// ---------------------------------------------------------------------------------------------
template <int K, int D>
__global__ void __launch_bounds__(256) k_spmm_struct(
    const long long* __restrict__ rowptr, const double* __restrict__ val, const int* __restrict__ nbr_ptr,
    const int* __restrict__ nbr, const int* __restrict__ ncell, const int* __restrict__ node_cells,
    const int* __restrict__ cell_nodes, long long block, int R, int C, int nv, const double* __restrict__ X,
    const double* __restrict__ B, double* __restrict__ Y, int mode, const double* __restrict__ valT, int split,
    uint32_t* __restrict__ T16) {
  constexpr int KD = K * D;
  constexpr int NP = D + 1;
  constexpr int MAXC = 1 << D;
  const int lane = threadIdx.x & 31;
  // lanes (columns) from split on multiply by J^T: its values on the same (symmetric) pattern
  if (lane >= split) val = valT;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long job = warp; job < (long long)R + C; job += nwarps) {
    if (job < R) {
      const int i = (int)job;
      const int p0 = nbr_ptr[i], nn = nbr_ptr[i + 1] - p0, nc = ncell[i];
      long long rp[KD];
      double acc[KD];
#pragma unroll
      for (int a = 0; a < K; ++a)
#pragma unroll
        for (int l = 0; l < D; ++l) {
          rp[a * D + l] = rowptr[a * block + (long long)l * R + i];
          acc[a * D + l] = 0.0;
        }
      for (int j = 0; j < nn; ++j) {
        const long long nj = nbr[p0 + j];
#pragma unroll
        for (int bb = 0; bb < K; ++bb)
#pragma unroll
          for (int m = 0; m < D; ++m) {
            const double xv = X[(bb * block + (long long)m * R + nj) * NR + lane];
#pragma unroll
            for (int a = 0; a < K; ++a) {
              const long long off = (long long)bb * D * nn + (bb > a ? NP * nc : 0) + (long long)m * nn + j;
#pragma unroll
              for (int l = 0; l < D; ++l) acc[a * D + l] += __ldg(val + rp[a * D + l] + off) * xv;
            }
          }
      }
      for (int t = 0; t < NP * nc; ++t) {
        const int ci = t / NP, q = t - ci * NP;
        const long long pc = (long long)D * R + (long long)node_cells[(long long)i * MAXC + ci] * NP + q;
#pragma unroll
        for (int a = 0; a < K; ++a) {
          const double xp = X[(a * block + pc) * NR + lane];
#pragma unroll
          for (int l = 0; l < D; ++l) acc[a * D + l] += __ldg(val + rp[a * D + l] + (long long)(a + 1) * D * nn + t) * xp;
        }
      }
#pragma unroll
      for (int a = 0; a < K; ++a)
#pragma unroll
        for (int l = 0; l < D; ++l) {
          const long long o = (a * block + (long long)l * R + i) * NR + lane;
          const double yv = mode == 1 ? B[o] - acc[a * D + l] : acc[a * D + l];
          Y[o] = yv;
          if (T16) {
            uint32_t h, lo;
            bf16_split_rn(yv, h, lo);
            T16[o] = (lo << 16) | h;
          }
        }
    } else {
      const long long c = job - R;
      long long rp[K * NP];
      double acc[K * NP];
#pragma unroll
      for (int a = 0; a < K; ++a)
#pragma unroll
        for (int q = 0; q < NP; ++q) {
          rp[a * NP + q] = rowptr[a * block + (long long)D * R + c * NP + q];
          acc[a * NP + q] = 0.0;
        }
      for (int t = 0; t < D * nv; ++t) {
        const int m = t / nv, jj = t - m * nv;
        const long long node = cell_nodes[c * nv + jj];
#pragma unroll
        for (int a = 0; a < K; ++a) {
          const double xa = X[(a * block + (long long)m * R + node) * NR + lane];
#pragma unroll
          for (int q = 0; q < NP; ++q) acc[a * NP + q] += __ldg(val + rp[a * NP + q] + t) * xa;
        }
      }
#pragma unroll
      for (int a = 0; a < K; ++a)
#pragma unroll
        for (int q = 0; q < NP; ++q) {
          const long long o = (a * block + (long long)D * R + c * NP + q) * NR + lane;
          const double yv = mode == 1 ? B[o] - acc[a * NP + q] : acc[a * NP + q];
          Y[o] = yv;
          if (T16) {
            uint32_t h, lo;
            bf16_split_rn(yv, h, lo);
            T16[o] = (lo << 16) | h;
          }
        }
    }
  }
}

stm_status spmm_structured(const Level& L, const double* X, const double* B, double* Y, int mode, cudaStream_t s,
                           int split, uint32_t* T16) {
  if (split < NR && !L.valT) {
    set_error("multi-RHS SpMM: the values of J^T are not built");
    return STM_ERR_STATE;
  }
  const long long jobs = (long long)L.R + L.C;
  const int blocks = (int)std::min<long long>((jobs * 32 + 255) / 256, (long long)msms() * 8);
  const int key = L.dim * 10 + L.K;
#define SPMM(K, D) \
  k_spmm_struct<K, D><<<blocks, 256, 0, s>>>(L.rowptr, L.val, L.nbr_ptr, L.nbr, L.ncell, L.node_cells, L.cell_nodes, \
                                             L.block, L.R, L.C, L.nv, X, B, Y, mode, L.valT, split, T16)
  switch (key) {
    case 21: SPMM(1, 2); break;
    case 22: SPMM(2, 2); break;
    case 23: SPMM(3, 2); break;
    case 31: SPMM(1, 3); break;
    case 32: SPMM(2, 3); break;
    case 33: SPMM(3, 3); break;
    default:
      set_error("multi-RHS SpMM: unsupported (dim, k)");
      return STM_ERR_INVALID_ARG;
  }
#undef SPMM
  note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}

// CSR (transfers) on 32 columns: warp per row, lane = column. mode 0: Y = A X; 2: Y += A X.
__global__ void __launch_bounds__(256) k_csr_multi(const long long* __restrict__ rowptr, const int* __restrict__ col,
                                                   const double* __restrict__ val, long long nrows,
                                                   const double* __restrict__ X, double* __restrict__ Y, int mode) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long row = warp; row < nrows; row += nwarps) {
    double s = 0.0;
    for (long long e = rowptr[row]; e < rowptr[row + 1]; ++e) s += __ldg(val + e) * X[(long long)__ldg(col + e) * NR + lane];
    if (mode == 2) Y[row * NR + lane] += s;
    else Y[row * NR + lane] = s;
  }
}
stm_status csr_multi(const long long* rowptr, const int* col, const double* val, long long nrows, const double* X,
                     double* Y, int mode, cudaStream_t s) {
  const int blocks = (int)std::min<long long>((nrows * 32 + 255) / 256, (long long)msms() * 8);
  k_csr_multi<<<blocks, 256, 0, s>>>(rowptr, col, val, nrows, X, Y, mode);
  note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}

// Packed BF16 hi + lo parts (lo << 16 | hi) of an interleaved multi-vector, for the tensor-core smoother
__global__ void k_pack_bf16_split(const double* __restrict__ X, uint32_t* __restrict__ P, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    uint32_t h, lo;
    bf16_split_rn(X[e], h, lo);
    P[e] = (lo << 16) | h;
  }
}

// ---------------------------------------------------------------------------------------------
// Vanka local solves on 32 columns
// ---------------------------------------------------------------------------------------------
// CUDA-core variant (FP32 / FP64 inverses; BF16 ones whose columns are not whole 16-byte units):
// lane = column, warps over rows, Inv read by broadcast; FP64 accumulation and Y for FP64 inverses,
// FP32 otherwise.
__device__ __forceinline__ float inv_to_acc(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float inv_to_acc(float v) { return v; }
__device__ __forceinline__ double inv_to_acc(double v) { return v; }

// Lanes from split on apply the transposed inverse (adjoint columns).
template <typename S, typename A>
__global__ void __launch_bounds__(256) k_vanka_mrhs_cc(const S* __restrict__ inv, const int* __restrict__ idx,
                                                       const double* __restrict__ T, A* __restrict__ Yout,
                                                       int ncells, int n, int ld, int split) {
  extern __shared__ __align__(16) unsigned char smc[];
  A* Ts = reinterpret_cast<A*>(smc);  // [n][32]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int c = blockIdx.x; c < ncells; c += gridDim.x) {
    __syncthreads();
    const int* ic = idx + (long long)c * n;
    for (int e = threadIdx.x; e < n * NR; e += blockDim.x) {
      const int k = e / NR, col = e - k * NR;
      Ts[e] = (A)T[(long long)ic[k] * NR + col];
    }
    __syncthreads();
    const S* M = inv + (size_t)c * n * ld;
    const bool adj = lane >= split;
    for (int i = warp; i < n; i += nwarps) {
      // forward: (J_T^{-1})_{ij} = M[j*ld + i]; adjoint: (J_T^{-T})_{ij} = M[i*ld + j]
      const S* mr = adj ? M + (size_t)i * ld : M + i;
      const size_t st = adj ? 1 : (size_t)ld;
      A s = 0;
      for (int j = 0; j < n; ++j) s += (A)inv_to_acc(mr[(size_t)j * st]) * Ts[j * NR + lane];
      Yout[((long long)c * n + i) * NR + lane] = s;
    }
  }
}

// d[i][c] += omega / m_i * sum over the owners of i of Y[pos][c]  (Y in FP32 or FP64)
template <typename A>
__global__ void k_vanka_gather_multi(double* __restrict__ d, const A* __restrict__ Y, const int* __restrict__ own_ptr,
                                     const int* __restrict__ own_pos, const double* __restrict__ wmult, long long N,
                                     double omega) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N * NR; e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / NR;
    const int col = (int)(e - i * NR);
    double s = 0.0;
    for (int p = own_ptr[i]; p < own_ptr[i + 1]; ++p) s += (double)Y[(long long)own_pos[p] * NR + col];
    d[e] += omega * wmult[i] * s;
  }
}

stm_status ensure_multi(Hierarchy& H) {
  for (Level& L : H.L) {
    if (L.mY && L.md && (L.mt16 || H.p.inv_precision != STM_BF16)) continue;
    if (!L.md) {
      STM_CUDA(cudaMalloc(&L.md, sizeof(double) * (size_t)L.N * NR));
      STM_CUDA(cudaMalloc(&L.mr, sizeof(double) * (size_t)L.N * NR));
      STM_CUDA(cudaMalloc(&L.mt, sizeof(double) * (size_t)L.N * NR));
    }
    if (!L.mY) STM_CUDA(cudaMalloc(&L.mY, sizeof(double) * (size_t)L.C * L.n * NR));
    if (!L.mt16 && H.p.inv_precision == STM_BF16) STM_CUDA(cudaMalloc(&L.mt16, sizeof(uint32_t) * (size_t)L.N * NR));
  }
  return STM_OK;
}

stm_status vanka_step_multi(Hierarchy& H, int g, const double* R, double* Dm, bool d_is_zero, cudaStream_t s,
                            int split) {
  Level& L = H.L[g];
  const double* T = R;
  if (split < NR) STM_TRY(ensure_transpose(H, g, s));
  const int prec = H.p.inv_precision;
  const InvLayout lay = inv_layout(L.n, prec);
  const bool fused = split == 16;
  if (split != NR && !fused) {
    set_error("multi-RHS smoothing: adjoint columns start at column 16");
    return STM_ERR_INVALID_ARG;
  }
  const bool tc = prec == STM_BF16 && (fused ? mrhs_tc_fused_supported(L.n, lay.ld) : mrhs_tc_supported(L.n, lay.ld));
  // the tensor-core products read the residual block as packed BF16 hi + lo parts: the defect product
  // writes them as it writes the block; a residual taken as it is gets a packing pass
  if (!d_is_zero) {
    ProfScope ps(&H, STM_KCLASS_JACOBIAN_SPMV, s, 8.0 * (double)L.nnz + 24.0 * NR * (double)L.N, g);
    STM_TRY(spmm_structured(L, Dm, R, L.mt, 1, s, split, tc ? L.mt16 : nullptr));
    T = L.mt;
  }
  const bool y64 = prec == STM_F64;
  {
    // algorithmic bytes: the stored inverses, the index map, the 32 gathered FP64 columns of every
    // local DoF and the 32 written columns of Y (FP64 with FP64 inverses, FP32 otherwise)
    ProfScope ps(&H, STM_KCLASS_VANKA_LOCAL, s,
                 (double)L.C * ((double)L.n * L.n * (prec == STM_F64 ? 8 : prec == STM_F32 ? 4 : 2) + 4.0 * L.n +
                                (8.0 + (y64 ? 8.0 : 4.0)) * NR * L.n),
                 g);
    if (tc) {
      if (d_is_zero) {
        const long long ne = L.N * NR;
        k_pack_bf16_split<<<(int)std::min<long long>((ne + 255) / 256, msms() * 16LL), 256, 0, s>>>(R, L.mt16, ne);
        note_launch();
        STM_CUDA(cudaGetLastError());
      }
      STM_TRY(mrhs_tc_apply(L, lay.ld, L.mt16, reinterpret_cast<float*>(L.mY), H.dkerr, s, fused));
    } else {
      const int blocks = std::min(L.C, msms() * 8);
#define MRHS_CC(S_, A_)                                                                                          \
  do {                                                                                                          \
    const size_t smem = sizeof(A_) * (size_t)L.n * NR;                                                          \
    STM_CUDA(cudaFuncSetAttribute(k_vanka_mrhs_cc<S_, A_>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
    k_vanka_mrhs_cc<S_, A_><<<blocks, 256, smem, s>>>((const S_*)L.inv, L.idx, T, reinterpret_cast<A_*>(L.mY), L.C, \
                                                      L.n, lay.ld, split);                                      \
  } while (0)
      if (prec == STM_F64) MRHS_CC(double, double);
      else if (prec == STM_F32) MRHS_CC(float, float);
      else MRHS_CC(__nv_bfloat16, float);
#undef MRHS_CC
      note_launch();
      STM_CUDA(cudaGetLastError());
    }
  }
  ProfScope ps(&H, STM_KCLASS_VANKA_COMBINE, s, 0.0, g);
  const int blocks = (int)std::min<long long>((L.N * NR + 255) / 256, msms() * 16LL);
  if (y64)
    k_vanka_gather_multi<double><<<blocks, 256, 0, s>>>(Dm, L.mY, L.own_ptr, L.own_pos, L.wmult, L.N, H.p.omega);
  else
    k_vanka_gather_multi<float><<<blocks, 256, 0, s>>>(Dm, reinterpret_cast<const float*>(L.mY), L.own_ptr, L.own_pos,
                                                       L.wmult, L.N, H.p.omega);
  note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}

// Coarse solve on 32 columns: D = Cinv R (FP64), warp per row of Cinv, lane = column.
__global__ void __launch_bounds__(256) k_dense_gemm_multi(const double* __restrict__ A, long long n,
                                                          const double* __restrict__ R, double* __restrict__ Dm) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long row = warp; row < n; row += nwarps) {
    const double* a = A + row * n;
    double s = 0.0;
    for (long long k = 0; k < n; ++k) s += __ldg(a + k) * R[k * NR + lane];
    Dm[row * NR + lane] = s;
  }
}

stm_status vcycle_multi(Hierarchy& H, const double* R_fine, double* D_fine, cudaStream_t s) {
  const int G = (int)H.L.size();
  const double* r = R_fine;
  for (int g = G - 1; g >= 1; --g) {
    Level& L = H.L[g];
    double* d = (g == G - 1) ? D_fine : L.md;
    STM_CUDA(cudaMemsetAsync(d, 0, sizeof(double) * (size_t)L.N * NR, s));
    for (int it = 0; it < H.p.nu1; ++it) STM_TRY(vanka_step_multi(H, g, r, d, it == 0, s));
    if (H.p.nu1 > 0) {
      ProfScope ps(&H, STM_KCLASS_JACOBIAN_SPMV, s, 8.0 * (double)L.nnz + 24.0 * NR * (double)L.N, g);
      STM_TRY(spmm_structured(L, d, r, L.mt, 1, s));
    } else {
      STM_CUDA(cudaMemcpyAsync(L.mt, r, sizeof(double) * (size_t)L.N * NR, cudaMemcpyDeviceToDevice, s));
    }
    Level& Lc = H.L[g - 1];
    {
      ProfScope ps(&H, STM_KCLASS_TRANSFER, s, 0.0);
      STM_TRY(csr_multi(L.Rt_rowptr, L.Rt_col, L.Rt_val, Lc.N, L.mt, Lc.mr, 0, s));
    }
    r = Lc.mr;
  }
  {
    ProfScope ps(&H, STM_KCLASS_COARSE, s, H.coarse_slab ? 0.0 : 8.0 * (double)H.N0 * H.N0);
    if (H.coarse_slab) {
      STM_TRY(coarse_slab_apply_multi(H, r, H.L[0].md, s));
    } else {
      const int blocks = (int)std::min<long long>((H.N0 * 32 + 255) / 256, (long long)msms() * 8);
      k_dense_gemm_multi<<<blocks, 256, 0, s>>>(H.cinv, H.N0, r, H.L[0].md);
      note_launch();
      STM_CUDA(cudaGetLastError());
    }
  }
  for (int g = 1; g < G; ++g) {
    Level& L = H.L[g];
    double* d = (g == G - 1) ? D_fine : L.md;
    const double* rg = (g == G - 1) ? R_fine : L.mr;
    {
      ProfScope ps(&H, STM_KCLASS_TRANSFER, s, 0.0);
      STM_TRY(csr_multi(L.P_rowptr, L.P_col, L.P_val, L.N, H.L[g - 1].md, d, 2, s));
    }
    for (int it = 0; it < H.p.nu2; ++it) STM_TRY(vanka_step_multi(H, g, rg, d, false, s));
  }
  return STM_OK;
}

// ---------------------------------------------------------------------------------------------
// Krylov building blocks on 32 columns (column-wise dot products, updates, scaling)
// ---------------------------------------------------------------------------------------------
// part[v][blk][c] = partial of sum_i V_v[i][c] w[i][c]; threads: lane = column, warps stride rows
__global__ void __launch_bounds__(256) k_mdots_partial(const double* __restrict__ V, int nv, const double* __restrict__ w,
                                                       long long n, double* __restrict__ part) {
  __shared__ double red[8][NR];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int v = 0; v < nv; ++v) {
    const double* a = V + (size_t)v * n * NR;
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * nw + wid; i < n; i += (long long)gridDim.x * nw)
      s += a[i * NR + lane] * w[i * NR + lane];
    red[wid][lane] = s;
    __syncthreads();
    if (wid == 0) {
      double t = 0.0;
      for (int k = 0; k < nw; ++k) t += red[k][lane];
      part[((size_t)v * gridDim.x + blockIdx.x) * NR + lane] = t;
    }
    __syncthreads();
  }
}
__global__ void k_mdots_final(const double* __restrict__ part, int nv, int nblk, double* __restrict__ out) {
  const int v = blockIdx.x, lane = threadIdx.x;
  if (v >= nv || lane >= NR) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[((size_t)v * nblk + b) * NR + lane];
  out[v * NR + lane] = s;
}
stm_status mdots(const double* V, int nv, const double* w, long long n, double* out, double* part, int nblk,
                 cudaStream_t s) {
  k_mdots_partial<<<nblk, 256, 0, s>>>(V, nv, w, n, part);
  note_launch();
  k_mdots_final<<<nv, 32, 0, s>>>(part, nv, nblk, out);
  note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}
// w[i][c] -= sum_v h[v][c] V_v[i][c]   (sign = -1)   or   x[i][c] += sum_v h[v][c] Z_v[i][c] (sign = +1)
__global__ void k_mupdate(const double* __restrict__ V, int nv, const double* __restrict__ h, double* __restrict__ w,
                          long long n, double sign) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n * NR; e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e % NR);
    double s = w[e];
    for (int v = 0; v < nv; ++v) s += sign * h[v * NR + c] * V[(size_t)v * n * NR + e];
    w[e] = s;
  }
}
stm_status mupdate(const double* V, int nv, const double* h, double* w, long long n, double sign, cudaStream_t s) {
  k_mupdate<<<(int)std::min<long long>((n * NR + 255) / 256, msms() * 16LL), 256, 0, s>>>(V, nv, h, w, n, sign);
  note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}
// y[i][c] = x[i][c] * f[c]
__global__ void k_mscale(double* __restrict__ y, const double* __restrict__ x, const double* __restrict__ f, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n * NR; e += (long long)gridDim.x * blockDim.x)
    y[e] = x[e] * f[e % NR];
}
stm_status mscale(double* y, const double* x, const double* f, long long n, cudaStream_t s) {
  k_mscale<<<(int)std::min<long long>((n * NR + 255) / 256, msms() * 16LL), 256, 0, s>>>(y, x, f, n);
  note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}
__global__ void k_madd_small(double* a, const double* b, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) a[i] += b[i];
}
stm_status madd_small(double* a, const double* b, int n, cudaStream_t s) {
  k_madd_small<<<1, 256, 0, s>>>(a, b, n);
  note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}

}  // namespace stm
