// Cell inverses and the coarse direct solver (FP64 arithmetic).
//
// Sec. 4.3: for every cell T of a level the inverse of the local Jacobian J_T is precomputed after
// each Jacobian update. J_T holds the rows and columns of the ASSEMBLED global matrix on the
// cell's DoFs (Sec. 4.4), gathered here straight from the CSR values through the structured
// position map. Inversion: Gauss-Jordan elimination with partial pivoting (largest |pivot| in the
// column, lowest row on ties) in shared memory, one CTA per cell; the result is stored
// column-major per cell in the requested precision (FP64 / FP32 / BF16).
#include <cfloat>

#include "internal.h"

namespace stm {

template <typename S> __device__ __forceinline__ S to_store(double v);
template <> __device__ __forceinline__ double to_store<double>(double v) { return v; }
template <> __device__ __forceinline__ float to_store<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ __nv_bfloat16 to_store<__nv_bfloat16>(double v) {
  return __float2bfloat16_rn((float)v);
}

// Position in the CSR values of J_g of the entry (local row al, local col be) of cell c.
__device__ __forceinline__ long long entry_pos(int c, int al, int be, const int* __restrict__ idx,
                                               const int* __restrict__ cell_nodes,
                                               const unsigned char* __restrict__ rank,
                                               const unsigned char* __restrict__ cellrank,
                                               const int* __restrict__ nn, const int* __restrict__ ncell,
                                               const long long* __restrict__ rowptr, int d, int nv,
                                               int np, int nt, int n) {
  const int a = al / nt, ra = al - a * nt;
  const int b = be / nt, rb = be - b * nt;
  const long long row = idx[(long long)c * n + al];
  const int dnv = d * nv;
  if (ra < dnv) {
    const int i = ra % nv;
    const int node = cell_nodes[(long long)c * nv + i];
    const int nni = nn[node];
    if (rb < dnv) {
      const int m = rb / nv, j = rb - m * nv;
      return rowptr[row] + (long long)b * d * nni + (b > a ? np * ncell[node] : 0) + (long long)m * nni +
             rank[((long long)c * nv + i) * nv + j];
    }
    if (b != a) return -1;
    const int q = rb - dnv;
    return rowptr[row] + (long long)a * d * nni + (long long)d * nni + (long long)cellrank[(long long)c * nv + i] * np + q;
  }
  if (rb >= dnv || b != a) return -1;
  return rowptr[row] + rb;  // pressure row: columns (a, m, j) in order m * nv + j
}

// Gauss-Jordan inversion of the n x n row-major matrix A in shared memory (in place).
// Returns false (in every thread) if a pivot is zero or not finite.
__device__ bool gj_invert_smem(double* A, short* perm, int n, volatile int* s_piv, volatile int* s_bad) {
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int k = 0; k < n; ++k) {
    if (tid < 32) {
      double best = -1.0;
      int bi = n;
      for (int i = k + tid; i < n; i += 32) {
        const double v = fabs(A[i * n + k]);
        if (v > best) { best = v; bi = i; }  // strict: the lowest row of this lane wins ties
      }
      for (int off = 16; off > 0; off >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (tid == 0) {
        *s_piv = bi;
        if (!(best > 0.0) || !(best <= DBL_MAX)) *s_bad = 1;
        perm[k] = (short)bi;
      }
    }
    __syncthreads();
    if (*s_bad) return false;
    const int p = *s_piv;
    if (p != k)
      for (int j = tid; j < n; j += nth) {
        const double t = A[k * n + j];
        A[k * n + j] = A[p * n + j];
        A[p * n + j] = t;
      }
    __syncthreads();
    const double pinv = 1.0 / A[k * n + k];
    for (int j = tid; j < n; j += nth)
      if (j != k) A[k * n + j] *= pinv;
    __syncthreads();
    for (int e = tid; e < n * n; e += nth) {
      const int i = e / n, j = e - i * n;
      if (i != k && j != k) A[e] -= A[i * n + k] * A[k * n + j];
    }
    __syncthreads();
    for (int i = tid; i < n; i += nth) A[i * n + k] = (i == k) ? pinv : -A[i * n + k] * pinv;
    __syncthreads();
  }
  // undo the row interchanges as column interchanges, last first
  for (int k = n - 1; k >= 0; --k) {
    const int p = perm[k];
    if (p != k)
      for (int i = tid; i < n; i += nth) {
        const double t = A[i * n + k];
        A[i * n + k] = A[i * n + p];
        A[i * n + p] = t;
      }
    __syncthreads();
  }
  return true;
}

template <typename S>
__global__ void __launch_bounds__(512) k_cell_inverse(
    const int* __restrict__ idx, const int* __restrict__ cell_nodes, const unsigned char* __restrict__ rank,
    const unsigned char* __restrict__ cellrank, const int* __restrict__ nn, const int* __restrict__ ncell,
    const long long* __restrict__ rowptr, const double* __restrict__ val, S* __restrict__ inv, int C, int d,
    int nv, int np, int nt, int n, int ld, int* flag, long long* bad) {
  extern __shared__ double sm[];
  double* A = sm;
  short* perm = reinterpret_cast<short*>(A + (size_t)n * n);
  __shared__ int s_piv, s_bad;
  for (int c = blockIdx.x; c < C; c += gridDim.x) {
    if (threadIdx.x == 0) s_bad = 0;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int al = e / n, be = e - al * n;
      const long long pos = entry_pos(c, al, be, idx, cell_nodes, rank, cellrank, nn, ncell, rowptr, d, nv, np, nt, n);
      A[e] = pos >= 0 ? val[pos] : 0.0;
    }
    __syncthreads();
    const bool ok = gj_invert_smem(A, perm, n, &s_piv, &s_bad);
    if (!ok) {
      if (threadIdx.x == 0 && atomicCAS(flag, 0, 1) == 0) *bad = c;
      __syncthreads();
      continue;
    }
    S* out = inv + (size_t)c * n * ld;
    for (int e = threadIdx.x; e < n * ld; e += blockDim.x) {
      const int j = e / ld, i = e - j * ld;  // column-major store: element (i, j) at j * ld + i
      out[e] = to_store<S>(i < n ? A[i * n + j] : 0.0);
    }
    __syncthreads();
  }
}

static size_t storage_bytes(int prec) { return prec == STM_F64 ? 8 : prec == STM_F32 ? 4 : 2; }

stm_status factor_level(Hierarchy& H, int g, cudaStream_t s) {
  Level& L = H.L[g];
  const size_t nn2 = (size_t)L.n * L.n;
  const InvLayout lay = inv_layout(L.n, H.p.inv_precision);
  if (!L.inv) STM_CUDA(cudaMalloc(&L.inv, storage_bytes(H.p.inv_precision) * (size_t)L.n * lay.ld * L.C));
  const size_t smem = sizeof(double) * nn2 + sizeof(short) * L.n + 16;
  int dev = 0, maxsm = 0;
  STM_CUDA(cudaGetDevice(&dev));
  STM_CUDA(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (smem + 64 > (size_t)maxsm) {
    set_error("factor_cells: cell matrix does not fit in shared memory");
    return STM_ERR_INVALID_ARG;
  }
  const int threads = L.n >= 128 ? 512 : 256;
  int sms = 0;
  STM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = std::min(L.C, sms * 16);
#define LAUNCH_INV(T)                                                                                  \
  do {                                                                                                \
    STM_CUDA(cudaFuncSetAttribute(k_cell_inverse<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
    k_cell_inverse<T><<<blocks, threads, smem, s>>>(L.idx, L.cell_nodes, L.rank, L.cellrank, L.nn, L.ncell,  \
                                                    L.rowptr, L.val, (T*)L.inv, L.C, L.dim, L.nv, L.np,     \
                                                    L.nt, L.n, lay.ld, H.dflag, H.dbad); note_launch();                            \
  } while (0)
  if (H.p.inv_precision == STM_F64) LAUNCH_INV(double);
  else if (H.p.inv_precision == STM_F32) LAUNCH_INV(float);
  else LAUNCH_INV(__nv_bfloat16);
#undef LAUNCH_INV
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}

// ---------------------------------------------------------------------------------------------
// Coarse level: explicit FP64 inverse of J_0 by Gauss-Jordan with partial pivoting in global memory
// ---------------------------------------------------------------------------------------------
__global__ void k_densify(const long long* __restrict__ rowptr, const int* __restrict__ col,
                          const double* __restrict__ val, double* __restrict__ A, long long n) {
  for (long long r = blockIdx.x; r < n; r += gridDim.x)
    for (long long e = rowptr[r] + threadIdx.x; e < rowptr[r + 1]; e += blockDim.x) A[r * n + col[e]] = val[e];
}

// scal[0] = 1/pivot, scal[1] = old A[k][k]; piv[k] = pivot row
__global__ void k_gj_pivot(double* A, long long n, int k, int* piv, double* scal, int* flag) {
  __shared__ double sb[32];
  __shared__ int si[32];
  double best = -1.0;
  int bi = (int)n;
  for (long long i = k + threadIdx.x; i < n; i += blockDim.x) {
    const double v = fabs(A[i * n + k]);
    if (v > best) { best = v; bi = (int)i; }
  }
  for (int off = 16; off > 0; off >>= 1) {
    const double ob = __shfl_down_sync(0xffffffffu, best, off);
    const int oi = __shfl_down_sync(0xffffffffu, bi, off);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  if ((threadIdx.x & 31) == 0) { sb[threadIdx.x / 32] = best; si[threadIdx.x / 32] = bi; }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int nw = blockDim.x / 32;
    best = threadIdx.x < nw ? sb[threadIdx.x] : -1.0;
    bi = threadIdx.x < nw ? si[threadIdx.x] : (int)n;
    for (int off = 16; off > 0; off >>= 1) {
      const double ob = __shfl_down_sync(0xffffffffu, best, off);
      const int oi = __shfl_down_sync(0xffffffffu, bi, off);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (threadIdx.x == 0) {
      if (!(best > 0.0) || !(best <= DBL_MAX)) {
        *flag = 1;
        bi = k;
        scal[0] = 0.0;
      } else {
        scal[0] = 1.0 / A[(long long)bi * n + k];
      }
      piv[k] = bi;
      scal[1] = A[(long long)k * n + k];
    }
  }
}

// rows k <-> p for all columns j != k, then scale row k
__global__ void k_gj_swap_scale(double* A, long long n, int k, const int* piv, const double* scal) {
  const int p = piv[k];
  const double pinv = scal[0];
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
    if (j == k) continue;
    const double t = A[(long long)k * n + j];
    const double u = A[(long long)p * n + j];
    A[(long long)p * n + j] = t;
    A[(long long)k * n + j] = u * pinv;
  }
}

// A[i][j] -= A[i][k] A[k][j] for i != k, j != k; column k is still unswapped: row p holds old row k
__global__ void k_gj_update(double* A, long long n, int k, const int* piv, const double* scal) {
  const int p = piv[k];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n * n; e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / n, j = e - i * n;
    if (i == k || j == k) continue;
    const double aik = (i == p) ? scal[1] : A[i * n + k];
    A[e] -= aik * A[(long long)k * n + j];
  }
}

__global__ void k_gj_column(double* A, long long n, int k, const int* piv, const double* scal) {
  const int p = piv[k];
  const double pinv = scal[0];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if (i == k) {
      A[(long long)k * n + k] = pinv;
    } else {
      const double aik = (i == p) ? scal[1] : A[i * n + k];
      A[i * n + k] = -aik * pinv;
    }
  }
}

__global__ void k_gj_colswap(double* A, long long n, int k, const int* piv) {
  const int p = piv[k];
  if (p == k) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double t = A[i * n + k];
    A[i * n + k] = A[i * n + p];
    A[i * n + p] = t;
  }
}

stm_status factor_coarse(Hierarchy& H, cudaStream_t s) {
  Level& L = H.L[0];
  const long long n = L.N;
  H.N0 = n;
  if (!H.cinv) STM_CUDA(cudaMalloc(&H.cinv, sizeof(double) * n * n));
  STM_CUDA(cudaMemsetAsync(H.cinv, 0, sizeof(double) * n * n, s));
  k_densify<<<(int)std::min<long long>(n, 152 * 32), 128, 0, s>>>(L.rowptr, L.colidx, L.val, H.cinv, n); note_launch();
  STM_CUDA(cudaGetLastError());
  int* piv = nullptr;
  double* scal = nullptr;
  STM_CUDA(cudaMalloc(&piv, sizeof(int) * n));
  STM_CUDA(cudaMalloc(&scal, sizeof(double) * 2));
  const int vb = (int)std::min<long long>((n + 255) / 256, 152 * 8);
  const int mb = (int)std::min<long long>((n * n + 255) / 256, 152 * 32);
  for (int k = 0; k < n; ++k) {
    k_gj_pivot<<<1, 1024, 0, s>>>(H.cinv, n, k, piv, scal, H.dflag + 1); note_launch();
    k_gj_swap_scale<<<vb, 256, 0, s>>>(H.cinv, n, k, piv, scal); note_launch();
    k_gj_update<<<mb, 256, 0, s>>>(H.cinv, n, k, piv, scal); note_launch();
    k_gj_column<<<vb, 256, 0, s>>>(H.cinv, n, k, piv, scal); note_launch();
  }
  for (int k = (int)n - 1; k >= 0; --k) k_gj_colswap<<<vb, 256, 0, s>>>(H.cinv, n, k, piv); note_launch();
  STM_CUDA(cudaGetLastError());
  STM_CUDA(cudaStreamSynchronize(s));
  cudaFree(piv);
  cudaFree(scal);
  return STM_OK;
}

}  // namespace stm
