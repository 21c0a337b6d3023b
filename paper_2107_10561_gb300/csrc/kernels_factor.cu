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
  return __ushort_as_bfloat16((unsigned short)bf16_bits_rn(v));  // one rounding, straight from FP64
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

// ---------------------------------------------------------------------------------------------
// Coarse direct solver (Algorithm 1, level 1): the explicit inverse of J_0 from a block LU over
// x-slabs. Velocity DoFs go to the slab of their node's lattice plane (planes 2b, 2b+1 -> slab b,
// the last plane with the last slab), the pressure of cell i to slab i+1 (the last cell's to the
// last slab). A Q2 cell spans the planes 2i..2i+2, so J_0 is block tridiagonal in this order, and
// every slab's pressure is eliminated after the velocities of the cell that carries it, which keeps
// the Schur complements regular (with the pressure of cell b in slab b, S_0 is singular: its
// pressure sees only velocities whose neighbours across the slab face were cut away). Block LU
// without pivoting across slabs, Gauss-Jordan with partial pivoting inside each Schur complement:
//   S_0 = A_00,  S_b = A_bb - A_{b,b-1} W_{b-1},  W_b = S_b^{-1} A_{b,b+1},  G_b = S_b^{-1} A_{b,b-1};
// then the inverse, L^{-1} forward (Z_bb = S_b^{-1}, Z_bj = -G_b Z_{b-1,j}) and U^{-1} backward
// (X_b = Z_b - W_b X_{b+1}), and finally the slab permutation is undone.
// ---------------------------------------------------------------------------------------------

// C = beta C + alpha A B, row-major, FP64. 64x64 tile per 256-thread CTA, 4x4 outputs per thread.
__global__ void __launch_bounds__(256) k_dgemm_rm(int m, int n, int k, double alpha, const double* __restrict__ A,
                                                  long long lda, const double* __restrict__ B, long long ldb,
                                                  double beta, double* __restrict__ C, long long ldc) {
  __shared__ double As[16][64 + 1];
  __shared__ double Bs[16][64];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int r0 = blockIdx.y * 64, c0 = blockIdx.x * 64;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int k0 = 0; k0 < k; k0 += 16) {
    for (int e = threadIdx.x; e < 64 * 16; e += 256) {
      const int rr = e / 16, kk = e - rr * 16;
      const int gr = r0 + rr, gk = k0 + kk;
      As[kk][rr] = (gr < m && gk < k) ? A[(long long)gr * lda + gk] : 0.0;
      const int kb = e / 64, cc = e - kb * 64;
      const int gkb = k0 + kb, gc = c0 + cc;
      Bs[kb][cc] = (gkb < k && gc < n) ? B[(long long)gkb * ldb + gc] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = As[kk][ty + 16 * q];
        b[q] = Bs[kk][tx + 16 * q];
      }
#pragma unroll
      for (int qa = 0; qa < 4; ++qa)
#pragma unroll
        for (int qb = 0; qb < 4; ++qb) acc[qa][qb] += a[qa] * b[qb];
    }
    __syncthreads();
  }
#pragma unroll
  for (int qa = 0; qa < 4; ++qa)
#pragma unroll
    for (int qb = 0; qb < 4; ++qb) {
      const int gr = r0 + ty + 16 * qa, gc = c0 + tx + 16 * qb;
      if (gr < m && gc < n) {
        double* c = C + (long long)gr * ldc + gc;
        *c = (beta == 0.0 ? 0.0 : beta * *c) + alpha * acc[qa][qb];
      }
    }
}

static void dgemm(int m, int n, int k, double alpha, const double* A, long long lda, const double* B, long long ldb,
                  double beta, double* C, long long ldc, cudaStream_t s) {
  if (m <= 0 || n <= 0) return;
  dim3 grid((n + 63) / 64, (m + 63) / 64);
  k_dgemm_rm<<<grid, 256, 0, s>>>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
  note_launch();
}

// Dense slab blocks from the CSR of J_0: row r of slab b (permuted index pr = iperm[r]) scatters its
// entries into D_b (same slab), Lo_b (slab b-1) or Up_b (slab b+1); anything else flags an error.
__global__ void k_slab_blocks(const long long* __restrict__ rowptr, const int* __restrict__ col,
                              const double* __restrict__ val, long long n, const int* __restrict__ iperm,
                              const int* __restrict__ blk, const long long* __restrict__ off,
                              const long long* __restrict__ dpos, const long long* __restrict__ lpos,
                              const long long* __restrict__ upos, double* __restrict__ store, int* flag) {
  for (long long r = blockIdx.x; r < n; r += gridDim.x) {
    const int pr = iperm[r];
    const int b = blk[pr];
    const long long i = pr - off[b];
    const long long nb = off[b + 1] - off[b];
    for (long long e = rowptr[r] + threadIdx.x; e < rowptr[r + 1]; e += blockDim.x) {
      const int pc = iperm[col[e]];
      const int bc = blk[pc];
      if (bc == b) {
        store[dpos[b] + i * nb + (pc - off[b])] = val[e];
      } else if (bc == b - 1) {
        store[lpos[b] + i * (off[b] - off[b - 1]) + (pc - off[b - 1])] = val[e];
      } else if (bc == b + 1) {
        store[upos[b] + i * (off[b + 2] - off[b + 1]) + (pc - off[b + 1])] = val[e];
      } else {
        atomicExch(flag, 1);
      }
    }
  }
}

// Single-CTA Gauss-Jordan inverse of a small dense block (in place, through shared memory).
__global__ void __launch_bounds__(1024) k_block_inverse_smem(double* __restrict__ M, int n, int* flag) {
  extern __shared__ double sm[];
  double* A = sm;
  short* perm = reinterpret_cast<short*>(A + (size_t)n * n);
  __shared__ int s_piv, s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) A[e] = M[e];
  __syncthreads();
  if (!gj_invert_smem(A, perm, n, &s_piv, &s_bad)) {
    if (threadIdx.x == 0) atomicExch(flag, 1);
    return;
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) M[e] = A[e];
}

// Explicit inverse of a dense n x n block in global memory, one pivot at a time (larger blocks).
static void block_inverse_global(double* M, long long n, int* piv, double* scal, int* flag, cudaStream_t s) {
  const int vb = (int)std::min<long long>((n + 255) / 256, sm_count() * 8LL);
  const int mb = (int)std::min<long long>((n * n + 255) / 256, sm_count() * 32LL);
  for (int k = 0; k < n; ++k) {
    k_gj_pivot<<<1, 1024, 0, s>>>(M, n, k, piv, scal, flag); note_launch();
    k_gj_swap_scale<<<vb, 256, 0, s>>>(M, n, k, piv, scal); note_launch();
    k_gj_update<<<mb, 256, 0, s>>>(M, n, k, piv, scal); note_launch();
    k_gj_column<<<vb, 256, 0, s>>>(M, n, k, piv, scal); note_launch();
  }
  for (int k = (int)n - 1; k >= 0; --k) {
    k_gj_colswap<<<vb, 256, 0, s>>>(M, n, k, piv);
    note_launch();
  }
}

__global__ void k_copy_block(const double* __restrict__ src, long long rows, long long cols, long long lds,
                             double* __restrict__ dst, long long ldd) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < rows * cols;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / cols, j = e - i * cols;
    dst[i * ldd + j] = src[i * lds + j];
  }
}

// cinv[i][j] = Xp[iperm[i]][iperm[j]]
__global__ void k_unpermute(const double* __restrict__ Xp, const int* __restrict__ iperm, long long n,
                            double* __restrict__ out) {
  for (long long i = blockIdx.y; i < n; i += gridDim.y) {
    const double* src = Xp + (long long)iperm[i] * n;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x)
      out[i * n + j] = src[iperm[j]];
  }
}

// dst (cols x rows) = src^T (src rows x cols, both row-major)
__global__ void k_transpose(const double* __restrict__ src, long long rows, long long cols, double* __restrict__ dst) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < rows * cols;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / cols, j = e - i * cols;
    dst[j * rows + i] = src[e];
  }
}
static void transpose_block(const double* src, long long rows, long long cols, double* dst, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return;
  k_transpose<<<(int)std::min<long long>((rows * cols + 255) / 256, sm_count() * 8LL), 256, 0, s>>>(src, rows, cols, dst);
  note_launch();
}

// Coarse levels from this size on are solved through the twisted slab factors instead of an explicit
// inverse: the dense inverse costs N^2 FP64 FMAs per solve (0.5 ms at 18,000 DoFs), the factors about a
// fifth of that in about nx dependent slab steps.
constexpr long long kCoarseSlabMinDofs = 8000;

// Slab ordering of level 0 (host, once). The pressure of cell i goes to slab i + 1 (the last cell's to the
// last slab) when the slabs are eliminated upwards (i < tw), and to slab i when they are eliminated
// downwards (i >= tw, the lower half of the twisted factorisation): either way it is eliminated after the
// velocities of the cell's far plane, which keeps the Schur complements regular.
static void coarse_slabs(const Level& L, int tw, std::vector<int>& iperm, std::vector<int>& blk,
                         std::vector<long long>& off) {
  const int d = L.dim, nx = L.cells[0];
  const long long n = L.N;
  std::vector<int> slab(n);
  for (int a = 0; a < L.K; ++a) {
    for (int l = 0; l < d; ++l)
      for (int nd = 0; nd < L.R; ++nd) {
        const int lx = L.h_node_lat[nd] % L.lat[0];
        slab[a * L.block + (long long)l * L.R + nd] = std::min(lx / 2, nx - 1);
      }
    for (int c = 0; c < L.C; ++c)
      for (int q = 0; q < L.np; ++q)
        slab[a * L.block + (long long)d * L.R + (long long)c * L.np + q] =
            L.h_cell_xyz[3 * c] < tw ? std::min(L.h_cell_xyz[3 * c] + 1, nx - 1) : L.h_cell_xyz[3 * c];
  }
  off.assign(nx + 2, 0);
  for (long long r = 0; r < n; ++r) off[slab[r] + 1]++;
  for (int b = 0; b < nx; ++b) off[b + 1] += off[b];
  off[nx + 1] = off[nx];
  iperm.assign(n, 0);
  blk.assign(n, 0);
  std::vector<long long> fill(off.begin(), off.begin() + nx);
  for (long long r = 0; r < n; ++r) {
    const long long pr = fill[slab[r]]++;
    iperm[r] = (int)pr;
    blk[pr] = slab[r];
  }
}

// In-place inverse of one dense FP64 block (Gauss-Jordan, partial pivoting): in shared memory when it
// fits, else column by column in global memory.
static void invert_block(double* Db, long long nb, int* piv, double* scal, int* flag, int maxsm, cudaStream_t s) {
  const size_t smem = sizeof(double) * nb * nb + sizeof(short) * nb + 16;
  if (smem + 64 <= (size_t)maxsm) {
    cudaFuncSetAttribute(k_block_inverse_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_block_inverse_smem<<<1, 1024, smem, s>>>(Db, (int)nb, flag);
    note_launch();
  } else {
    block_inverse_global(Db, nb, piv, scal, flag, s);
  }
}

// Twisted block factorisation of J_0 in slab order, eliminated from both ends towards slab t = nx / 2
// (A_bc the blocks of J_0, nb_b the rows of slab b):
//   top    b < t :  S_b = A_bb - A_{b,b-1} W_{b-1},            W_b = S_b^{-1} A_{b,b+1},  G_b  = S_b^{-1} A_{b,b-1}
//   bottom b > t :  S_b = A_bb - A_{b,b+1} V_{b+1},            V_b = S_b^{-1} A_{b,b-1},  G'_b = S_b^{-1} A_{b,b+1}
//   middle b = t :  S_t = A_tt - A_{t,t-1} W_{t-1} - A_{t,t+1} V_{t+1},  G_t, G'_t as above.
// Then J_0 x = r is z_b = S_b^{-1} r_b (all slabs); y_b = z_b - G_b y_{b-1} (b = 1 .. t-1) together with
// y_b = z_b - G'_b y_{b+1} (b = nx-2 .. t+1); x_t = z_t - G_t y_{t-1} - G'_t y_{t+1}; x_b = y_b - W_b x_{b+1}
// (b = t-1 .. 0) together with x_b = y_b - V_b x_{b-1} (b = t+1 .. nx-1): about half the dependent steps
// of the one-sided block LU. The Schur complements of J_0^T in the same order are the S_b^T, so the
// transposed system needs no inversion of its own: its blocks are S_b^{-T}, (A_{b-1,b} S_b^{-1})^T (lower
// chain, or back-substitution below the twist) and (A_{b+1,b} S_b^{-1})^T (upper chain, or back-
// substitution above the twist). Every block is kept row-major in H.cs_store at H.cs_pos[kind][b], kinds
// 0..3 (inverse, lower chain G, upper chain G', back-substitution W or V) for J_0 and 4..7 for J_0^T.
static stm_status twisted_slab_factors(Hierarchy& H, const Level& L, const std::vector<long long>& off,
                                       const std::vector<int>& iperm, const std::vector<int>& blk, double* raw,
                                       const std::vector<long long>& dpos, const std::vector<long long>& lpos,
                                       const std::vector<long long>& upos, int* piv, double* scal, int maxsm,
                                       cudaStream_t s) {
  enum { K_INV = 0, K_LO = 1, K_UP = 2, K_BACK = 3, K_T = 4 };
  const int nx = L.cells[0];
  const long long n = L.N;
  const int t = nx / 2;
  auto rows = [&](int b) { return off[b + 1] - off[b]; };
  std::vector<long long> cpos(8 * (size_t)nx, -1);
  long long ct = 0, maxe = 0;
  for (int b = 0; b < nx; ++b) {
    const long long nb = rows(b), npv = b > 0 ? rows(b - 1) : 0, nnx = b + 1 < nx ? rows(b + 1) : 0;
    for (int sys = 0; sys < 2; ++sys) {
      const int k0 = sys * K_T;
      cpos[(k0 + K_INV) * nx + b] = ct; ct += nb * nb;
      if (b >= 1 && b <= t) { cpos[(k0 + K_LO) * nx + b] = ct; ct += nb * npv; }
      if (b >= t && b + 1 < nx) { cpos[(k0 + K_UP) * nx + b] = ct; ct += nb * nnx; }
      if (b < t) { cpos[(k0 + K_BACK) * nx + b] = ct; ct += nb * nnx; }
      if (b > t) { cpos[(k0 + K_BACK) * nx + b] = ct; ct += nb * npv; }
    }
    maxe = std::max(maxe, std::max(npv, nnx) * nb);
  }
  double* E = nullptr;
  if ((!H.cs_store && cudaMalloc(&H.cs_store, sizeof(double) * ct)) || cudaMalloc(&E, sizeof(double) * std::max(maxe, 1LL)) ||
      (!H.cs_u && cudaMalloc(&H.cs_u, sizeof(double) * n)) || (!H.cs_v && cudaMalloc(&H.cs_v, sizeof(double) * n)) ||
      (!H.cs_off && cudaMalloc(&H.cs_off, sizeof(long long) * (nx + 1))) ||
      (!H.cs_pos && cudaMalloc(&H.cs_pos, sizeof(long long) * 8 * nx)) ||
      (!H.cs_rowslab && cudaMalloc(&H.cs_rowslab, sizeof(int) * n)) || (!H.cs_perm && cudaMalloc(&H.cs_perm, sizeof(int) * n))) {
    cudaGetLastError();
    if (E) cudaFree(E);
    set_error("coarse factorisation: out of device memory");
    return STM_ERR_OOM;
  }
  double* cs = H.cs_store;
  auto at = [&](int kind, int b) { return cs + cpos[kind * nx + b]; };
  const double* D = raw;  // raw blocks: A_bb at dpos, A_{b,b-1} at lpos (b >= 1), A_{b,b+1} at upos (b < nx-1)
  auto Lo = [&](int b) { return D + lpos[b]; };
  auto Up = [&](int b) { return D + upos[b]; };
  auto copy = [&](const double* src, long long r, long long c, double* dst) {
    k_copy_block<<<(int)std::min<long long>((r * c + 255) / 256, sm_count() * 8LL), 256, 0, s>>>(src, r, c, c, dst, c);
    note_launch();
  };
  // one slab: S_b from A_bb and the neighbours already eliminated, its inverse, then its chain blocks
  auto slab = [&](int b) {
    const long long nb = rows(b), npv = b > 0 ? rows(b - 1) : 0, nnx = b + 1 < nx ? rows(b + 1) : 0;
    double* Sb = at(K_INV, b);
    copy(D + dpos[b], nb, nb, Sb);
    if (b > 0 && b <= t)  // - A_{b,b-1} W_{b-1}
      dgemm((int)nb, (int)nb, (int)npv, -1.0, Lo(b), npv, at(K_BACK, b - 1), nb, 1.0, Sb, nb, s);
    if (b + 1 < nx && b >= t)  // - A_{b,b+1} V_{b+1}
      dgemm((int)nb, (int)nb, (int)nnx, -1.0, Up(b), nnx, at(K_BACK, b + 1), nb, 1.0, Sb, nb, s);
    invert_block(Sb, nb, piv, scal, H.dflag + 1, maxsm, s);
    if (b >= 1 && b <= t) dgemm((int)nb, (int)npv, (int)nb, 1.0, Sb, nb, Lo(b), npv, 0.0, at(K_LO, b), npv, s);
    if (b >= t && b + 1 < nx) dgemm((int)nb, (int)nnx, (int)nb, 1.0, Sb, nb, Up(b), nnx, 0.0, at(K_UP, b), nnx, s);
    if (b < t) dgemm((int)nb, (int)nnx, (int)nb, 1.0, Sb, nb, Up(b), nnx, 0.0, at(K_BACK, b), nnx, s);
    if (b > t) dgemm((int)nb, (int)npv, (int)nb, 1.0, Sb, nb, Lo(b), npv, 0.0, at(K_BACK, b), npv, s);
    // J_0^T: S_b^{-T}; (A_{b-1,b} S_b^{-1})^T and (A_{b+1,b} S_b^{-1})^T
    transpose_block(Sb, nb, nb, at(K_T + K_INV, b), s);
    if (b > 0) {
      dgemm((int)npv, (int)nb, (int)nb, 1.0, Up(b - 1), nb, Sb, nb, 0.0, E, nb, s);
      transpose_block(E, npv, nb, at(K_T + (b <= t ? K_LO : K_BACK), b), s);
    }
    if (b + 1 < nx) {
      dgemm((int)nnx, (int)nb, (int)nb, 1.0, Lo(b + 1), nb, Sb, nb, 0.0, E, nb, s);
      transpose_block(E, nnx, nb, at(K_T + (b < t ? K_BACK : K_UP), b), s);
    }
  };
  for (int b = 0; b < t; ++b) slab(b);
  for (int b = nx - 1; b > t; --b) slab(b);
  slab(t);
  std::vector<long long> hoff(off.begin(), off.begin() + nx + 1);
  cudaMemcpyAsync(H.cs_off, hoff.data(), sizeof(long long) * (nx + 1), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(H.cs_pos, cpos.data(), sizeof(long long) * 8 * nx, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(H.cs_rowslab, blk.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(H.cs_perm, iperm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s);
  const cudaError_t e1 = cudaGetLastError(), e2 = cudaStreamSynchronize(s);
  cudaFree(E);
  if (e1 != cudaSuccess || e2 != cudaSuccess) {
    set_error("coarse factorisation: CUDA error");
    return STM_ERR_CUDA;
  }
  H.cs_nx = nx;
  H.cs_t = t;
  H.coarse_slab = true;
  return STM_OK;
}

stm_status factor_coarse(Hierarchy& H, cudaStream_t s) {
  Level& L = H.L[0];
  const long long n = L.N;
  const int nx = L.cells[0];
  H.N0 = n;
  const bool use_slab = n >= kCoarseSlabMinDofs && nx >= 2;
  std::vector<int> iperm, blk;
  std::vector<long long> off;
  coarse_slabs(L, use_slab ? nx / 2 : nx, iperm, blk, off);
  // dense block storage: D_b, Lo_b (b >= 1), Up_b (b < nx-1), W_b, G_b
  std::vector<long long> dpos(nx), lpos(nx, 0), upos(nx, 0), wpos(nx, 0), gpos(nx, 0);
  long long tot = 0;
  long long maxnb = 0;
  for (int b = 0; b < nx; ++b) {
    const long long nb = off[b + 1] - off[b];
    maxnb = std::max(maxnb, nb);
    dpos[b] = tot; tot += nb * nb;
    if (b > 0) { lpos[b] = tot; tot += nb * (off[b] - off[b - 1]); }
    if (b + 1 < nx) { upos[b] = tot; tot += nb * (off[b + 2] - off[b + 1]); }
  }
  for (int b = 0; b < nx; ++b) {
    const long long nb = off[b + 1] - off[b];
    if (b + 1 < nx) { wpos[b] = tot; tot += nb * (off[b + 2] - off[b + 1]); }
    if (b > 0) { gpos[b] = tot; tot += nb * (off[b] - off[b - 1]); }
  }
  int *d_iperm = nullptr, *d_blk = nullptr, *piv = nullptr;
  long long *d_off = nullptr, *d_dpos = nullptr, *d_lpos = nullptr, *d_upos = nullptr;
  double *store = nullptr, *Xp = nullptr, *scal = nullptr;
  stm_status st = STM_OK;
  auto fail = [&](stm_status e) { st = e; };
  do {
    if (cudaMalloc(&d_iperm, sizeof(int) * n) || cudaMalloc(&d_blk, sizeof(int) * n) ||
        cudaMalloc(&d_off, sizeof(long long) * (nx + 2)) || cudaMalloc(&d_dpos, sizeof(long long) * nx) ||
        cudaMalloc(&d_lpos, sizeof(long long) * nx) || cudaMalloc(&d_upos, sizeof(long long) * nx) ||
        cudaMalloc(&store, sizeof(double) * tot) || (!use_slab && cudaMalloc(&Xp, sizeof(double) * n * n)) ||
        cudaMalloc(&piv, sizeof(int) * maxnb) || cudaMalloc(&scal, sizeof(double) * 2)) {
      cudaGetLastError();
      set_error("coarse factorisation: out of device memory");
      fail(STM_ERR_OOM);
      break;
    }
    if (!use_slab && !H.cinv && cudaMalloc(&H.cinv, sizeof(double) * n * n)) {
      cudaGetLastError();
      set_error("coarse factorisation: out of device memory");
      fail(STM_ERR_OOM);
      break;
    }
    // the transposed inverse for the adjoint coarse solve
    if (!use_slab && !H.cinvT && cudaMalloc(&H.cinvT, sizeof(double) * n * n)) {
      cudaGetLastError();
      set_error("coarse factorisation: out of device memory");
      fail(STM_ERR_OOM);
      break;
    }
    cudaMemcpyAsync(d_iperm, iperm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_blk, blk.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_off, off.data(), sizeof(long long) * (nx + 2), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_dpos, dpos.data(), sizeof(long long) * nx, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_lpos, lpos.data(), sizeof(long long) * nx, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_upos, upos.data(), sizeof(long long) * nx, cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(store, 0, sizeof(double) * tot, s);
    if (Xp) cudaMemsetAsync(Xp, 0, sizeof(double) * n * n, s);
    k_slab_blocks<<<(int)std::min<long long>(n, sm_count() * 32LL), 128, 0, s>>>(L.rowptr, L.colidx, L.val, n, d_iperm, d_blk,
                                                                          d_off, d_dpos, d_lpos, d_upos, store,
                                                                          H.dflag + 1);
    note_launch();
    int dev = 0, maxsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (use_slab) {
      st = twisted_slab_factors(H, L, off, iperm, blk, store, dpos, lpos, upos, piv, scal, maxsm, s);
      break;
    }
    // forward block LU
    for (int b = 0; b < nx; ++b) {
      const long long nb = off[b + 1] - off[b];
      double* Db = store + dpos[b];
      if (b > 0) {  // S_b = A_bb - A_{b,b-1} W_{b-1}
        const long long np_ = off[b] - off[b - 1];
        dgemm((int)nb, (int)nb, (int)np_, -1.0, store + lpos[b], np_, store + wpos[b - 1], nb, 1.0, Db, nb, s);
      }
      invert_block(Db, nb, piv, scal, H.dflag + 1, maxsm, s);
      if (b + 1 < nx) {  // W_b = S_b^{-1} A_{b,b+1}
        const long long nn_ = off[b + 2] - off[b + 1];
        dgemm((int)nb, (int)nn_, (int)nb, 1.0, Db, nb, store + upos[b], nn_, 0.0, store + wpos[b], nn_, s);
      }
      if (b > 0) {  // G_b = S_b^{-1} A_{b,b-1}
        const long long np_ = off[b] - off[b - 1];
        dgemm((int)nb, (int)np_, (int)nb, 1.0, Db, nb, store + lpos[b], np_, 0.0, store + gpos[b], np_, s);
      }
    }
    // Z = L^{-1} (block lower triangular) into the block rows of Xp
    for (int b = 0; b < nx; ++b) {
      const long long nb = off[b + 1] - off[b];
      double* rowb = Xp + off[b] * n;
      k_copy_block<<<(int)std::min<long long>((nb * nb + 255) / 256, sm_count() * 8LL), 256, 0, s>>>(
          store + dpos[b], nb, nb, nb, rowb + off[b], n);
      note_launch();
      if (b > 0) {
        const long long np_ = off[b] - off[b - 1];
        dgemm((int)nb, (int)off[b], (int)np_, -1.0, store + gpos[b], np_, Xp + off[b - 1] * n, n, 0.0, rowb, n, s);
      }
    }
    // X = U^{-1} Z, last block row first
    for (int b = nx - 2; b >= 0; --b) {
      const long long nb = off[b + 1] - off[b], nn_ = off[b + 2] - off[b + 1];
      dgemm((int)nb, (int)n, (int)nn_, -1.0, store + wpos[b], nn_, Xp + off[b + 1] * n, n, 1.0, Xp + off[b] * n, n, s);
    }
    dim3 ug((unsigned)std::min<long long>((n + 255) / 256, 64), (unsigned)std::min<long long>(n, 65535));
    k_unpermute<<<ug, 256, 0, s>>>(Xp, d_iperm, n, H.cinv);
    note_launch();
    transpose_block(H.cinv, n, n, H.cinvT, s);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
      set_error("coarse factorisation: CUDA error");
      fail(STM_ERR_CUDA);
    }
  } while (false);
  void* ptrs[] = {d_iperm, d_blk, piv, d_off, d_dpos, d_lpos, d_upos, store, Xp, scal};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  return st;
}

}  // namespace stm
