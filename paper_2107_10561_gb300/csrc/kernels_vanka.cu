// Cell-based space-time Vanka smoother (Sec. 4.2, Eq. LocVanka, damping of Sec. 5.3).
//
// Local step for cell T: y_T = J_T^{-1} t_T with t = r - J d gathered over all (k+1) time nodes
// of the cell's DoFs. The inverse is streamed once per sweep (the dominant HBM traffic), stored
// column-major per cell so that consecutive threads read consecutive rows of one column.
// Shared DoFs are combined in a second, deterministic pass:
//   additive : d_i += omega / m_i * sum over the owners of i of y_T[alpha]
//   overwrite: d_i += omega * y_Tlast[alpha] (highest-index owning cell, "last update wins")
//   coloured : cells of one colour share no DoF, so y is scattered directly (d_T += omega y_T).
#include "internal.h"

namespace stm {

template <typename S> struct Acc { using T = float; };
template <> struct Acc<double> { using T = double; };

template <typename S> __device__ __forceinline__ float ld_f(const S* p);
template <> __device__ __forceinline__ float ld_f<float>(const float* p) { return __ldg(p); }
template <> __device__ __forceinline__ float ld_f<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}
__device__ __forceinline__ double ld_d(const double* p) { return __ldg(p); }

// One CTA per cell (grid-stride). Threads are split into G column groups of n rows: thread
// (g, i) accumulates sum_{j = g (mod G)} Inv[j][i] t_j (forward) and the G partial sums are added
// in shared memory. transpose = 1 computes y = Inv^T t: each warp owns whole columns.
template <typename S>
__global__ void __launch_bounds__(256) k_vanka_local(
    const S* __restrict__ inv, const int* __restrict__ idx, const double* __restrict__ t,
    double* __restrict__ Y, const int* __restrict__ cell_list, int ncells, int n, int G,
    int transpose, double* __restrict__ d_scatter, double omega) {
  using A = typename Acc<S>::T;
  extern __shared__ double smd[];
  double* tl = smd;                                 // [n]
  A* part = reinterpret_cast<A*>(smd + n);          // [G][n]
  const int tid = threadIdx.x;
  for (int ci = blockIdx.x; ci < ncells; ci += gridDim.x) {
    const int c = cell_list ? cell_list[ci] : ci;
    const int* ic = idx + (long long)c * n;
    __syncthreads();
    for (int i = tid; i < n; i += blockDim.x) tl[i] = t[ic[i]];
    __syncthreads();
    const S* M = inv + (size_t)c * n * n;
    if (!transpose) {
      if (tid < G * n) {
        const int g = tid / n, i = tid - g * n;
        A acc = 0;
        const S* col = M + (size_t)g * n + i;
        const size_t stride = (size_t)G * n;
        int j = g;
#pragma unroll 4
        for (; j < n; j += G, col += stride) {
          if constexpr (sizeof(S) == 8) acc += ld_d((const double*)col) * tl[j];
          else acc += ld_f<S>(col) * (A)tl[j];
        }
        part[g * n + i] = acc;
      }
      __syncthreads();
      for (int i = tid; i < n; i += blockDim.x) {
        A y = 0;
        for (int g = 0; g < G; ++g) y += part[g * n + i];
        if (d_scatter) d_scatter[ic[i]] += omega * (double)y;
        else Y[(long long)c * n + i] = (double)y;
      }
    } else {
      const int lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
      for (int j = wid; j < n; j += nw) {
        const S* col = M + (size_t)j * n;
        A acc = 0;
        for (int i = lane; i < n; i += 32) {
          if constexpr (sizeof(S) == 8) acc += ld_d((const double*)(col + i)) * tl[i];
          else acc += ld_f<S>(col + i) * (A)tl[i];
        }
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
        if (lane == 0) {
          if (d_scatter) d_scatter[ic[j]] += omega * (double)acc;
          else Y[(long long)c * n + j] = (double)acc;
        }
      }
    }
  }
}

// Second pass of the additive / overwrite variants (one thread per global DoF).
__global__ void k_vanka_gather(double* __restrict__ d, const double* __restrict__ Y,
                               const int* __restrict__ own_ptr, const int* __restrict__ own_pos,
                               const int* __restrict__ last_owner, const double* __restrict__ wmult,
                               long long N, double omega, int overwrite) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    if (overwrite) {
      d[i] += omega * Y[last_owner[i]];
    } else {
      double s = 0.0;
      for (int p = own_ptr[i]; p < own_ptr[i + 1]; ++p) s += Y[own_pos[p]];
      d[i] += omega * wmult[i] * s;
    }
  }
}

static int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 152;
  }
  return n;
}

static stm_status launch_local(Hierarchy& H, Level& L, const double* t, const int* cells, int nc,
                               int transpose, double* scatter, cudaStream_t s) {
  if (nc <= 0) return STM_OK;
  const int threads = 256;
  const int G = std::max(1, threads / L.n);
  const int prec = H.p.inv_precision;
  const size_t smem = sizeof(double) * L.n + (prec == STM_F64 ? 8 : 4) * (size_t)G * L.n + 16;
  const int blocks = std::min(nc, sm_count() * 8);
  ProfScope ps(&H, STM_KCLASS_VANKA_LOCAL, s,
               (double)nc * ((double)L.n * L.n * (prec == STM_F64 ? 8 : prec == STM_F32 ? 4 : 2) + 20.0 * L.n));
  if (prec == STM_F64) {
    k_vanka_local<double><<<blocks, threads, smem, s>>>((const double*)L.inv, L.idx, t, L.Y, cells, nc, L.n, G,
                                                        transpose, scatter, H.p.omega);
  } else if (prec == STM_F32) {
    k_vanka_local<float><<<blocks, threads, smem, s>>>((const float*)L.inv, L.idx, t, L.Y, cells, nc, L.n, G,
                                                       transpose, scatter, H.p.omega);
  } else {
    k_vanka_local<__nv_bfloat16><<<blocks, threads, smem, s>>>((const __nv_bfloat16*)L.inv, L.idx, t, L.Y, cells,
                                                               nc, L.n, G, transpose, scatter, H.p.omega);
  }
  note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}

stm_status vanka_step(Hierarchy& H, int g, const double* r, double* d, int transpose, bool d_is_zero,
                      cudaStream_t s) {
  Level& L = H.L[g];
  const double omega = H.p.omega;
  if (H.p.smoother == STM_VANKA_COLOURED) {
    for (int col = 0; col < (1 << L.dim); ++col) {
      const int nc = L.colour_off[col + 1] - L.colour_off[col];
      const double* t = r;
      if (!(d_is_zero && col == 0)) {
        stm_status st = jacobian_apply(H, g, d, r, L.t, 1, transpose, s);
        if (st != STM_OK) return st;
        t = L.t;
      }
      stm_status st = launch_local(H, L, t, L.colour_cells + L.colour_off[col], nc, transpose, d, s);
      if (st != STM_OK) return st;
    }
    return STM_OK;
  }
  const double* t = r;
  if (!d_is_zero) {
    stm_status st = jacobian_apply(H, g, d, r, L.t, 1, transpose, s);
    if (st != STM_OK) return st;
    t = L.t;
  }
  stm_status st = launch_local(H, L, t, nullptr, L.C, transpose, nullptr, s);
  if (st != STM_OK) return st;
  const int blocks = (int)std::min<long long>((L.N + 255) / 256, sm_count() * 16LL);
  ProfScope ps(&H, STM_KCLASS_VANKA_COMBINE, s, 0.0);
  k_vanka_gather<<<blocks, 256, 0, s>>>(d, L.Y, L.own_ptr, L.own_pos, L.last_owner, L.wmult, L.N, omega,
                                        H.p.smoother == STM_VANKA_PAPER_OVERWRITE); note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}

}  // namespace stm
