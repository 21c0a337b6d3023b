// Allocation-free variant of the additive Vanka correction (see stm_vanka_apply_noalloc in stm.h).
//
// The regular smoother keeps its per-cell corrections and owner lists in memory that
// stm_build_hierarchy allocates. This variant needs no library-owned allocation at all: all of
// its scratch lives in one fixed-size, file-scope device array that exists from the moment the
// library is loaded on a device until the process exits.
#include "internal.h"

namespace stm {

// Largest number of global DoFs one call may touch.
constexpr long long kNoAllocMaxDofs = 1LL << 20;  // 1,048,576 DoFs -> 16 MiB of scratch

// Scratch: [0, kNoAllocMaxDofs) summed local corrections, [kNoAllocMaxDofs, 2 kNoAllocMaxDofs)
// number of cells that contributed to each DoF (stored as doubles, exact for small counts).
static __device__ __align__(256) double g_noalloc_scratch[2 * kNoAllocMaxDofs];

__global__ void k_noalloc_clear(double* __restrict__ scratch, long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    scratch[i] = 0.0;
    scratch[kNoAllocMaxDofs + i] = 0.0;
  }
}

// One CTA per cell: y = Inv_T t_T (Inv_T column-major, FP64), then each local row adds y_i and a
// count of one to the scratch slot of its global DoF.
// Local DoF indices outside [0, N) are ignored (their t is read as 0 and they receive nothing).
__global__ void k_noalloc_local(const double* __restrict__ inv, const int* __restrict__ idx,
                                const double* __restrict__ t, double* __restrict__ scratch, long long C, int n,
                                long long N) {
  extern __shared__ double tl[];
  for (long long c = blockIdx.x; c < C; c += gridDim.x) {
    const int* ic = idx + c * n;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int g = ic[i];
      tl[i] = (g >= 0 && g < N) ? t[g] : 0.0;
    }
    __syncthreads();
    const double* M = inv + (size_t)c * n * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int g = ic[i];
      if (g < 0 || g >= N) continue;
      double y = 0.0;
      for (int j = 0; j < n; ++j) y += M[(size_t)j * n + i] * tl[j];
      atomicAdd(&scratch[g], y);
      atomicAdd(&scratch[kNoAllocMaxDofs + g], 1.0);
    }
  }
}

__global__ void k_noalloc_combine(const double* __restrict__ scratch, double* __restrict__ d, long long N,
                                  double omega) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double m = scratch[kNoAllocMaxDofs + i];
    if (m > 0.0) d[i] += omega * scratch[i] / m;
  }
}

// Device address of the scratch array on the current device. Looked up on every call (a cheap
// query once the library's module is loaded on the device), so a call after cudaDeviceReset or on
// another device never uses an address from an earlier context.
static stm_status noalloc_scratch(double** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
  *out = static_cast<double*>(p);
  return STM_OK;
}

static int noalloc_sms() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      n <= 0)
    n = 1;
  return n;
}

}  // namespace stm

using namespace stm;

extern "C" stm_status stm_vanka_apply_noalloc(long long n_cells, int n_local, long long n_dofs, const double* inv_dev,
                                              const int* idx_dev, const double* t_dev, double* d_dev, double omega,
                                              void* stream) {
  if (!inv_dev || !idx_dev || !t_dev || !d_dev) {
    set_error("stm_vanka_apply_noalloc: NULL argument");
    return STM_ERR_INVALID_ARG;
  }
  if (n_cells < 0 || n_local < 1 || n_local > 1024 || n_dofs < 0) {
    set_error("stm_vanka_apply_noalloc: sizes must satisfy n_cells >= 0, 1 <= n_local <= 1024, n_dofs >= 0");
    return STM_ERR_INVALID_ARG;
  }
  if (n_dofs > kNoAllocMaxDofs) {
    set_error("stm_vanka_apply_noalloc: n_dofs exceeds the fixed scratch capacity of 1048576 DoFs");
    return STM_ERR_INVALID_ARG;
  }
  if (n_dofs == 0 || n_cells == 0) return STM_OK;
  double* scratch = nullptr;
  stm_status st = noalloc_scratch(&scratch);
  if (st != STM_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int sms = noalloc_sms();
  const int vb = (int)std::min<long long>((n_dofs + 255) / 256, sms * 8LL);
  k_noalloc_clear<<<vb, 256, 0, s>>>(scratch, n_dofs);
  note_launch();
  const int cb = (int)std::min<long long>(n_cells, sms * 16LL);
  k_noalloc_local<<<cb, 128, sizeof(double) * n_local, s>>>(inv_dev, idx_dev, t_dev, scratch, n_cells, n_local,
                                                               n_dofs);
  note_launch();
  k_noalloc_combine<<<vb, 256, 0, s>>>(scratch, d_dev, n_dofs, omega);
  note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}
