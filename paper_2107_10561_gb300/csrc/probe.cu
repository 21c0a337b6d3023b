// Measurement support: FP64 FMA throughput of the current device (the peak against which the
// FP64-pipe-bound kernels of the solve are reported). Eight independent FMA chains per thread,
// 8 CTAs of 256 threads per SM; the result is FLOP/s = 2 x FMAs / CUDA-event time.
// Verification support: the bounded mbarrier wait of the pipelined kernels, run against a barrier
// that nothing completes.
#include "internal.h"

namespace stm {

__global__ void k_fp64_fma_probe(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

}  // namespace stm

using namespace stm;

extern "C" stm_status stm_measure_fp64_peak(double* tflops, void* stream) {
  if (!tflops) {
    set_error("stm_measure_fp64_peak: NULL argument");
    return STM_ERR_INVALID_ARG;
  }
  int dev = 0, sms = 0;
  STM_CUDA(cudaGetDevice(&dev));
  STM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256, iters = 4096;
  double* out = nullptr;
  STM_CUDA(cudaMalloc(&out, sizeof(double) * blocks * threads));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  STM_CUDA(cudaEventCreate(&e0));
  STM_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    STM_CUDA(cudaEventRecord(e0, s));
    k_fp64_fma_probe<<<blocks, threads, 0, s>>>(out, iters, 0.999999, 1e-7);
    STM_CUDA(cudaEventRecord(e1, s));
    STM_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    STM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (rep > 0 && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  *tflops = 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e-3) / 1e12;
  return STM_OK;
}

extern "C" stm_status stm_selftest_bounded_wait(int* timed_out, double* ms, void* stream) {
  if (!timed_out || !ms) {
    set_error("stm_selftest_bounded_wait: NULL argument");
    return STM_ERR_INVALID_ARG;
  }
  int* err = nullptr;
  STM_CUDA(cudaMalloc(&err, sizeof(int)));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  stm_status st = STM_OK;
  int e = 0;
  float t = 0.f;
  if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    set_error("stm_selftest_bounded_wait: CUDA error");
    cudaFree(err);
    return STM_ERR_CUDA;
  }
  cudaEventRecord(e0, s);
  st = bounded_wait_selftest(err, s);
  cudaEventRecord(e1, s);
  if (st == STM_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess ||
                       cudaMemcpy(&e, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)) {
    set_error("stm_selftest_bounded_wait: CUDA error");
    st = STM_ERR_CUDA;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(err);
  *timed_out = (e & 128) ? 1 : 0;
  *ms = t;
  return st;
}
