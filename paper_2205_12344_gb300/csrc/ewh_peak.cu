// Arithmetic-throughput probe of the current GPU (no counterpart in the
// paper): the FP32 and FP64 CUDA-core FMA rates that bound the step kernels
// whose time is spent in arithmetic rather than memory traffic.
//
// Every thread runs CHAINS independent FMA recurrences a <- a * b + c for
// `iters` rounds; enough warps per SM keep every FMA pipe busy, so the rate is
// the device's FMA throughput.  One FMA counts as two floating-point
// operations.
#include <cuda_runtime.h>

#include <string>

#include "../../include/ewh.h"
#include "ewh_internal.cuh"

namespace ewh {
namespace {

constexpr int PEAK_CHAINS = 8;
constexpr int PEAK_THREADS = 256;
constexpr int PEAK_BLOCKS_PER_SM = 8;

__device__ double g_peak_sink;  // written only if the chains reach an impossible value

template <typename T>
__global__ void __launch_bounds__(PEAK_THREADS) fma_rate_kernel(int iters, T b, T c) {
  T a[PEAK_CHAINS];
#pragma unroll
  for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = T(threadIdx.x + k) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = fma(a[k], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < PEAK_CHAINS; ++k) s += a[k];
  if (s == T(-1.2345)) g_peak_sink = (double)s;  // keeps the chains live; never true for these inputs
}

template <typename T>
cudaError_t time_fma(cudaStream_t st, double* flops) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const dim3 grid(sms * PEAK_BLOCKS_PER_SM);
  // size the run to about 50 ms from a short first launch
  int iters = sizeof(T) == 8 ? 256 : 4096;
  float ms = 0.f;
  for (int round = 0; round < 3 && e == cudaSuccess; ++round) {
    cudaEventRecord(e0, st);
    fma_rate_kernel<T><<<grid, PEAK_THREADS, 0, st>>>(iters, T(0.999999), T(1e-7));
    cudaEventRecord(e1, st);
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
    cudaEventElapsedTime(&ms, e0, e1);
    if (round < 2 && ms < 40.f) {
      const double scale = 50.0 / (ms > 0.01f ? ms : 0.01f);
      iters = (int)(iters * (scale > 1000.0 ? 1000.0 : scale));
    }
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess)
    *flops = 2.0 * PEAK_CHAINS * (double)iters * grid.x * PEAK_THREADS / (ms * 1e-3);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

}  // namespace
}  // namespace ewh

extern "C" ewh_status ewh_fma_rate(int precision, double* flops_per_second, void* cuda_stream) {
  using namespace ewh;
  if (!flops_per_second || (precision != EWH_FP64 && precision != EWH_FP32_STENCIL)) {
    set_global_error("ewh_fma_rate: precision must be EWH_FP64 or EWH_FP32_STENCIL and the output non-null");
    return EWH_EINVAL;
  }
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  const cudaError_t e = precision == EWH_FP64 ? time_fma<double>(st, flops_per_second)
                                              : time_fma<float>(st, flops_per_second);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_global_error(std::string("ewh_fma_rate: ") + cudaGetErrorString(e));
    return EWH_ECUDA;
  }
  return EWH_OK;
}
