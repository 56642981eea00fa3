// Measurement utility: the FP64 fused-multiply-add rate of the device, the
// denominator of the FP64 step kernel's roofline. Not part of the method.
//
// Every thread runs 8 independent FMA chains x <- x * a + b (a, b runtime
// values, |a| < 1 so the chains stay bounded) for `iters` rounds; the grid
// is 4 CTAs of 512 threads per SM, enough warps to cover the FP64 latency.
// FLOP = 2 * 8 * iters * threads. The launch is timed with CUDA events on
// the given stream after one untimed warm-up launch.

#include <cuda_runtime.h>

#include "mc_internal.h"

namespace {

constexpr int PROBE_THREADS = 512;
constexpr int PROBE_CHAINS = 8;

__global__ void __launch_bounds__(PROBE_THREADS) dfma_rate_kernel(double* out, int iters, double a,
                                                                  double b) {
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double x[PROBE_CHAINS];
#pragma unroll
  for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = 1e-3 * (double)(gid & 1023) + (double)k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < PROBE_CHAINS; ++k) s += x[k];
  out[gid] = s;
}

}  // namespace

extern "C" mc_status mc_fp64_fma_rate(void* stream, double* tflops) {
  if (!tflops) return MC_E_ARG;
  *tflops = 0.0;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MC_E_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MC_E_CUDA;
  const int blocks = 4 * sms;
  const long long threads = (long long)blocks * PROBE_THREADS;
  const int iters = 4096;
  double* out = nullptr;
  if (cudaMallocAsync((void**)&out, threads * sizeof(double), st) != cudaSuccess) return MC_E_ALLOC;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  mc_status rs = MC_OK;
  float ms = 0.0f;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rs = MC_E_CUDA;
  } else {
    dfma_rate_kernel<<<blocks, PROBE_THREADS, 0, st>>>(out, iters, 0.999999, 1e-7);
    cudaEventRecord(e0, st);
    dfma_rate_kernel<<<blocks, PROBE_THREADS, 0, st>>>(out, iters, 0.999999, 1e-7);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
        cudaGetLastError() != cudaSuccess)
      rs = MC_E_CUDA;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(out, st);
  cudaStreamSynchronize(st);
  if (rs != MC_OK) return rs;
  if (!(ms > 0.0f)) return MC_E_CUDA;
  const double flop = 2.0 * PROBE_CHAINS * (double)iters * (double)threads;
  *tflops = flop / (ms * 1e-3) / 1e12;
  return MC_OK;
}
