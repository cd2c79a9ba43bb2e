// FMA throughput of the current device, measured: the denominators of the
// arithmetic rooflines that the benchmark reports beside the HBM one.  Each
// thread runs eight independent fused multiply-add chains, so the FMA pipes
// stay busy and nothing else (memory, branches) is timed.  No clock or power
// setting is touched; the result is what the part delivers as it is.
#include <cuda_runtime.h>

#include <algorithm>

#include "pic.h"

namespace {

__device__ double g_peak_sink;  // keeps the chains live; written only on a value no chain reaches

template <class R> __global__ void __launch_bounds__(256) k_fma_chains(int iters) {
  R a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = R(threadIdx.x + k);
  const R m = R(0.9999999), c = R(1e-7);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], m, c);
  }
  R s = R(0);
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  if (s == R(-1)) g_peak_sink = (double)s;
}

template <class R> double time_chains(int iters, cudaStream_t st) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = nsm * 8, threads = 256;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fma_chains<R><<<blocks, threads, 0, st>>>(iters);  // warm-up
  float best = 1e30f;
  for (int r = 0; r < 3; ++r) {
    cudaEventRecord(e0, st);
    k_fma_chains<R><<<blocks, threads, 0, st>>>(iters);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double flops = 2.0 * 8.0 * (double)iters * blocks * threads;
  return flops / (best * 1e-3) / 1e12;
}

}  // namespace

extern "C" int pic_alu_peak(double *fp32_tflops, double *fp64_tflops, void *stream) {
  if (!fp32_tflops || !fp64_tflops) return PIC_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  *fp32_tflops = time_chains<float>(1 << 16, st);
  *fp64_tflops = time_chains<double>(1 << 11, st);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PIC_OK : PIC_ECUDA;
}
