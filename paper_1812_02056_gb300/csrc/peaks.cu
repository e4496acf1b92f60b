// gb_measure_fma_peak: register-only fused multiply-add throughput of the
// device's FP64 (DFMA) or FP32 (FFMA) pipes, used as the arithmetic roofline
// of the SIMT kernels.  Eight independent FMA chains per thread hide the
// pipe latency; the grid fills every SM several times over.
#include <cuda_runtime.h>

#include "gb_internal.cuh"

namespace gb {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) fma_chain_kernel(T *out, int iters, T b, T c) {
  T a[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) a[q] = (T)(threadIdx.x + q) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int q = 0; q < 8; ++q) a[q] = fma(a[q], b, c);
  }
  T s = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += a[q];
  if (s == (T)-12345.0) out[threadIdx.x] = s;  // keeps the loop alive, never true
}

template <typename T>
gb_status measure(gb_handle *h, double *rate) {
  const int blocks = h->sm_count * 8, threads = 256;
  const int iters = sizeof(T) == 8 ? 64 : 4096;
  T *out = nullptr;
  GB_CUDA_TRY(cudaMalloc(&out, 256 * sizeof(T)));
  cudaEvent_t a, b;
  GB_CUDA_TRY(cudaEventCreate(&a));
  GB_CUDA_TRY(cudaEventCreate(&b));
  fma_chain_kernel<T><<<blocks, threads>>>(out, iters / 8, (T)0.999999, (T)1e-7);  // warm-up
  count_launch();
  GB_CUDA_TRY(cudaEventRecord(a));
  fma_chain_kernel<T><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7);
  count_launch();
  GB_CUDA_TRY(cudaEventRecord(b));
  GB_CUDA_TRY(cudaEventSynchronize(b));
  float ms = 0;
  GB_CUDA_TRY(cudaEventElapsedTime(&ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(out);
  const double fmas = (double)blocks * threads * iters * 16.0 * 8.0;
  *rate = 2.0 * fmas / (ms * 1e-3);
  return GB_OK;
}

}  // namespace
}  // namespace gb

extern "C" gb_status gb_measure_fma_peak(gb_handle *h, gb_dtype dt, double *flops_per_s) {
  if (!h) return -1;
  if (dt != GB_F64 && dt != GB_F32) return -2;
  if (!flops_per_s) return -3;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(h->device);
  std::lock_guard<std::mutex> lk(h->mu);
  gb_status r = dt == GB_F64 ? gb::measure<double>(h, flops_per_s) : gb::measure<float>(h, flops_per_s);
  cudaSetDevice(prev);
  return r;
}
