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

// f64 tensor MMA (mma.sync m8n8k4, 512 flop per warp instruction): eight
// independent accumulator pairs per thread, operands in registers.
__global__ void __launch_bounds__(256) dmma_chain_kernel(double *out, int iters) {
  const double a = (double)(threadIdx.x & 7) * 1e-3, b = 0.999999;
  double c[8][2];
#pragma unroll
  for (int q = 0; q < 8; ++q) c[q][0] = c[q][1] = (double)q * 1e-7;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < 8; ++q)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(c[q][0]), "+d"(c[q][1])
                   : "d"(a), "d"(b));
  }
  double s = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += c[q][0] + c[q][1];
  if (s == -12345.0) out[threadIdx.x] = s;  // keeps the loop alive, never true
}

// DFMA and f64 MMA chains interleaved in one thread: whether the two run on
// separate units (a combined rate above either alone) or share one.  Per
// iteration 8 MMAs (4096 flop per warp) and 64 FMAs (4096 flop per warp).
__global__ void __launch_bounds__(256) dual_chain_kernel(double *out, int iters) {
  const double a = (double)(threadIdx.x & 7) * 1e-3, b = 0.999999, cc = 1e-9;
  double c[8][2], f[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    c[q][0] = c[q][1] = (double)q * 1e-7;
    f[q] = (double)(threadIdx.x + q) * 1e-3;
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(c[q][0]), "+d"(c[q][1])
                   : "d"(a), "d"(b));
#pragma unroll
      for (int u = 0; u < 8; ++u) f[u] = fma(f[u], b, cc);
    }
  }
  double s = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += c[q][0] + c[q][1] + f[q];
  if (s == -12345.0) out[threadIdx.x] = s;  // keeps the loop alive, never true
}

gb_status measure_dual(gb_handle *h, double *rate) {
  const int blocks = h->sm_count * 8, threads = 256, iters = 128;
  double *out = nullptr;
  GB_CUDA_TRY(cudaMalloc(&out, 256 * sizeof(double)));
  cudaEvent_t a, b;
  GB_CUDA_TRY(cudaEventCreate(&a));
  GB_CUDA_TRY(cudaEventCreate(&b));
  dual_chain_kernel<<<blocks, threads>>>(out, iters / 8);  // warm-up
  count_launch();
  GB_CUDA_TRY(cudaEventRecord(a));
  dual_chain_kernel<<<blocks, threads>>>(out, iters);
  count_launch();
  GB_CUDA_TRY(cudaEventRecord(b));
  GB_CUDA_TRY(cudaEventSynchronize(b));
  float ms = 0;
  GB_CUDA_TRY(cudaEventElapsedTime(&ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(out);
  const double warps = (double)blocks * (threads / 32) * iters;
  *rate = warps * 8.0 * (512.0 + 8.0 * 64.0) / (ms * 1e-3);
  return GB_OK;
}

gb_status measure_dmma(gb_handle *h, double *rate) {
  const int blocks = h->sm_count * 8, threads = 256, iters = 256;
  double *out = nullptr;
  GB_CUDA_TRY(cudaMalloc(&out, 256 * sizeof(double)));
  cudaEvent_t a, b;
  GB_CUDA_TRY(cudaEventCreate(&a));
  GB_CUDA_TRY(cudaEventCreate(&b));
  dmma_chain_kernel<<<blocks, threads>>>(out, iters / 8);  // warm-up
  count_launch();
  GB_CUDA_TRY(cudaEventRecord(a));
  dmma_chain_kernel<<<blocks, threads>>>(out, iters);
  count_launch();
  GB_CUDA_TRY(cudaEventRecord(b));
  GB_CUDA_TRY(cudaEventSynchronize(b));
  float ms = 0;
  GB_CUDA_TRY(cudaEventElapsedTime(&ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(out);
  const double warp_mmas = (double)blocks * (threads / 32) * iters * 8.0;
  *rate = warp_mmas * 512.0 / (ms * 1e-3);
  return GB_OK;
}

}  // namespace
}  // namespace gb

extern "C" gb_status gb_measure_peak(gb_handle *h, gb_peak kind, double *flops_per_s) {
  if (!h) return -1;
  if (kind < GB_PEAK_DFMA || kind > GB_PEAK_DFMA_DMMA) return -2;
  if (!flops_per_s) return -3;
  if (kind == GB_PEAK_DFMA) return gb_measure_fma_peak(h, GB_F64, flops_per_s);
  if (kind == GB_PEAK_FFMA) return gb_measure_fma_peak(h, GB_F32, flops_per_s);
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(h->device);
  gb_status r = GB_OK;
  {
    std::lock_guard<std::mutex> lk(h->mu);
    if (kind == GB_PEAK_DMMA) {
      r = gb::measure_dmma(h, flops_per_s);
    } else if (kind == GB_PEAK_DFMA_DMMA) {
      r = gb::measure_dual(h, flops_per_s);
    } else {
      const cudaError_t e = gb::measure_tc_peak((int)kind - (int)GB_PEAK_TC_BF16, h->sm_count,
                                                flops_per_s);
      if (e == cudaErrorNotSupported) r = GB_ERR_UNSUPPORTED;
      else if (e == cudaErrorLaunchTimeout) r = GB_ERR_TIMEOUT;
      else if (e != cudaSuccess) {
        gb::record_cuda_error(e, "measure_tc_peak", __FILE__, __LINE__);
        r = GB_ERR_CUDA;
      }
    }
  }
  cudaSetDevice(prev);
  return r;
}

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
