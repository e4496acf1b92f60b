// gb_chol_solve_noalloc: forward and back substitution with a Cholesky
// factor for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside a memory budget
// it does not own (a host application that hands this library a fixed
// arena, or a pool that is already fully reserved), a latency-critical
// section where an allocation (which may synchronize the whole device) is
// not allowed, or a plugin loaded into another program that must not touch
// that program's allocator.  The regular gb_chol_solve needs a handle, and
// gb_create allocates the handle's scratch words (the ticket and per-block
// flags that order the single-launch triangular solve).  This entry point
// takes no handle: its scratch is the file-scope array below, which every
// GPU that loads the library holds until the process exits.
//
// Properties:
//  * at most NOALLOC_MAX_N rows (NOALLOC_BLOCKS blocks of 32 rows);
//  * device pointers on the current device only (staging host buffers would
//    allocate; another GPU's memory is rejected);
//  * the call waits for `stream`: it reads the breakdown word before the
//    substitutions and the error word after them on the host;
//  * every call shares the one array and it keeps the last call's contents:
//    the ticket, the error word and the breakdown word are cleared by each
//    call, and the per-block flags are compared against a fresh epoch, so
//    stale flags never match;
//  * calls that overlap on the GPU (two streams, one device) race on the
//    array and must not be issued;
//  * the first call on a device looks up the array's device address
//    (cudaGetSymbolAddress, with that device current): that set-up happens
//    once per device, and the first call should come before any stream
//    capture.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

#include "gb_internal.cuh"

namespace gb {
namespace {

constexpr int NOALLOC_BLOCKS = 4096;           // 32-row blocks
constexpr int64_t NOALLOC_MAX_N = 4096LL * 32;  // 131072 rows
// [0] ticket, [1 .. NOALLOC_BLOCKS] block flags, then the error word and the
// breakdown word
constexpr int NOALLOC_WORDS = 1 + NOALLOC_BLOCKS + 2;
static_assert(NOALLOC_BLOCKS + 1 <= SYNC_WORDS, "flag layout");

static __device__ __align__(256) int g_noalloc_scratch[NOALLOC_WORDS];

struct DeviceScratch {
  std::once_flag once;
  cudaError_t status = cudaSuccess;
  int *ptr = nullptr;
  std::atomic<unsigned> epoch{0};
};
constexpr int MAX_DEVICES = 64;
DeviceScratch g_scratch[MAX_DEVICES];

unsigned next_epoch(DeviceScratch &d) {
  unsigned e = ++d.epoch;
  if (e == 0) e = ++d.epoch;  // 0 is the value of a never-written flag
  return e;
}

// Device (or managed) memory that the kernels on device `dev` can address:
// plain device memory must belong to `dev` itself.
bool is_device_pointer(const void *p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

template <typename Tf>
gb_status solve_static(const Tf *L, int64_t ldl, double *X, int64_t ldx, int64_t n, int64_t nrhs,
                       DeviceScratch &d, cudaStream_t st) {
  int *sync = d.ptr;
  int *err = d.ptr + 1 + NOALLOC_BLOCKS;
  int *bad = err + 1;
  GB_CUDA_TRY(cudaMemsetAsync(err, 0, 2 * sizeof(int), st));
  GB_CUDA_TRY(launch_check_diag<Tf>(L, ldl, n, bad, st));
  int words[2] = {0, 0};
  GB_CUDA_TRY(cudaMemcpyAsync(&words[1], bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  GB_CUDA_TRY(cudaStreamSynchronize(st));
  if (words[1]) return GB_ERR_BREAKDOWN;
  const int64_t wait = (int64_t)1 << 26;  // x 100 ns
  GB_CUDA_TRY((launch_trsm<Tf, Tf>(L, ldl, X, ldx, n, nrhs, TRSM_LOWER, sync, next_epoch(d), err,
                                   wait, st)));
  GB_CUDA_TRY((launch_trsm<Tf, Tf>(L, ldl, X, ldx, n, nrhs, TRSM_LOWER_T, sync, next_epoch(d), err,
                                   wait, st)));
  GB_CUDA_TRY(cudaMemcpyAsync(&words[0], err, sizeof(int), cudaMemcpyDeviceToHost, st));
  GB_CUDA_TRY(cudaStreamSynchronize(st));
  if (words[0] & DEV_ERR_TIMEOUT) return GB_ERR_TIMEOUT;
  return words[0] ? GB_ERR_CUDA : GB_OK;
}

}  // namespace
}  // namespace gb

extern "C" gb_status gb_chol_solve_noalloc(int64_t n, int64_t nrhs, gb_dtype factor_dt,
                                           const void *L, int64_t ldl, const double *B,
                                           int64_t ldb, double *X, int64_t ldx, void *stream) {
  using namespace gb;
  if (n < 0) return -1;
  if (nrhs < 0) return -2;
  if (factor_dt < GB_F64 || factor_dt > GB_MIX_BF16X3) return -3;
  if (n > 0 && !L) return -4;
  if (ldl < (n > 1 ? n : 1)) return -5;
  if (n > 0 && nrhs > 0 && !B) return -6;
  if (ldb < (nrhs > 1 ? nrhs : 1)) return -7;
  if (n > 0 && nrhs > 0 && !X) return -8;
  if (ldx < (nrhs > 1 ? nrhs : 1)) return -9;
  if (n > NOALLOC_MAX_N) {
    record_cuda_error(cudaErrorInvalidValue, "gb_chol_solve_noalloc: n exceeds 131072 rows",
                      __FILE__, __LINE__);
    return GB_ERR_UNSUPPORTED;
  }
  if (n == 0 || nrhs == 0) return GB_OK;
  int dev = 0;
  GB_CUDA_TRY(cudaGetDevice(&dev));
  if (!is_device_pointer(L, dev)) return -4;
  if (!is_device_pointer(B, dev)) return -6;
  if (!is_device_pointer(X, dev)) return -8;
  if (dev < 0 || dev >= MAX_DEVICES) return GB_ERR_UNSUPPORTED;
  DeviceScratch &d = g_scratch[dev];
  // once per device, with that device current: the array's device address
  std::call_once(d.once, [&] {
    void *p = nullptr;
    d.status = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (d.status == cudaSuccess) d.ptr = static_cast<int *>(p);
    else cudaGetLastError();
  });
  if (d.status != cudaSuccess || !d.ptr) {
    record_cuda_error(d.status, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
    return GB_ERR_CUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (X != B)
    GB_CUDA_TRY(cudaMemcpy2DAsync(X, ldx * 8, B, ldb * 8, nrhs * 8, n, cudaMemcpyDeviceToDevice, st));
  if (factor_dt == GB_F64)
    return solve_static<double>((const double *)L, ldl, X, ldx, n, nrhs, d, st);
  return solve_static<float>((const float *)L, ldl, X, ldx, n, nrhs, d, st);
}
