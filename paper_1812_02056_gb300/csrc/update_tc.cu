// Delayed rank-s update of Algorithms 1 and 2 (arXiv:1812.02056, Sec. 2) on
// the 5th-generation tensor cores (tcgen05) for the mixed-precision dtypes:
//   C (FP32) -= X Y^T   (Cholesky, lower tiles only; X = Y = R)
//   C (FP32) -= X Y     (LU, full square; X = R_L, Y = R_U)
// with X and Y rounded to BF16 (or FP16) and the products accumulated in FP32.
// This is the paper's "S := R R^T using a fast rectangular multiplication"
// followed by "A -= S", with S held in tensor memory and subtracted in the
// epilogue instead of being stored.
//
// 1. pack: the FP32 panel is rounded to 16 bits into a dense K-major buffer
//    (rows x Kp, Kp = K rounded up to 64, zero padded), transposing R_U for LU.
// 2. update kernel, one CTA of 128 threads per 128 x 256 output tile:
//      warp 0 lane 0  TMA producer: 128-byte-swizzled 128x64 and 256x64 tiles
//                     into a 4-stage shared-memory ring (mbarrier complete_tx)
//      warp 1 lane 0  MMA issuer: 4 x tcgen05.mma.kind::f16 (M=128, N=256,
//                     K=16) per stage into a 256-column FP32 accumulator in
//                     tensor memory; tcgen05.commit releases the stage
//      all 4 warps    epilogue: tcgen05.ld 32x32b (warp w reads lanes
//                     32w..32w+31 = rows), C -= acc with the lower mask.
//    Every mbarrier wait is bounded by a %globaltimer deadline; on expiry the
//    CTA raises DEV_ERR_TIMEOUT, skips its stores, frees its tensor memory and
//    returns.
#include <cuda.h>  // CUtensorMap and its enums (types only; the encoder is
                   // fetched through the runtime's driver entry point)
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "gb_internal.cuh"

namespace gb {
namespace {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr int THREADS = 128;
constexpr uint32_t TMEM_COLS = 256;
constexpr uint32_t A_STAGE = BM * BK * 2;  // 16 KiB
constexpr uint32_t B_STAGE = BN * BK * 2;  // 32 KiB
constexpr size_t SMEM_BYTES = (size_t)STAGES * (A_STAGE + B_STAGE) + 1024 + 256;

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on phase `parity` of `bar`: false on timeout or abort.
__device__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned long long deadline, int *err,
                          volatile int *abort_flag) {
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (now_ns() > deadline) {
      atomicOr(err, DEV_ERR_TIMEOUT);
      *abort_flag = 1;
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, both K-major, 16-bit inputs, FP32 accumulate.
__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrive on `bar` once every tcgen05 operation this thread issued so far is done.
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// 32 lanes x 32 consecutive 32-bit columns: thread t gets lane (base + t).
__device__ __forceinline__ void tmem_ld_32x32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor of a K-major tile written by TMA with the
// 128-byte swizzle: rows of 64 16-bit elements (128 B), 8-row groups 1024 B
// apart (stride byte offset), descriptor version 1, layout SWIZZLE_128B.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// ---------------------------------------------------------------- kernels
template <bool LOWER>
__global__ void __launch_bounds__(THREADS, 1)
    tc_update_kernel(const __grid_constant__ CUtensorMap map_a,
                     const __grid_constant__ CUtensorMap map_b, float *__restrict__ C, int64_t ldc,
                     int64_t M, int64_t N, int nk, int64_t diag, uint32_t idesc, const int *status,
                     int *err, long long wait_ns, int vec_ok) {
  extern __shared__ uint8_t smem_raw[];
  const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
  if (LOWER && m0 + BM - 1 + diag < n0) return;  // tile strictly above the diagonal
  if (*reinterpret_cast<const volatile int *>(status) != 0) return;
  // a CTA whose wait expired has already raised the error word: later CTAs
  // leave at once instead of waiting out their own deadlines
  if (*reinterpret_cast<const volatile int *>(err) & DEV_ERR_TIMEOUT) return;

  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint8_t *sA = smem;
  uint8_t *sB = smem + STAGES * A_STAGE;
  uint64_t *full = reinterpret_cast<uint64_t *>(sB + STAGES * B_STAGE);
  uint64_t *empty = full + STAGES;
  uint64_t *done = empty + STAGES;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tmem_slot, TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const unsigned long long deadline = now_ns() + (unsigned long long)wait_ns;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------ TMA producer
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
      if (kb >= STAGES && !mbar_wait(&empty[s], ph ^ 1u, deadline, err, abort_flag)) break;
      mbar_expect_tx(&full[s], A_STAGE + B_STAGE);
      tma_load_2d(sA + s * A_STAGE, &map_a, &full[s], kb * BK, (int)m0);
      tma_load_2d(sB + s * B_STAGE, &map_b, &full[s], kb * BK, (int)n0);
    }
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------ MMA issuer
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
      if (!mbar_wait(&full[s], ph, deadline, err, abort_flag)) break;
      tc_fence_after();
      const uint32_t a0 = smem_u32(sA + s * A_STAGE), b0 = smem_u32(sB + s * B_STAGE);
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk)
        mma_f16(tmem, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), idesc,
                (kb | kk) != 0 ? 1u : 0u);
      mma_commit(&empty[s]);
    }
    mma_commit(done);
  }
  __syncwarp();

  // ---------------------------------------------------- epilogue
  const bool ok = mbar_wait(done, 0, deadline, err, abort_flag);
  tc_fence_after();
  const int64_t row = m0 + warp * 32 + lane;
  const bool store = ok && !*abort_flag && row < M;
#pragma unroll 1
  for (int c = 0; c < BN / 32; ++c) {
    const int64_t col0 = n0 + c * 32;
    if (col0 >= N) break;  // uniform over the CTA
    if (LOWER && m0 + BM - 1 + diag < col0) break;
    float v[32];
    tmem_ld_32x32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 32), v);
    if (!store) continue;
    float *crow = C + row * ldc + col0;
    const bool full_row = col0 + 32 <= N && (!LOWER || row + diag >= col0 + 31);
    if (vec_ok && full_row) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        float4 x = *reinterpret_cast<float4 *>(crow + 4 * q);
        x.x -= v[4 * q + 0];
        x.y -= v[4 * q + 1];
        x.z -= v[4 * q + 2];
        x.w -= v[4 * q + 3];
        *reinterpret_cast<float4 *>(crow + 4 * q) = x;
      }
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int64_t col = col0 + j;
        if (col < N && (!LOWER || row + diag >= col)) crow[j] -= v[j];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, TMEM_COLS);
}

template <typename T16>
__device__ __forceinline__ T16 to16(float x);
template <>
__device__ __forceinline__ __nv_bfloat16 to16<__nv_bfloat16>(float x) {
  return __float2bfloat16_rn(x);
}
template <>
__device__ __forceinline__ __half to16<__half>(float x) {
  return __float2half_rn(x);
}

// out[i * Kp + k] = round16(X[i * ldx + k]) for k < K, 0 for K <= k < Kp.
template <typename T16>
__global__ void pack_rows_kernel(const float *__restrict__ X, int64_t ldx, int64_t rows,
                                 int64_t K, int64_t Kp, T16 *__restrict__ out) {
  const int64_t total = rows * Kp;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / Kp, k = e % Kp;
    out[e] = to16<T16>(k < K ? X[i * ldx + k] : 0.0f);
  }
}

// out[j * Kp + k] = round16(Y[k * ldy + j]) (K x N row-major -> N x Kp K-major).
template <typename T16>
__global__ void pack_transpose_kernel(const float *__restrict__ Y, int64_t ldy, int64_t K,
                                      int64_t N, int64_t Kp, T16 *__restrict__ out) {
  __shared__ float t[32][33];
  const int64_t k0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t k = k0 + r, j = j0 + threadIdx.x;
    t[r][threadIdx.x] = (k < K && j < N) ? Y[k * ldy + j] : 0.0f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t j = j0 + r, k = k0 + threadIdx.x;
    if (j < N && k < Kp) out[j * Kp + k] = to16<T16>(t[threadIdx.x][r]);
  }
}

// ------------------------------------------------------------ host helpers
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return (EncodeTiledFn) nullptr;
    }
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// 2-D map over a dense rows x Kp 16-bit K-major buffer, box 64 x box_rows.
bool make_map(CUtensorMap *map, void *base, int64_t rows, int64_t Kp, int box_rows, bool f16) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                   base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

template <typename T16>
cudaError_t pack_operands(const TcUpdateArgs &a, int64_t Kp, T16 *xp, T16 *yp, bool same,
                          cudaStream_t st) {
  const int threads = 256;
  {
    const int64_t total = a.M * Kp;
    const unsigned grid = (unsigned)std::min<int64_t>((total + threads - 1) / threads, 65535 * 4);
    pack_rows_kernel<T16><<<grid, threads, 0, st>>>(a.X, a.ldx, a.M, a.K, Kp, xp);
    count_launch();
  }
  if (!same) {
    if (a.nn) {
      dim3 grid((unsigned)((a.N + 31) / 32), (unsigned)((Kp + 31) / 32));
      pack_transpose_kernel<T16><<<grid, dim3(32, 8), 0, st>>>(a.Y, a.ldy, a.K, a.N, Kp, yp);
    } else {
      const int64_t total = a.N * Kp;
      const unsigned grid = (unsigned)std::min<int64_t>((total + threads - 1) / threads, 65535 * 4);
      pack_rows_kernel<T16><<<grid, threads, 0, st>>>(a.Y, a.ldy, a.N, a.K, Kp, yp);
    }
    count_launch();
  }
  return cudaGetLastError();
}

}  // namespace

bool tc_supported(int device) {
  int major = 0, minor = 0;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return major == 10 && minor == 3 && encode_fn() != nullptr;
}

size_t tc_pack_bytes(int64_t M, int64_t N, int64_t K, bool nn) {
  const int64_t Kp = round_up(std::max<int64_t>(K, 1), BK);
  (void)nn;
  return (size_t)(round_up(M, 8) + round_up(N, 8)) * (size_t)Kp * 2 + 256;
}

cudaError_t launch_update_tc(const TcUpdateArgs &a, cudaStream_t st) {
  if (a.M <= 0 || a.N <= 0 || a.K <= 0) return cudaSuccess;
  int dev = 0;
  cudaGetDevice(&dev);
  if (!tc_supported(dev)) return cudaErrorNotSupported;
  if (a.M > INT32_MAX - BM || a.N > INT32_MAX - BN) return cudaErrorInvalidValue;
  const int64_t Kp = round_up(a.K, BK);
  if (tc_pack_bytes(a.M, a.N, a.K, a.nn) > a.pack_bytes) return cudaErrorInvalidValue;
  const bool same = !a.nn && a.X == a.Y && a.ldx == a.ldy && a.M == a.N;
  uint8_t *base = reinterpret_cast<uint8_t *>(a.pack);
  void *xp = base;
  void *yp = same ? base : base + (size_t)round_up(a.M, 8) * Kp * 2;
  cudaError_t e = a.f16 ? pack_operands<__half>(a, Kp, (__half *)xp, (__half *)yp, same, st)
                        : pack_operands<__nv_bfloat16>(a, Kp, (__nv_bfloat16 *)xp,
                                                       (__nv_bfloat16 *)yp, same, st);
  if (e != cudaSuccess) return e;
  CUtensorMap map_a, map_b;
  if (!make_map(&map_a, xp, a.M, Kp, BM, a.f16) || !make_map(&map_b, yp, a.N, Kp, BN, a.f16))
    return cudaErrorInvalidValue;
  // instruction descriptor: FP32 accumulator, A/B = BF16 (1) or FP16 (0),
  // both K-major, N >> 3 at bit 17, M >> 4 at bit 24
  const uint32_t ab = a.f16 ? 0u : 1u;
  const uint32_t idesc = (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(BN >> 3) << 17) |
                         ((uint32_t)(BM >> 4) << 24);
  const int vec_ok = ((reinterpret_cast<uintptr_t>(a.C) & 15) == 0 && (a.ldc & 3) == 0) ? 1 : 0;
  // a tile takes microseconds; one second bounds every wait of the kernel
  const long long wait_ns = std::min<long long>((long long)a.spin_limit * 100LL, 1000000000LL);
  dim3 grid((unsigned)((a.N + BN - 1) / BN), (unsigned)((a.M + BM - 1) / BM));
  if (grid.y > 65535) return cudaErrorInvalidConfiguration;
  if (a.lower) {
    static cudaError_t attr = cudaFuncSetAttribute(
        tc_update_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    if (attr != cudaSuccess) return attr;
    tc_update_kernel<true><<<grid, THREADS, SMEM_BYTES, st>>>(
        map_a, map_b, a.C, a.ldc, a.M, a.N, (int)(Kp / BK), a.diag, idesc, a.status, a.err,
        wait_ns, vec_ok);
  } else {
    static cudaError_t attr = cudaFuncSetAttribute(
        tc_update_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    if (attr != cudaSuccess) return attr;
    tc_update_kernel<false><<<grid, THREADS, SMEM_BYTES, st>>>(
        map_a, map_b, a.C, a.ldc, a.M, a.N, (int)(Kp / BK), a.diag, idesc, a.status, a.err,
        wait_ns, vec_ok);
  }
  count_launch();
  return cudaGetLastError();
}

}  // namespace gb
