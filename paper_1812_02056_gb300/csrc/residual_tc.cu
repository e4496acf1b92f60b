// Residual r = b - A x of the FP64 iterative refinement (the "r = b - Ax"
// step that brings the low-precision solves back to FP64 accuracy), computed
// to FP64 accuracy from exact integer products on the tensor cores.
//
// Splitting (error-free up to a truncation below 2^-55 of the scale).  Row i
// of A is scaled by sigma_i = 2^e_i, e_i the binary exponent of
// max_j |A_ij| (so |A_ij| / sigma_i < 1), and its fixed-point value is cut
// into RP digits of RW bits:
//   A_ij = sigma_i * sign * sum_{p=0..RP-1} d_p 2^{-RW (p+1)} + t_ij,
//   0 <= d_p < 2^RW,  |t_ij| < 2^{-RW RP} sigma_i = 2^-55 sigma_i.
// Column c of x likewise, with tau_c = 2^f_c.  Each signed digit is an
// integer of magnitude <= 31, stored exactly in BF16 (one plane per digit).
// The digits come from the FP64 bit pattern (sign, exponent, 53-bit
// significand shifted into a 55-bit fixed-point word): integer operations,
// no FP64 arithmetic.
//
// Products.  For each digit pair (p, q) with p + q <= RT the tensor cores
// compute S_pq[i][c] = sum_j a_p[i][j] b_q[j][c] with FP32 accumulation.
// Every product is an integer of magnitude <= 31^2 < 2^10, and over at most
// 2^14 terms of K every partial sum is an integer below 2^24, which FP32
// holds exactly (and the tensor cores' FP32 accumulation keeps exactly), so
// each S_pq is exact.  Then
//   (A x)_ic ~= sigma_i tau_c sum_{p+q<=RT} 2^{-RW (p+q+2)} S_pq[i][c]
// summed in FP64, smallest scales first.  Per term j the truncations and the
// dropped pairs (p + q > RT) are below 2^-53.7 sigma_i tau_c: within one
// FP64 rounding of the largest product of the row, where the plain FP64
// product carries one rounding of u = 2^-53 per product plus the rounding of
// its running sum.
//
// Kernel (one CTA per 128 rows x 16 right-hand sides x K range): warp 0 is
// the TMA producer (3-stage ring: up to three 128 x 64 digit planes of A and
// the 16 x 64 digit planes of x per stage, 128-byte swizzle), warp 1 issues
// tcgen05.mma.kind::f16 (M = 128, N = 16 x the x planes a digit of A pairs
// with) into a 512-column FP32 accumulator in tensor memory, warps 2..5 read
// it back (tcgen05.ld), sum the pairs of one scale exactly in int32 and
// accumulate the scaled sums in FP64.  The 76 pairs need 1216
// accumulator columns, so the digits of A go in four passes of at most three
// (512, 384, 240 and 80 columns), the smallest first.  A K range longer than
// 2^14 (or a small grid) is split over CTAs whose FP64 partial sums are added
// in a fixed order by a second kernel.  Every mbarrier wait is bounded.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "gb_internal.cuh"
#include "digits.cuh"
#include "tc_ptx.cuh"

namespace gb {
namespace {

using namespace tc;
using namespace dg;

constexpr int RT = 11;   // digit pairs kept: p + q <= RT (0-based digits)
constexpr int RBM = 128, RBN = 16, RBK = 64;
constexpr int RSTAGES = 3;
constexpr int RMAXP = 3;                               // digit planes of A per pass
constexpr uint32_t RA_SLOT = RBM * RBK * 2;            // 16 KiB
constexpr uint32_t RB_SLOT = RBN * RBK * 2;            // 2 KiB
constexpr uint32_t RSTAGE = RMAXP * RA_SLOT + RP * RB_SLOT;  // 70 KiB
constexpr size_t RSMEM = (size_t)RSTAGES * RSTAGE + 1024 + 256;
constexpr int RTHREADS = 192;                          // producer, MMA, 4 epilogue warps
constexpr uint32_t RTMEM_COLS = 512;
constexpr int NPASS = 4;
constexpr int64_t RK_MAX = 16384;                      // K per CTA: partial sums below 2^24
static_assert(RSMEM <= 232448, "shared memory per CTA");

// x digits a digit p of A pairs with (p + q <= RT)
__host__ __device__ constexpr int nq_of(int p) { return RT + 1 - p < RP ? RT + 1 - p : RP; }
// passes, smallest digits first: first digit of A and digit count
__host__ __device__ constexpr int pass_first(int k) { return k == 0 ? 9 : k == 1 ? 6 : k == 2 ? 3 : 0; }
__host__ __device__ constexpr int pass_count(int k) { return k == 0 ? 2 : 3; }
// accumulator column of digit p (the j-th of its pass)
__host__ __device__ constexpr int col_of(int k, int j) {
  int c = 0;
  for (int u = 0; u < j; ++u) c += RBN * nq_of(pass_first(k) + u);
  return c;
}
static_assert(col_of(3, 2) + RBN * nq_of(2) <= (int)RTMEM_COLS, "pass 0..2 fits tensor memory");
static_assert(col_of(2, 2) + RBN * nq_of(5) <= (int)RTMEM_COLS, "pass 3..5 fits tensor memory");

// Row scales and ||A||_inf in one read of A: rexp[i] = e_i; *anorm = max_i
// sum_j |A_ij| (NaN or Inf: Inf).  One warp per row; with `vec` (A 16-byte
// aligned, lda even) each lane reads 16 bytes per load, four loads in
// flight.  The largest magnitude is taken on the bit patterns (non-negative
// doubles order like their bits as integers; NaN above Inf), which keeps
// the FP64 pipe for the sum alone.
__global__ void split_rowstats_kernel(const double *__restrict__ A, int64_t lda, int64_t n,
                                      int *__restrict__ rexp, double *anorm, int vec) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (i >= n) return;
  const double *row = A + i * lda;
  constexpr unsigned long long ABS = 0x7fffffffffffffffull;
  double s = 0.0;
  unsigned long long mx = 0;
  int64_t k = 0;
  if (vec) {
    for (; k + 256 <= n; k += 256) {
      double2 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = *reinterpret_cast<const double2 *>(row + k + u * 64 + 2 * lane);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const unsigned long long a = (unsigned long long)__double_as_longlong(v[u].x) & ABS;
        const unsigned long long b = (unsigned long long)__double_as_longlong(v[u].y) & ABS;
        s += __longlong_as_double((long long)a) + __longlong_as_double((long long)b);
        mx = a > mx ? a : mx;
        mx = b > mx ? b : mx;
      }
    }
  }
  for (k += lane; k < n; k += 32) {
    const unsigned long long a = (unsigned long long)__double_as_longlong(row[k]) & ABS;
    s += __longlong_as_double((long long)a);
    mx = a > mx ? a : mx;
  }
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    const unsigned long long m2 = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = m2 > mx ? m2 : mx;
  }
  if (lane == 0) {
    rexp[i] = scale_exp(__longlong_as_double((long long)mx));
    if (anorm) atomic_max_nonneg_r(anorm, finite_abs_r(s));
  }
}

// Digit planes of A: plane p, row i at planes + p * pstride + i * ldk.
// Each thread converts 4 consecutive columns of one row (two 8-byte loads
// with `vec`, one 8-byte store per plane).
__global__ void split_rows_kernel(const double *__restrict__ A, int64_t lda, int64_t n,
                                  const int *__restrict__ rexp, uint16_t *__restrict__ planes,
                                  int64_t ldk, int64_t pstride, int vec) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j0 = g * 4;
  if (j0 >= n) return;
  for (int64_t i = blockIdx.y; i < n; i += gridDim.y) {
    const int e = rexp[i];
    const double *src = A + i * lda + j0;
    double v[4];
    if (vec && j0 + 4 <= n) {
      const double2 a = *reinterpret_cast<const double2 *>(src);
      const double2 b = *reinterpret_cast<const double2 *>(src + 2);
      v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = j0 + u < n ? src[u] : 0.0;
    }
    uint32_t lo[RP], hi[RP];
    digits2(v[0], v[1], e, lo);
    digits2(v[2], v[3], e, hi);
    uint16_t *dst = planes + i * ldk + j0;  // ldk % 4 == 0: 8-byte aligned
#pragma unroll
    for (int p = 0; p < RP; ++p) *reinterpret_cast<uint2 *>(dst + p * pstride) = make_uint2(lo[p], hi[p]);
  }
}

// xmax[c] = max_i |X[i][c]| (NaN or Inf: Inf); xmax zeroed by the caller.
__global__ void split_colmax_kernel(const double *__restrict__ X, int64_t ldx, int64_t n,
                                    int64_t nrhs, double *xmax) {
  const int64_t c = blockIdx.y;
  double mx = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    mx = fmax(mx, finite_abs_r(X[i * ldx + c]));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0.0) atomic_max_nonneg_r(&xmax[c], mx);
}

// Digit planes of x, transposed: plane q, right-hand side c at
// planes + q * pstride + c * ldk (K-major rows of the MMA's B operand).
__global__ void split_cols_kernel(const double *__restrict__ X, int64_t ldx, int64_t n,
                                  int64_t nrhs, const double *__restrict__ xmax,
                                  uint16_t *__restrict__ planes, int64_t ldk, int64_t pstride) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t c = blockIdx.y;
  if (j >= n) return;
  uint32_t d[RP];
  digits2(X[j * ldx + c], 0.0, scale_exp(xmax[c]), d);
#pragma unroll
  for (int q = 0; q < RP; ++q) planes[q * pstride + c * ldk + j] = (uint16_t)(d[q] & 0xffffu);
}


// The product kernel.  Grid: (row tiles of 128, groups of 16 right-hand
// sides, K ranges of `kchunk` columns).  With one K range it writes
// r = b - A x and the norms of r and b (max per column, by atomics; the
// norm of x is `xmax`); with several, the FP64 partial sums
// P[z][i][c] (the scaled digit sums, before sigma_i tau_c) for
// split_finish_kernel.
__global__ void __launch_bounds__(RTHREADS, 1)
    residual_split_kernel(const __grid_constant__ CUtensorMap map_a,
                          const __grid_constant__ CUtensorMap map_b, const int *__restrict__ rexp,
                          const double *__restrict__ xmax, const double *__restrict__ B,
                          int64_t ldb, double *__restrict__ R, int64_t ldr, int64_t n,
                          int64_t nrhs, int64_t kchunk, double *__restrict__ P, double *norms,
                          int *err, long long wait_ns) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + RSTAGES * RSTAGE);
  uint64_t *empty = full + RSTAGES;
  uint64_t *acc_full = empty + RSTAGES;
  uint64_t *acc_empty = acc_full + 1;
  uint64_t *drain = acc_empty + 1;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < RSTAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, 4);  // the four epilogue warps
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc<1>(tmem_slot, RTMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const unsigned long long deadline = (unsigned long long)wait_ns;

  const int m0 = (int)blockIdx.x * RBM;
  const int c0 = (int)blockIdx.y * RBN;
  const int64_t nkb = (n + RBK - 1) / RBK;
  const int kb0 = (int)(blockIdx.z * (kchunk / RBK));
  const int kb1 = (int)min64(nkb, kb0 + kchunk / RBK);

  if (warp == 0) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      uint32_t g = 0;
      bool ok = true;
#pragma unroll
      for (int k = 0; k < NPASS; ++k) {
        const int p0 = pass_first(k), np = pass_count(k), nb = nq_of(p0);
        const uint32_t bytes = np * RA_SLOT + nb * RB_SLOT;
        for (int kb = kb0; ok && kb < kb1; ++kb, ++g) {
          const uint32_t s = g % RSTAGES, ph = (g / RSTAGES) & 1u;
          if (g >= (uint32_t)RSTAGES && !mbar_wait(&empty[s], ph ^ 1u, deadline, err, abort_flag)) {
            ok = false;
            break;
          }
          uint8_t *st = smem + s * RSTAGE;
          mbar_expect_tx(&full[s], bytes);
          for (int j = 0; j < np; ++j)
            tma_load_3d(st + j * RA_SLOT, &map_a, &full[s], kb * RBK, m0, p0 + j);
          for (int q = 0; q < nb; ++q)
            tma_load_3d(st + RMAXP * RA_SLOT + q * RB_SLOT, &map_b, &full[s], kb * RBK, c0, q);
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t g = 0;
      bool ok = true;
#pragma unroll
      for (int k = 0; k < NPASS; ++k) {
        if (!ok) break;
        const int p0 = pass_first(k), np = pass_count(k);
        if (k > 0 && !mbar_wait(acc_empty, (k - 1) & 1u, deadline, err, abort_flag)) break;
        tc_fence_after();
        for (int kb = kb0; kb < kb1; ++kb, ++g) {
          const uint32_t s = g % RSTAGES, ph = (g / RSTAGES) & 1u;
          if (!mbar_wait(&full[s], ph, deadline, err, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = smem_u32(smem + s * RSTAGE);
          const uint32_t b0 = st + RMAXP * RA_SLOT;
#pragma unroll
          for (int j = 0; j < RMAXP; ++j) {
            if (j >= np) break;
            const int nn = RBN * nq_of(p0 + j);
            // FP32 accumulator, BF16 A and B, both K-major, N >> 3, M >> 4
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) |
                                   ((uint32_t)(nn >> 3) << 17) | ((uint32_t)(RBM >> 4) << 24);
            const uint32_t d = tmem + (uint32_t)col_of(k, j);
            const uint32_t a0 = st + j * RA_SLOT;
#pragma unroll
            for (int kk = 0; kk < RBK / 16; ++kk)
              mma_f16<1>(d, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), idesc,
                         (kb != kb0 || kk != 0) ? 1u : 0u);
          }
          mma_commit(&empty[s]);
        }
        if (!ok) break;
        mma_commit(acc_full);
      }
      // every MMA is done before the tensor memory is released
      mma_commit(drain);
      const unsigned long long until = now_ns() + deadline;
      while (!mbar_try_wait(drain, 0)) {
        if (now_ns() > until) {
          atomicOr(err, DEV_ERR_TIMEOUT);
          break;
        }
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------ epilogue (warps 2..5)
    const int qd = warp & 3;  // tensor-memory lane quarter this warp may read
    const int64_t row = (int64_t)m0 + qd * 32 + lane;
    double acc[RBN];
    float chk[RBN];
#pragma unroll
    for (int c = 0; c < RBN; ++c) acc[c] = 0.0, chk[c] = 0.0f;
    bool ok = true;
#pragma unroll
    for (int k = 0; k < NPASS; ++k) {
      if (!mbar_wait(acc_full, k & 1u, deadline, err, abort_flag)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const int p0 = pass_first(k), np = pass_count(k);
      // Pairs of one scale t = p + q (at most one per digit of the pass)
      // are summed exactly in int32 (each |S| < 2^24), then scaled into the
      // FP64 sum: smallest scales first.  `chk` carries a NaN or Inf of a
      // non-finite input through (the integer sums cannot).
#pragma unroll 1
      for (int t = RT; t >= p0; --t) {
        int32_t si[RBN];
        bool any = false;
#pragma unroll
        for (int j = 0; j < RMAXP; ++j) {
          const int p = p0 + j, q = t - p;
          if (j >= np || q < 0 || q >= nq_of(p)) continue;
          float v[RBN];
          tmem_ld_32x16(tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(col_of(k, j) + q * RBN), v);
#pragma unroll
          for (int c = 0; c < RBN; ++c) {
            const int32_t iv = __float2int_rn(v[c]);
            si[c] = any ? si[c] + iv : iv;
            chk[c] += v[c];
          }
          any = true;
        }
        if (!any) continue;
        const double sc = pow2_neg(RW * (t + 2));
#pragma unroll
        for (int c = 0; c < RBN; ++c) acc[c] = fma((double)si[c], sc, acc[c]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty);
    }
    if (ok && !*abort_flag) {
#pragma unroll
      for (int c = 0; c < RBN; ++c)
        if (!(fabsf(chk[c]) <= 3.4e38f)) acc[c] = (double)chk[c];  // NaN or Inf through
      const int cols = (int)min64(RBN, nrhs - c0);
      if (P) {
        if (row < n) {
          double *dst = P + ((int64_t)blockIdx.z * n + row) * nrhs + c0;
#pragma unroll
          for (int c = 0; c < RBN; ++c)
            if (c < cols) dst[c] = acc[c];
        }
      } else {
        const int ei = row < n ? rexp[row] : 0;
#pragma unroll
        for (int c = 0; c < RBN; ++c) {
          double rn = 0.0, bn = 0.0;
          if (c < cols && row < n) {
            const double b = B[row * ldb + c0 + c];
            const double rv = b - ldexp(acc[c], ei + scale_exp(xmax[c0 + c]));
            R[row * ldr + c0 + c] = rv;
            rn = finite_abs_r(rv);
            bn = finite_abs_r(b);
          }
          for (int o = 16; o > 0; o >>= 1) {
            rn = fmax(rn, __shfl_xor_sync(0xffffffffu, rn, o));
            bn = fmax(bn, __shfl_xor_sync(0xffffffffu, bn, o));
          }
          if (lane == 0 && c < cols && norms) {
            atomic_max_nonneg_r(&norms[c0 + c], rn);
            atomic_max_nonneg_r(&norms[2 * nrhs + c0 + c], bn);
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc<1>(tmem, RTMEM_COLS);
}

// r = b - sigma_i tau_c (P[0] + P[1] + ...), the K ranges summed in order;
// the norms of r and b as in residual_split_kernel.
__global__ void split_finish_kernel(const double *__restrict__ P, int parts,
                                    const int *__restrict__ rexp, const double *__restrict__ xmax,
                                    const double *__restrict__ B, int64_t ldb,
                                    double *__restrict__ R, int64_t ldr, int64_t n, int64_t nrhs,
                                    double *norms) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * nrhs) return;
  const int64_t i = e / nrhs, c = e % nrhs;
  double acc = P[e];
  for (int z = 1; z < parts; ++z) acc += P[(int64_t)z * n * nrhs + e];
  const double b = B[i * ldb + c];
  const double rv = b - ldexp(acc, rexp[i] + scale_exp(xmax[c]));
  R[i * ldr + c] = rv;
  if (norms) {
    atomic_max_nonneg_r(&norms[c], finite_abs_r(rv));
    atomic_max_nonneg_r(&norms[2 * nrhs + c], finite_abs_r(b));
  }
}

// ------------------------------------------------------------ host side
int64_t split_ldk(int64_t n) { return (n + 63) / 64 * 64; }
size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// 3-D map over RP planes of rows x K BF16 digits (K-major rows of ldk), box
// 64 x box_rows x 1 with the 128-byte swizzle; reads beyond K or rows give 0.
bool make_plane_map(CUtensorMap *map, const void *base, int64_t K, int64_t rows, int64_t ldk,
                    int box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)RP};
  cuuint64_t strides[2] = {(cuuint64_t)ldk * 2, (cuuint64_t)rows * ldk * 2};
  cuuint32_t box[3] = {(cuuint32_t)RBK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims,
                   strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// K ranges per row tile: as many as keep the CTAs within one wave (one CTA
// per SM), each range at least 16 k-blocks, and no range longer than RK_MAX.
int split_parts(int64_t n, int64_t nrhs, int sm_count, int64_t *kchunk) {
  const int64_t nkb = (n + RBK - 1) / RBK;
  const int64_t tiles = ((n + RBM - 1) / RBM) * ((nrhs + RBN - 1) / RBN);
  int64_t parts = std::max<int64_t>(1, std::min<int64_t>(sm_count / tiles, nkb / 16));
  parts = std::max<int64_t>(parts, (n + RK_MAX - 1) / RK_MAX);
  const int64_t kbs = (nkb + parts - 1) / parts;
  *kchunk = kbs * RBK;
  return (int)((nkb + kbs - 1) / kbs);
}

}  // namespace

size_t split_a_bytes(int64_t n) {
  return align256((size_t)RP * n * split_ldk(n) * 2) + align256((size_t)n * sizeof(int));
}

size_t split_x_bytes(int64_t n, int64_t nrhs, int sm_count) {
  int64_t kchunk;
  const int parts = split_parts(n, nrhs, sm_count, &kchunk);
  return align256((size_t)RP * nrhs * split_ldk(n) * 2) +
         (parts > 1 ? (size_t)parts * n * nrhs * sizeof(double) : 0);
}

cudaError_t launch_split_a(const double *A, int64_t lda, int64_t n, void *work, double *anorm,
                           cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  uint16_t *planes = reinterpret_cast<uint16_t *>(work);
  int *rexp = reinterpret_cast<int *>((char *)work + align256((size_t)RP * n * split_ldk(n) * 2));
  if (anorm) {
    cudaError_t e = cudaMemsetAsync(anorm, 0, sizeof(double), st);
    if (e != cudaSuccess) return e;
  }
  const int vec = ((reinterpret_cast<uintptr_t>(A) & 15) == 0 && (lda & 1) == 0) ? 1 : 0;
  split_rowstats_kernel<<<(unsigned)ceil_div(n, 8), 256, 0, st>>>(A, lda, n, rexp, anorm, vec);
  count_launch();
  const int64_t groups = (n + 3) / 4;
  const dim3 grid((unsigned)ceil_div(groups, 128), (unsigned)std::min<int64_t>(n, 65535));
  split_rows_kernel<<<grid, 128, 0, st>>>(A, lda, n, rexp, planes, split_ldk(n),
                                          n * split_ldk(n), vec);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_residual_split(const void *awork, int64_t n, const double *X, int64_t ldx,
                                  const double *B, int64_t ldb, double *R, int64_t ldr,
                                  int64_t nrhs, double *norms, void *xwork, int sm_count, int *err,
                                  long long wait_ns, cudaStream_t st) {
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  const int64_t ldk = split_ldk(n);
  const uint16_t *aplanes = reinterpret_cast<const uint16_t *>(awork);
  const int *rexp =
      reinterpret_cast<const int *>((const char *)awork + align256((size_t)RP * n * ldk * 2));
  uint16_t *xplanes = reinterpret_cast<uint16_t *>(xwork);
  int64_t kchunk;
  const int parts = split_parts(n, nrhs, sm_count, &kchunk);
  double *P = parts > 1 ? reinterpret_cast<double *>(
                              (char *)xwork + align256((size_t)RP * nrhs * ldk * 2))
                        : nullptr;
  double *xmax = norms + nrhs;
  cudaError_t e = cudaMemsetAsync(norms, 0, sizeof(double) * 3 * nrhs, st);
  if (e != cudaSuccess) return e;
  split_colmax_kernel<<<dim3((unsigned)std::min<int64_t>(ceil_div(n, 256), 64), (unsigned)nrhs),
                        256, 0, st>>>(X, ldx, n, nrhs, xmax);
  count_launch();
  split_cols_kernel<<<dim3((unsigned)ceil_div(n, 256), (unsigned)nrhs), 256, 0, st>>>(
      X, ldx, n, nrhs, xmax, xplanes, ldk, nrhs * ldk);
  count_launch();
  CUtensorMap ma, mb;
  if (!make_plane_map(&ma, aplanes, n, n, ldk, RBM) ||
      !make_plane_map(&mb, xplanes, n, nrhs, ldk, RBN))
    return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    e = cudaFuncSetAttribute(residual_split_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)RSMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const dim3 grid((unsigned)ceil_div(n, RBM), (unsigned)ceil_div(nrhs, RBN), (unsigned)parts);
  residual_split_kernel<<<grid, RTHREADS, RSMEM, st>>>(ma, mb, rexp, xmax, B, ldb, R, ldr, n,
                                                       nrhs, kchunk, P, norms, err, wait_ns);
  count_launch();
  if (parts > 1) {
    split_finish_kernel<<<(unsigned)ceil_div(n * nrhs, 256), 256, 0, st>>>(
        P, parts, rexp, xmax, B, ldb, R, ldr, n, nrhs, norms);
    count_launch();
  }
  return cudaGetLastError();
}

}  // namespace gb
