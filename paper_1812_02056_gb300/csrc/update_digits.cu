// The delayed rank-s update of Algorithm 1 in FP64 (arXiv:1812.02056,
// Sec. 2: "A -= S, S = R R^T") to FP64 accuracy on the tensor cores:
//   C (FP64) -= X Y^T     (Cholesky: lower, j <= i; X M x K, Y N x K rows)
//   C (FP64) -= X Y       (LU: every element; Y K x N, cut by columns)
// from exact products of the operands' digits (digits.cuh): row i of X is
// cut into RP = 11 signed 5-bit digits a_p[i][.] at scale 2^e_i, row j of Y
// likewise (b_q[j][.], 2^f_j), and
//   (X Y^T)_ij ~= 2^(e_i + f_j) sum_{t = 0..UT} 2^(-5 (t + 2)) D_t[i][j],
//   D_t = sum_{p + q = t} a_p b_q^T.
// Every digit product is an integer below 2^10; a D_t sums at most 11 pairs
// over K <= UK_MAX = 1024 terms, so every partial sum is an integer below
// 11 * 1024 * 961 < 2^24 and the tensor cores' FP32 accumulation keeps it
// exactly.  The D_t of a tile are combined exactly in 64-bit integers, four
// at a time, converted to FP64 and subtracted from C.  Per
// term of K the truncation of both operands (below 2^-55 of their row
// scales) and the dropped pairs (t > UT) stay below one FP64 rounding of
// 2^(e_i + f_j); the plain FP64 update rounds at every one of its K
// multiply-adds.
//
// Kernel: persistent CTAs over the valid 128 x 64 output tiles (lower
// trapezoid, dealt round-robin).  Warp 0 is the TMA producer (2-stage ring;
// a stage holds up to three 128 x 64 digit planes of X and up to seven
// 64 x 64 digit planes of Y that they pair with, 128-byte swizzle); warp 1
// issues tcgen05.mma.kind::f16 (M = 128, N = 64, K = 16); warps 2..5 are the
// epilogue.  The twelve scales go in three passes of four (0..3, 4..7,
// 8..11), each pass into a set of four 64-column FP32 accumulators in tensor
// memory; two sets alternate, so one pass's epilogue overlaps the next
// pass's MMAs.  The epilogue reads a set back (tcgen05.ld), folds its four
// scales exactly into one 64-bit integer per element and subtracts it from
// C (three roundings of C per tile), C loaded ahead and written through a
// transpose in shared memory (16 lanes per row, coalesced).  Every mbarrier
// wait is bounded; a failed column step (`status`) or an expired wait skips
// the work.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "digits.cuh"
#include "gb_internal.cuh"
#include "tc_ptx.cuh"

namespace gb {
namespace {

using namespace tc;
using namespace dg;

constexpr int UT = 11;                   // scales kept: t = p + q <= UT
constexpr int USC = 4;                   // scales per pass: 0..3, 4..7, 8..11
constexpr int UNP = 3;                   // scale passes per tile
constexpr int UBM = 128, UBN = 64, UBK = 64;
constexpr int USTAGES = 2;
constexpr uint32_t UA_SLOT = UBM * UBK * 2;  // 16 KiB: a 128 x 64 digit plane of X
constexpr uint32_t UB_SLOT = UBN * UBK * 2;  // 8 KiB: a 64 x 64 digit plane of Y
constexpr int UMAXA = 3, UMAXB = 7;          // planes per stage
constexpr uint32_t USTAGE = UMAXA * UA_SLOT + UMAXB * UB_SLOT;  // 104 KiB
constexpr int UTP = 17;                  // pitch (doubles) of an epilogue warp's 32 x 16 block
constexpr uint32_t UEPI = 4 * 32 * UTP * 8;  // the four epilogue warps' blocks
constexpr size_t USMEM = (size_t)USTAGES * USTAGE + UEPI + 1024 + 256;
constexpr int UTHREADS = 192;
constexpr uint32_t UTMEM_COLS = 512;     // two sets of four 64-column accumulators
constexpr uint32_t UACC = USC * UBN;     // columns of one set (256)
constexpr int64_t UK_MAX = 1024;         // K per launch: D_t partial sums below 2^24
static_assert(USMEM <= 232448, "shared memory per CTA");
static_assert(2 * UACC <= UTMEM_COLS, "two accumulator sets fit tensor memory");

// The streams of a tile: (scale pass, first digit of X, digits of X, first
// digit of Y, digits of Y).  Each runs over the tile's K range; together
// they hold every pair (p, q) with p + q <= UT exactly once, in the scale
// pass of p + q, and no stage needs more than UMAXA + UMAXB planes.
constexpr int USTREAMS = 9;
__host__ __device__ constexpr int us_pass(int i) { return i < 2 ? 0 : i < 5 ? 1 : 2; }
__host__ __device__ constexpr int us_p0(int i) {
  return i == 0 ? 0 : i == 1 ? 3 : i == 2 ? 0 : i == 3 ? 3 : i == 4 ? 6
       : i == 5 ? 0 : i == 6 ? 3 : i == 7 ? 6 : 9;
}
__host__ __device__ constexpr int us_np(int i) {
  return i == 1 ? 1 : (i == 4 || i == 8) ? 2 : 3;
}
__host__ __device__ constexpr int us_q0(int i) {
  return i == 2 ? 2 : i == 5 ? 6 : i == 6 ? 3 : 0;
}
__host__ __device__ constexpr int us_nq(int i) {
  return i == 0 ? 4 : i == 1 ? 1 : i == 2 ? 6 : i == 3 ? 5 : i == 4 ? 2
       : i == 5 ? 5 : i == 6 ? 6 : i == 7 ? 6 : 3;
}

// Digits of the rows of X (M x K, ldx): planes[p][i][k] (row pitch kp), and
// the row scale exponents.  One warp per row; lane l converts columns
// 2l, 2l + 1, 2l + 64, ... (two digits per 4-byte store).
__global__ void digits_rows_kernel(const double *__restrict__ X, int64_t ldx, int64_t M,
                                   int64_t K, uint16_t *__restrict__ planes, int64_t kp,
                                   int64_t pstride, int *__restrict__ rexp, const int *status) {
  if (status && *reinterpret_cast<const volatile int *>(status) != 0) return;
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (i >= M) return;
  const double *row = X + i * ldx;
  constexpr unsigned long long ABS = 0x7fffffffffffffffull;
  unsigned long long mx = 0;
  for (int64_t k = lane; k < K; k += 32) {
    const unsigned long long a = (unsigned long long)__double_as_longlong(row[k]) & ABS;
    mx = a > mx ? a : mx;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long m2 = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = m2 > mx ? m2 : mx;
  }
  const int e = scale_exp(__longlong_as_double((long long)mx));
  if (lane == 0) rexp[i] = e;
  uint16_t *dst = planes + i * kp;
  for (int64_t k = 2 * lane; k < K; k += 64) {
    uint32_t d[RP];
    digits2(row[k], k + 1 < K ? row[k + 1] : 0.0, e, d);
    if (k + 1 < K) {  // kp even, k even: 4-byte aligned
#pragma unroll
      for (int p = 0; p < RP; ++p) *reinterpret_cast<uint32_t *>(dst + p * pstride + k) = d[p];
    } else {
#pragma unroll
      for (int p = 0; p < RP; ++p) dst[p * pstride + k] = (uint16_t)(d[p] & 0xffffu);
    }
  }
}

// Digits of the columns of Y (K x N, ldy, row-major: column j of Y is row
// j of the B operand): planes[q][j][k] (row pitch kp), and the column scale
// exponents.  One CTA of 256 threads per 32 columns: the scales from
// coalesced row reads, then 64 x 32 tiles transposed in shared memory so
// that each warp writes consecutive k of one column (two digits per
// 4-byte store).
__global__ void __launch_bounds__(256)
    digits_cols_kernel(const double *__restrict__ Y, int64_t ldy, int64_t N, int64_t K,
                       uint16_t *__restrict__ planes, int64_t kp, int64_t pstride,
                       int *__restrict__ cexp, const int *status) {
  if (status && *reinterpret_cast<const volatile int *>(status) != 0) return;
  __shared__ double tile[64][33];
  __shared__ unsigned long long smax[8][32];
  __shared__ int se[32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t j0 = (int64_t)blockIdx.x * 32, j = j0 + tx;
  constexpr unsigned long long ABS = 0x7fffffffffffffffull;
  unsigned long long mx = 0;
  if (j < N)
    for (int64_t k = ty; k < K; k += 8) {
      const unsigned long long a = (unsigned long long)__double_as_longlong(Y[k * ldy + j]) & ABS;
      mx = a > mx ? a : mx;
    }
  smax[ty][tx] = mx;
  __syncthreads();
  if (ty == 0) {
    for (int t = 1; t < 8; ++t) mx = smax[t][tx] > mx ? smax[t][tx] : mx;
    const int e = scale_exp(__longlong_as_double((long long)mx));
    se[tx] = e;
    if (j < N) cexp[j] = e;
  }
  __syncthreads();
  for (int64_t k0 = 0; k0 < K; k0 += 64) {
    for (int r = ty; r < 64; r += 8)
      tile[r][tx] = (k0 + r < K && j < N) ? Y[(k0 + r) * ldy + j] : 0.0;
    __syncthreads();
    const int64_t k = k0 + 2 * tx;
    for (int c = ty; c < 32; c += 8) {
      const int64_t jc = j0 + c;
      if (jc < N && k < K) {
        uint32_t d[RP];
        digits2(tile[2 * tx][c], tile[2 * tx + 1][c], se[c], d);
        uint16_t *dst = planes + jc * kp + k;
        if (k + 1 < K) {  // kp even, k even: 4-byte aligned
#pragma unroll
          for (int p = 0; p < RP; ++p) *reinterpret_cast<uint32_t *>(dst + p * pstride) = d[p];
        } else {
#pragma unroll
          for (int p = 0; p < RP; ++p) dst[p * pstride] = (uint16_t)(d[p] & 0xffffu);
        }
      }
    }
    __syncthreads();
  }
}

// The valid tiles of the lower trapezoid (M x N, j <= i; row tile bi of UBM
// rows holds min(ntj, 2 bi + 2) column tiles of UBN), or of the whole
// rectangle, counted row by row; index v goes to the CTA v mod gridDim.x.
struct UTileIter {
  int64_t v, total, ntj, bi, base;
  int lower;  // 0: every tile of the M x N rectangle
  __device__ int64_t count(int64_t b) const {
    if (!lower) return ntj;
    const int64_t c = (b * UBM + UBM - 1) / UBN + 1;
    return c < ntj ? c : ntj;
  }
  __device__ bool next(int64_t &m0, int64_t &n0) {
    if (v >= total) return false;
    while (v >= base + count(bi)) {
      base += count(bi);
      ++bi;
    }
    m0 = bi * UBM;
    n0 = (v - base) * UBN;
    v += gridDim.x;
    return true;
  }
};

__global__ void __launch_bounds__(UTHREADS, 1)
    update_digits_kernel(const __grid_constant__ CUtensorMap map_a,
                         const __grid_constant__ CUtensorMap map_b, const int *__restrict__ ea,
                         const int *__restrict__ eb, double *__restrict__ C, int64_t ldc,
                         int64_t M, int64_t N, int nkb, int64_t total, int lower,
                         const int *status, int *err, long long wait_ns) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  double *sT = reinterpret_cast<double *>(smem + USTAGES * USTAGE);  // epilogue transposes
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + USTAGES * USTAGE + UEPI);
  uint64_t *empty = full + USTAGES;
  uint64_t *acc_full = empty + USTAGES;    // per accumulator set
  uint64_t *acc_empty = acc_full + 2;
  uint64_t *drain = acc_empty + 2;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  volatile int *skip = abort_flag + 1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < USTAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);  // the four epilogue warps
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    // skip the work after a failed column step or an expired wait
    *skip = (*reinterpret_cast<const volatile int *>(status) != 0 ||
             (*reinterpret_cast<const volatile int *>(err) & DEV_ERR_TIMEOUT))
                ? 1
                : 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc<1>(tmem_slot, UTMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const unsigned long long deadline = (unsigned long long)wait_ns;
  const int64_t ntj = (N + UBN - 1) / UBN;
  UTileIter it{(int64_t)blockIdx.x, total, ntj, 0, 0, lower};
  int64_t m0 = 0, n0 = 0;

  if (*skip) {
    // nothing issued: straight to the teardown
  } else if (warp == 0) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      uint32_t g = 0;
      bool ok = true;
      while (ok && it.next(m0, n0)) {
#pragma unroll
        for (int si = 0; si < USTREAMS; ++si) {
          const int p0 = us_p0(si), np = us_np(si), q0 = us_q0(si), nq = us_nq(si);
          const uint32_t bytes = np * UA_SLOT + nq * UB_SLOT;
          for (int kb = 0; ok && kb < nkb; ++kb, ++g) {
            const uint32_t s = g % USTAGES, ph = (g / USTAGES) & 1u;
            if (g >= (uint32_t)USTAGES && !mbar_wait(&empty[s], ph ^ 1u, deadline, err, abort_flag)) {
              ok = false;
              break;
            }
            uint8_t *st = smem + s * USTAGE;
            mbar_expect_tx(&full[s], bytes);
            for (int j = 0; j < np; ++j)
              tma_load_3d(st + j * UA_SLOT, &map_a, &full[s], kb * UBK, (int)m0, p0 + j);
            for (int q = 0; q < nq; ++q)
              tma_load_3d(st + UMAXA * UA_SLOT + q * UB_SLOT, &map_b, &full[s], kb * UBK, (int)n0,
                          q0 + q);
          }
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      // FP32 accumulator, BF16 A and B, both K-major, N = 64, M = 128
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(UBN >> 3) << 17) |
                             ((uint32_t)(UBM >> 4) << 24);
      uint32_t g = 0, i = 0;  // i: scale passes issued; pass i uses set i & 1
      bool ok = true;
      while (ok && it.next(m0, n0)) {
        uint32_t started = 0;  // accumulators written in this scale pass
        uint32_t dset = 0;
#pragma unroll
        for (int si = 0; si < USTREAMS; ++si) {
          const int pass = us_pass(si);
          if (si == 0 || pass != us_pass(si - 1)) {
            // a new scale pass: the epilogue of pass i - 2 has freed its set
            if (i >= 2 && !mbar_wait(&acc_empty[i & 1u], ((i >> 1) - 1) & 1u, deadline, err,
                                     abort_flag)) {
              ok = false;
              break;
            }
            tc_fence_after();
            started = 0;
            dset = (i & 1u) * UACC;
          }
          const int p0 = us_p0(si), np = us_np(si), q0 = us_q0(si), nq = us_nq(si);
          const int tlo = pass * USC, thi = tlo + USC - 1;
          for (int kb = 0; ok && kb < nkb; ++kb, ++g) {
            const uint32_t s = g % USTAGES, ph = (g / USTAGES) & 1u;
            if (!mbar_wait(&full[s], ph, deadline, err, abort_flag)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t st = smem_u32(smem + s * USTAGE);
            const uint32_t b0 = st + UMAXA * UA_SLOT;
            for (int j = 0; j < np; ++j) {
              const int p = p0 + j;
              const uint32_t a0 = st + j * UA_SLOT;
              const int qa = max(q0, tlo - p), qb = min(q0 + nq - 1, thi - p);
              for (int q = qa; q <= qb; ++q) {
                const int t = p + q - tlo;
                const uint32_t d = tmem + dset + (uint32_t)(t * UBN);
                const uint32_t bq = b0 + (q - q0) * UB_SLOT;
#pragma unroll
                for (int kk = 0; kk < UBK / 16; ++kk) {
                  mma_f16<1>(d, sw128_desc(a0 + kk * 32), sw128_desc(bq + kk * 32), idesc,
                             (started >> t) & 1u);
                  started |= 1u << t;
                }
              }
            }
            mma_commit(&empty[s]);
          }
          if (!ok) break;
          if (si == USTREAMS - 1 || us_pass(si + 1) != pass) {  // the scale pass is complete
            mma_commit(&acc_full[i & 1u]);
            ++i;
          }
        }
      }
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
    double *blk = sT + (warp - 2) * 32 * UTP;
    uint32_t i = 0;
    bool ok = true;
    while (ok && it.next(m0, n0)) {
      // row m0 + 32 qd + lane is this thread's in tensor memory; C is then
      // written through a transpose in shared memory, 16 lanes per row
      const int64_t r0 = m0 + qd * 32;
      const int e_r = r0 + lane < M ? ea[r0 + lane] : 0;  // row scales, shared by shuffles
      for (int pass = 0; pass < UNP; ++pass, ++i) {
        if (!mbar_wait(&acc_full[i & 1u], (i >> 1) & 1u, deadline, err, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const int thi = pass * USC + USC - 1;
        const uint32_t dset = (i & 1u) * UACC;
#pragma unroll 1
        for (int h = 0; h < UBN / 16; ++h) {
          // this lane's 16 entries of C for the chunk (row 2 it2 + lane / 16,
          // column lane % 16), loaded first: they arrive while the
          // accumulators are read and folded
          const int cl = lane & 15;
          const int64_t j = n0 + h * 16 + cl;
          double cv[16];
#pragma unroll
          for (int it2 = 0; it2 < 16; ++it2) {
            const int64_t row = r0 + 2 * it2 + (lane >> 4);
            cv[it2] = (row < M && j < N && (!lower || j <= row)) ? C[row * ldc + j] : 0.0;
          }
          // the pass's six scales folded exactly: v = sum S_t 2^(5 (thi - t)),
          // below 2^50; its weight is 2^(-5 (thi + 2))
          long long v[16];
          uint32_t bad = 0;  // columns with a non-finite sum (from a non-finite input)
#pragma unroll
          for (int c = 0; c < 16; ++c) v[c] = 0;
#pragma unroll
          for (int t = 0; t < USC; ++t) {
            float w[16];
            tmem_ld_32x16(tmem + ((uint32_t)(qd * 32) << 16) + dset + (uint32_t)(t * UBN + h * 16),
                          w);
#pragma unroll
            for (int c = 0; c < 16; ++c) {
              // every finite sum is an integer below 2^24: NaN or Inf otherwise
              bad |= (fabsf(w[c]) < 3.0e7f ? 0u : 1u) << c;
              v[c] = v[c] * 32 + (long long)__float2int_rn(w[c]);
            }
          }
#pragma unroll
          for (int c = 0; c < 16; ++c)
            blk[lane * UTP + c] = ((bad >> c) & 1u) ? __longlong_as_double(0x7ff8000000000000LL)
                                                     : (double)v[c];
          __syncwarp();
          const int e_j = j < N ? eb[j] : 0;
          if (!*abort_flag) {
#pragma unroll
            for (int it2 = 0; it2 < 16; ++it2) {
              const int r = 2 * it2 + (lane >> 4);
              const int64_t row = r0 + r;
              const int e = __shfl_sync(0xffffffffu, e_r, r) + e_j - RW * (thi + 2);
              if (row < M && j < N && (!lower || j <= row)) {
                const double sc = __longlong_as_double((long long)(1023 + e) << 52);
                C[row * ldc + j] = cv[it2] - blk[r * UTP + cl] * sc;
              }
            }
          }
          __syncwarp();
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[i & 1u]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc<1>(tmem, UTMEM_COLS);
}

int64_t digits_kp(int64_t K) { return (K + 7) / 8 * 8; }
size_t align256u(size_t b) { return (b + 255) / 256 * 256; }

// 3-D map over RP planes of rows x K BF16 digits (row pitch kp), box 64 x
// box_rows x 1, 128-byte swizzle; reads beyond K or rows give 0.
bool make_digit_map(CUtensorMap *map, const void *base, int64_t K, int64_t rows, int64_t kp,
                    int box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)RP};
  cuuint64_t strides[2] = {(cuuint64_t)kp * 2, (cuuint64_t)rows * kp * 2};
  cuuint32_t box[3] = {(cuuint32_t)UBK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims,
                   strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

size_t digit_set_bytes(int64_t rows, int64_t K) {
  const int64_t k = std::min<int64_t>(K, UK_MAX);
  return align256u((size_t)RP * rows * digits_kp(k) * 2) + align256u((size_t)rows * sizeof(int));
}

}  // namespace

size_t update_digits_bytes(int64_t M, int64_t N, int64_t K, bool same) {
  return digit_set_bytes(M, K) + (same ? 0 : digit_set_bytes(N, K));
}

cudaError_t launch_update_digits(double *C, int64_t ldc, const double *X, int64_t ldx,
                                 const double *Y, int64_t ldy, int64_t M, int64_t N, int64_t K,
                                 bool lower, bool y_kxn, const int *status, int *err,
                                 int64_t spin_limit, void *work, size_t work_bytes, int max_ctas,
                                 cudaStream_t st) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  // Y's rows are X's first N rows (a Cholesky update): one set of digits
  const bool same = !y_kxn && X == Y && ldx == ldy && N <= M;
  if (!work || work_bytes < update_digits_bytes(M, N, K, same)) return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(update_digits_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)USMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  // a launch takes milliseconds; one second bounds every single wait
  const long long wait_ns = std::min<long long>((long long)spin_limit * 100LL, 1000000000LL);
  const int64_t nbi = (M + UBM - 1) / UBM, ntj = (N + UBN - 1) / UBN;
  int64_t total = 0;
  for (int64_t b = 0; b < nbi; ++b)
    total += lower ? std::min<int64_t>(ntj, (b * UBM + UBM - 1) / UBN + 1) : ntj;
  for (int64_t k0 = 0; k0 < K; k0 += UK_MAX) {
    const int64_t kc = std::min<int64_t>(UK_MAX, K - k0), kp = digits_kp(kc);
    uint16_t *pa = reinterpret_cast<uint16_t *>(work);
    int *ea = reinterpret_cast<int *>((char *)work + align256u((size_t)RP * M * kp * 2));
    uint16_t *pb = pa;
    int *eb = ea;
    digits_rows_kernel<<<(unsigned)ceil_div(M, 8), 256, 0, st>>>(X + k0, ldx, M, kc, pa, kp,
                                                                  M * kp, ea, status);
    count_launch();
    int64_t rows_b = M;
    if (!same) {
      char *wb = (char *)work + digit_set_bytes(M, K);
      pb = reinterpret_cast<uint16_t *>(wb);
      eb = reinterpret_cast<int *>(wb + align256u((size_t)RP * N * kp * 2));
      if (y_kxn)
        digits_cols_kernel<<<(unsigned)ceil_div(N, 32), 256, 0, st>>>(Y + k0 * ldy, ldy, N, kc, pb,
                                                                       kp, N * kp, eb, status);
      else
        digits_rows_kernel<<<(unsigned)ceil_div(N, 8), 256, 0, st>>>(Y + k0, ldy, N, kc, pb, kp,
                                                                      N * kp, eb, status);
      count_launch();
      rows_b = N;
    }
    CUtensorMap ma, mb;
    if (!make_digit_map(&ma, pa, kc, M, kp, UBM) || !make_digit_map(&mb, pb, kc, rows_b, kp, UBN))
      return cudaErrorInvalidValue;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(total, max_ctas));
    update_digits_kernel<<<grid, UTHREADS, USMEM, st>>>(ma, mb, ea, eb, C, ldc, M, N,
                                                        (int)((kc + UBK - 1) / UBK), total,
                                                        lower ? 1 : 0, status, err, wait_ns);
    count_launch();
  }
  return cudaGetLastError();
}

}  // namespace gb
