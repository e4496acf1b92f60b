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
// 3. pair variant (CL = 2): clusters of two CTAs on two SMs compute a
//    256 x 256 tile with tcgen05.mma.cta_group::2 (M = 256): each CTA stages
//    its own 128 rows of A and one 128-row half of B, and the MMA issued by
//    the even CTA reads both CTAs' shared memory and accumulates each CTA's
//    128 x 256 half in that CTA's tensor memory.  Per SM and k-block this
//    moves 32 KiB through shared memory instead of 48 KiB (TMA writes plus
//    MMA reads), which frees shared-memory bandwidth and room for 6 stages.
//    TMA loads of both CTAs complete on the even CTA's stage barrier; the
//    MMA issuer's commits arrive on both CTAs' barriers (multicast); the odd
//    CTA's epilogue releases the accumulator on the even CTA's barrier.
//    Before leaving, each producer waits for the last stage releases and
//    the MMA issuer for its last MMAs, so no copy, MMA or arrival targets a
//    CTA that has exited.
#include <cuda.h>  // CUtensorMap and its enums (types only; the encoder is
                   // fetched through the runtime's driver entry point)
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "gb_internal.cuh"
#include "tc_ptx.cuh"

namespace gb {
namespace {

using namespace tc;

constexpr int BM = 128, BN = 256, BK = 64;
constexpr uint32_t TMEM_COLS = 512;           // two 128 x 256 FP32 accumulators
constexpr uint32_t A_STAGE = BM * BK * 2;     // 16 KiB
constexpr uint32_t STAGING = 32 * 32 * 4;     // one 32 x 32 FP32 reduce box
// per CTA: CL = 1 stages all 256 rows of B, CL = 2 one half of them, which
// leaves room for 6 stages.  (Eight epilogue warps with 5 stages measured
// slower than four with 6: the main loop wants the deeper ring.)
template <int CL>
struct Cfg {
  static constexpr uint32_t B_STAGE = BN / CL * BK * 2;  // 32 / 16 KiB
  static constexpr int STAGES = CL == 1 ? 4 : 6;
  static constexpr int EPI_WARPS = 4;
  static constexpr int THREADS = 64 + EPI_WARPS * 32;  // producer, MMA, epilogue warps
  static constexpr size_t SMEM =
      (size_t)STAGES * (A_STAGE + B_STAGE) + EPI_WARPS * 2 * STAGING + 1024 + 256;
};
constexpr int MAX_STAGES = 6;
static_assert(Cfg<1>::SMEM <= 232448 && Cfg<2>::SMEM <= 232448, "shared memory per CTA");

// The valid output tiles, counted in row-major order of groups of `cl`
// vertically adjacent tiles and dealt out round-robin: index v goes to the
// persistent CTA (cl = 1) or cluster (cl = 2) v mod stride, so every CTA
// gets the same number of tiles to within one.  A group row holds a prefix
// of valid tiles (lower mode: up to the diagonal of its lowest tile); `rank`
// picks the tile of the group.
struct TileIter {
  int64_t v, total, stride;  // next index, number of valid groups, stride
  int64_t row, row_start;    // group row of index v and the index of its first tile
  int64_t nbj, diag;
  int rank, cl;
  bool lower;
  __device__ int64_t row_count(int64_t bg) const {
    if (!lower) return nbj;
    const int64_t last = bg * cl * BM + cl * BM - 1 + diag;  // last column on/below the diagonal
    return last < 0 ? 0 : min64(nbj, last / BN + 1);
  }
  __device__ bool next(int64_t &m0, int64_t &n0) {
    if (v >= total) return false;
    for (int64_t c = row_count(row); v >= row_start + c; c = row_count(row)) {
      row_start += c;
      ++row;
    }
    m0 = row * cl * BM + rank * BM;
    n0 = (v - row_start) * BN;
    v += stride;
    return true;
  }
};

// ---------------------------------------------------------------- kernel
// Persistent: one CTA per SM (CL = 1) or one CTA pair per two SMs (CL = 2)
// walks the tile list.  Warp 0 = TMA producer, warp 1 = MMA issuer (even CTA
// only for a pair) and tensor-memory owner, warps 2..5 = epilogue.  Two
// 256-column accumulators let the epilogue of one tile run while the MMAs of
// the next accumulate.
template <bool LOWER, int CL>
__global__ void __launch_bounds__(Cfg<CL>::THREADS, 1)
    tc_update_kernel(const __grid_constant__ CUtensorMap map_a,
                     const __grid_constant__ CUtensorMap map_b,
                     const __grid_constant__ CUtensorMap map_c, float *__restrict__ C, int64_t ldc,
                     int64_t M, int64_t N, int nk, int64_t diag, int64_t total, uint32_t idesc,
                     const int *status, int *err, long long wait_ns, int use_tma_store,
                     int vec_ok, int kbs, uint32_t bstripe) {
  static_assert(CL == 1 || CL == 2, "one CTA or a CTA pair");
  constexpr int STAGES = Cfg<CL>::STAGES;
  constexpr uint32_t B_STAGE = Cfg<CL>::B_STAGE;
  constexpr int EPI_WARPS = Cfg<CL>::EPI_WARPS;
  static_assert(EPI_WARPS % 4 == 0 && STAGES <= MAX_STAGES, "epilogue warps per lane quarter");
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint8_t *sA = smem;
  uint8_t *sB = sA + STAGES * A_STAGE;
  uint8_t *sStage = sB + STAGES * B_STAGE;  // EPI_WARPS x 2 x 4 KiB, 1 KiB aligned
  uint64_t *full = reinterpret_cast<uint64_t *>(sStage + EPI_WARPS * 2 * STAGING);
  uint64_t *empty = full + MAX_STAGES;
  uint64_t *acc_full = empty + MAX_STAGES;
  uint64_t *acc_empty = acc_full + 2;
  uint64_t *drain = acc_empty + 2;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  volatile uint32_t *skip = reinterpret_cast<volatile uint32_t *>(tmem_slot + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = CL > 1 ? cluster_ctarank() : 0u;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);   // the even CTA's producer arrives (with the byte count)
      mbar_init(&empty[s], 1);  // one commit of the MMA issuer
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], CL * EPI_WARPS);  // every epilogue warp of the pair
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // Skip the work after a failed column step, or when a CTA whose wait
    // expired has already raised the error word.  Rank 0 decides for the
    // whole cluster, so that both CTAs of a pair skip or both work.
    if (rank == 0) {
      const uint32_t v = (*reinterpret_cast<const volatile int *>(status) != 0 ||
                          (*reinterpret_cast<const volatile int *>(err) & DEV_ERR_TIMEOUT))
                             ? 1u
                             : 0u;
      if (CL > 1) {
        for (uint32_t r = 0; r < (uint32_t)CL; ++r) st_cluster_u32((void *)skip, r, v);
      } else {
        *skip = v;
      }
    }
  }
  if (warp == 1) tmem_alloc<CL>(tmem_slot, TMEM_COLS);
  tc_fence_before();
  if (CL > 1) cluster_sync();  // barriers initialised and tensor memory allocated in both CTAs
  else __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const unsigned long long deadline = (unsigned long long)wait_ns;  // per wait

  const int64_t nbj = (N + BN - 1) / BN;
  const int64_t group = CL > 1 ? (int64_t)cluster_id_x() : (int64_t)blockIdx.x;
  const int64_t ngroups = CL > 1 ? (int64_t)num_clusters_x() : (int64_t)gridDim.x;
  TileIter it{group, total, ngroups, 0, 0, nbj, diag, (int)rank, CL, LOWER};
  int64_t m0 = 0, n0 = 0;

  if (*skip) {
    // nothing issued: straight to the teardown
  } else if (warp == 0) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      uint32_t g = 0;
      bool ok = true;
      // stage barrier the copies complete on: this CTA's, or the even CTA's
      const uint32_t full0 = CL > 1 ? cluster_addr(full, 0) : smem_u32(full);
      while (ok && it.next(m0, n0)) {
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const uint32_t s = g % STAGES, ph = (g / STAGES) & 1u;
          // B's k-block: stripe table entry of this term, same offset inside it
          const int t = kb / kbs;
          const int kbb = (int)((bstripe >> (4 * t)) & 15u) * kbs + (kb - t * kbs);
          if (g >= (uint32_t)STAGES && !mbar_wait(&empty[s], ph ^ 1u, deadline, err, abort_flag)) {
            ok = false;
            break;
          }
          if (CL == 1) {
            mbar_expect_tx(&full[s], A_STAGE + B_STAGE);
            tma_load_2d(sA + s * A_STAGE, &map_a, &full[s], kb * BK, (int)m0);
            tma_load_2d(sB + s * B_STAGE, &map_b, &full[s], kbb * BK, (int)n0);
          } else {
            // the even CTA's barrier counts the bytes of both CTAs
            if (rank == 0) mbar_expect_tx(&full[s], CL * (A_STAGE + B_STAGE));
            const uint32_t bar = full0 + s * 8u;
            tma_load_2d_pair(sA + s * A_STAGE, &map_a, bar, kb * BK, (int)m0);
            tma_load_2d_pair(sB + s * B_STAGE, &map_b, bar, kbb * BK,
                             (int)(n0 + rank * (BN / 2)));
          }
        }
      }
      // Pair: wait for the last stage releases, so that no commit arrives on
      // this CTA's barriers after it exits (every copy into this CTA was
      // waited for by the MMA issuer before it released the stage).
      if (CL > 1 && ok) {
        for (uint32_t j = g > (uint32_t)STAGES ? g - STAGES : 0u; j < g; ++j)
          if (!mbar_wait(&empty[j % STAGES], (j / STAGES) & 1u, deadline, err, abort_flag)) break;
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0 && rank == 0) {
      uint32_t g = 0, i = 0;
      bool ok = true;
      while (ok && it.next(m0, n0)) {
        const uint32_t buf = i & 1u, use = i >> 1;
        if (use > 0 && !mbar_wait(&acc_empty[buf], (use - 1) & 1u, deadline, err, abort_flag))
          break;
        tc_fence_after();
        const uint32_t d = tmem + buf * (TMEM_COLS / 2);
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const uint32_t s = g % STAGES, ph = (g / STAGES) & 1u;
          if (!mbar_wait(&full[s], ph, deadline, err, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(sA + s * A_STAGE), b0 = smem_u32(sB + s * B_STAGE);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk)
            mma_f16<CL>(d, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), idesc,
                        (kb | kk) != 0 ? 1u : 0u);
          if (CL == 1) mma_commit(&empty[s]);
          else mma_commit_pair_mc(&empty[s], (uint16_t)0x3);
        }
        if (!ok) break;
        if (CL == 1) mma_commit(&acc_full[buf]);
        else mma_commit_pair_mc(&acc_full[buf], (uint16_t)0x3);
        ++i;
      }
      // every MMA issued (into both CTAs' tensor memory, for a pair) is done
      // before the tensor memory is released
      if (CL == 1) mma_commit(drain);
      else mma_commit_pair(drain);
      const unsigned long long until = now_ns() + deadline;  // bounded, even after an abort
      while (!mbar_try_wait(drain, 0)) {
        if (now_ns() > until) {
          atomicOr(err, DEV_ERR_TIMEOUT);
          break;
        }
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------ epilogue (warps 2..)
    const int e = warp - 2;                // 0 .. EPI_WARPS - 1
    const int q = warp & 3;                // tensor-memory lane quarter this warp may read
    constexpr int CPW = BN / 32 / (EPI_WARPS / 4);  // 32-column chunks per warp
    const int c_begin = (e / 4) * CPW;     // this warp's share of the tile's columns
    uint8_t *stage0 = sStage + (size_t)e * 2 * STAGING;
    // accumulator release goes to the MMA issuer's CTA (the even one)
    const uint32_t acc_empty0 = CL > 1 ? cluster_addr(acc_empty, 0) : smem_u32(acc_empty);
    uint32_t i = 0, chunks = 0;
    while (it.next(m0, n0)) {
      const uint32_t buf = i & 1u, use = i >> 1;
      if (!mbar_wait(&acc_full[buf], use & 1u, deadline, err, abort_flag)) break;
      tc_fence_after();
      const int64_t row0 = m0 + q * 32;
      const int64_t row = row0 + lane;
      for (int c = c_begin; c < c_begin + CPW; ++c) {
        const int64_t col0 = n0 + c * 32;
        if (col0 >= N || row0 >= M) break;                  // warp-uniform
        if (LOWER && row0 + 31 + diag < col0) break;        // chunk above the diagonal
        float v[32];
        tmem_ld_32x32(tmem + buf * (TMEM_COLS / 2) + ((uint32_t)(q * 32) << 16) + (uint32_t)(c * 32),
                      v);
        if (*abort_flag) continue;
        if (use_tma_store) {
          uint8_t *sb = stage0 + (chunks & 1u) * STAGING;
          if (chunks >= 2) {
            if (lane == 0) bulk_wait_read<1>();  // the reduce that last read `sb` is done
            __syncwarp();
          }
#pragma unroll
          for (int q4 = 0; q4 < 8; ++q4) {
            float4 w;
            float *wp = &w.x;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int64_t col = col0 + q4 * 4 + u;
              wp[u] = (!LOWER || row + diag >= col) ? -v[q4 * 4 + u] : -0.0f;  // x + -0 == x
            }
            // 128-byte swizzle: 16-byte chunk q4 of row `lane` sits at q4 ^ (lane % 8)
            *reinterpret_cast<float4 *>(sb + lane * 128 + ((q4 ^ (lane & 7)) * 16)) = w;
          }
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) {
            tma_reduce_add_2d(&map_c, sb, (int)col0, (int)row0);
            bulk_commit();
          }
          ++chunks;
        } else if (row < M) {
          float *crow = C + row * ldc + col0;
          const bool full_row = col0 + 32 <= N && (!LOWER || row + diag >= col0 + 31);
          if (vec_ok && full_row) {
#pragma unroll
            for (int q4 = 0; q4 < 8; ++q4) {
              float4 x = *reinterpret_cast<float4 *>(crow + 4 * q4);
              x.x -= v[4 * q4 + 0];
              x.y -= v[4 * q4 + 1];
              x.z -= v[4 * q4 + 2];
              x.w -= v[4 * q4 + 3];
              *reinterpret_cast<float4 *>(crow + 4 * q4) = x;
            }
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int64_t col = col0 + j;
              if (col < N && (!LOWER || row + diag >= col)) crow[j] -= v[j];
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if (CL == 1) mbar_arrive(&acc_empty[buf]);
        else mbar_arrive_cluster(acc_empty0 + buf * 8u);
      }
      ++i;
    }
    if (lane == 0) bulk_wait_all();
    __syncwarp();
  }
  tc_fence_before();
  if (CL > 1) cluster_sync();
  else __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc<CL>(tmem, TMEM_COLS);
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
template <typename T16>
__device__ __forceinline__ float from16(T16 x);
template <>
__device__ __forceinline__ float from16<__nv_bfloat16>(__nv_bfloat16 x) {
  return __bfloat162float(x);
}
template <>
__device__ __forceinline__ float from16<__half>(__half x) {
  return __half2float(x);
}

// Planes of x: p0 = round16(x), p1 = round16(x - p0), p2 = round16(x - p0 - p1)
// (each difference is exact in FP32).  Term t of the packed row uses plane
// (code >> 2t) & 3.
template <typename T16>
__device__ __forceinline__ void split_planes(float x, T16 (&p)[3]) {
  p[0] = to16<T16>(x);
  const float r1 = x - from16<T16>(p[0]);
  p[1] = to16<T16>(r1);
  p[2] = to16<T16>(r1 - from16<T16>(p[1]));
}

// out[i * ldo + t * Kp + k] = plane_t(X[i * ldx + k]) for k < K, 0 for K <= k < Kp.
// Each thread converts 8 consecutive k of one row (Kp is a multiple of 64):
// two 16-byte loads and one 16-byte store per plane when `vec_in` (X 16-byte
// aligned, ldx % 4 == 0) and `vec_out` (out 16-byte aligned, ldo % 8 == 0).
template <typename T16>
__global__ void pack_rows_kernel(const float *__restrict__ X, int64_t ldx, int64_t rows,
                                 int64_t K, int64_t Kp, int terms, uint32_t code,
                                 T16 *__restrict__ out, int64_t ldo, int vec_in, int vec_out) {
  const int64_t groups = Kp >> 3;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= groups) return;
  const int64_t k0 = g << 3;
  for (int64_t i = (int64_t)blockIdx.y * blockDim.y + threadIdx.y; i < rows;
       i += (int64_t)gridDim.y * blockDim.y) {
    const float *src = X + i * ldx + k0;
    float x[8];
    if (vec_in && k0 + 8 <= K) {
      const float4 a = __ldg(reinterpret_cast<const float4 *>(src));
      const float4 b = __ldg(reinterpret_cast<const float4 *>(src + 4));
      x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
      x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
    } else {
#pragma unroll
      for (int u = 0; u < 8; ++u) x[u] = k0 + u < K ? src[u] : 0.0f;
    }
    T16 p[3][8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      T16 q[3];
      split_planes<T16>(x[u], q);
      p[0][u] = q[0];
      p[1][u] = q[1];
      p[2][u] = q[2];
    }
    T16 *o = out + i * ldo + k0;
    for (int t = 0; t < terms; ++t) {
      const T16 *v = p[(code >> (2 * t)) & 3u];
      if (vec_out) {
        uint4 w;
        memcpy(&w, v, 16);
        *reinterpret_cast<uint4 *>(o + t * Kp) = w;
      } else {
#pragma unroll
        for (int u = 0; u < 8; ++u) o[t * Kp + u] = v[u];
      }
    }
  }
}

// Same from a K x N row-major Y: out[j][t * Kp + k] = plane_t(Y[k * ldy + j]).
template <typename T16>
__global__ void pack_transpose_kernel(const float *__restrict__ Y, int64_t ldy, int64_t K,
                                      int64_t N, int64_t Kp, int terms, uint32_t code,
                                      T16 *__restrict__ out) {
  __shared__ float t[32][33];
  const int64_t k0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t k = k0 + r, j = j0 + threadIdx.x;
    t[r][threadIdx.x] = (k < K && j < N) ? Y[k * ldy + j] : 0.0f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t j = j0 + r, k = k0 + threadIdx.x;
    if (j < N && k < Kp) {
      T16 p[3];
      split_planes<T16>(t[threadIdx.x][r], p);
      T16 *o = out + j * (Kp * terms) + k;
      for (int u = 0; u < terms; ++u) o[u * Kp] = p[(code >> (2 * u)) & 3u];
    }
  }
}

// ------------------------------------------------------------ host helpers
// 2-D map over a dense rows x cols 16-bit K-major buffer, box 64 x box_rows.
bool make_operand_map(CUtensorMap *map, const void *base, int64_t rows, int64_t cols,
                      int box_rows, bool f16, int64_t row_stride) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)row_stride * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                   const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// FP32 map over C (M x N, ldc), 32 x 32 boxes with the 128-byte swizzle, for
// the reduce-add epilogue.  Needs a 16-byte aligned C and ldc % 4 == 0.
bool make_c_map(CUtensorMap *map, float *C, int64_t ldc, int64_t M, int64_t N) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  if ((reinterpret_cast<uintptr_t>(C) & 15) != 0 || (ldc & 3) != 0) return false;
  cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)M};
  cuuint64_t strides[1] = {(cuuint64_t)ldc * 4};
  cuuint32_t box[2] = {32, 32};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, C, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// Operand planes per term: 1 term (plain) or the 6 leading products of a
// three-way split, smallest first: (2,0) (1,1) (0,2) (1,0) (0,1) (0,0).
int split_terms(int split) { return split == 3 ? 6 : 1; }
uint32_t code_of(const int *planes, int terms) {
  uint32_t c = 0;
  for (int t = 0; t < terms; ++t) c |= (uint32_t)planes[t] << (2 * t);
  return c;
}
constexpr int X3_PLANES[6] = {2, 1, 0, 1, 0, 0};
constexpr int Y3_PLANES[6] = {0, 1, 2, 0, 1, 0};

// For Y packed as X (the same rows): term t's B stripe is the first X
// stripe that holds plane Y3_PLANES[t].
uint32_t stripes_of_y_in_x() {
  uint32_t code = 0;
  for (int t = 0; t < 6; ++t) {
    int st = 0;
    while (X3_PLANES[st] != Y3_PLANES[t]) ++st;
    code |= (uint32_t)st << (4 * t);
  }
  return code;
}

template <typename T16>
void launch_pack_rows(const float *X, int64_t ldx, int64_t rows, int64_t K, int64_t Kp, int terms,
                      uint32_t code, T16 *out, int64_t ldo, cudaStream_t st) {
  // a block is gx groups of 8 columns by gy rows, about 128 threads
  const int64_t groups = Kp / 8;
  const int gx = (int)std::min<int64_t>(groups, 128), gy = std::max(1, 128 / gx);
  const dim3 grid((unsigned)((groups + gx - 1) / gx),
                  (unsigned)std::min<int64_t>((rows + gy - 1) / gy, 65535));
  const dim3 block((unsigned)gx, (unsigned)gy);
  const int vec_in = ((reinterpret_cast<uintptr_t>(X) & 15) == 0 && (ldx & 3) == 0) ? 1 : 0;
  const int vec_out = ((reinterpret_cast<uintptr_t>(out) & 15) == 0 && (ldo & 7) == 0) ? 1 : 0;
  pack_rows_kernel<T16><<<grid, block, 0, st>>>(X, ldx, rows, K, Kp, terms, code, out, ldo,
                                                vec_in, vec_out);
  count_launch();
}

template <typename T16>
cudaError_t pack_operands(const TcUpdateArgs &a, int64_t Kp, int terms, T16 *xp, T16 *yp, bool same,
                          cudaStream_t st) {
  const int one[1] = {0};
  const uint32_t cx = terms == 1 ? code_of(one, 1) : code_of(X3_PLANES, 6);
  const uint32_t cy = terms == 1 ? code_of(one, 1) : code_of(Y3_PLANES, 6);
  launch_pack_rows<T16>(a.X, a.ldx, a.M, a.K, Kp, terms, cx, xp, Kp * terms, st);
  if (!same) {
    if (a.nn) {
      dim3 grid((unsigned)((a.N + 31) / 32), (unsigned)((Kp + 31) / 32));
      pack_transpose_kernel<T16><<<grid, dim3(32, 8), 0, st>>>(a.Y, a.ldy, a.K, a.N, Kp, terms,
                                                                cy, yp);
      count_launch();
    } else {
      launch_pack_rows<T16>(a.Y, a.ldy, a.N, a.K, Kp, terms, cy, yp, Kp * terms, st);
    }
  }
  return cudaGetLastError();
}

struct TcKernelArgs {
  CUtensorMap map_a, map_b, map_c;
  float *C;
  int64_t ldc, M, N;
  int nk;
  int64_t diag, total;
  uint32_t idesc;
  const int *status;
  int *err;
  long long wait_ns;
  int use_tma_store, vec_ok;
  int kbs;           // k-blocks per term stripe (Kp / BK)
  uint32_t bstripe;  // B's stripe for term t in bits 4t..4t+3
};

// Launch over `valid` tile groups: clusters of CL CTAs, as many groups as can
// be resident at once (one CTA per SM), at most `valid`.
template <bool LOWER, int CL>
cudaError_t launch_kernel(const TcKernelArgs &k, int64_t valid, int dev, cudaStream_t st) {
  auto kern = tc_update_kernel<LOWER, CL>;
  static const cudaError_t attr =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg<CL>::SMEM);
  if (attr != cudaSuccess) return attr;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(Cfg<CL>::THREADS);
  cfg.dynamicSmemBytes = Cfg<CL>::SMEM;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int64_t slots = sms;
  if (CL > 1) {
    // SMs are paired within a GPC, so an odd GPC leaves one SM without a pair
    static const int max_clusters = [&] {
      cudaLaunchConfig_t q = cfg;
      q.gridDim = dim3((unsigned)(sms / CL * CL));
      q.stream = 0;
      int n = 0;
      if (cudaOccupancyMaxActiveClusters(&n, kern, &q) != cudaSuccess || n <= 0) {
        cudaGetLastError();
        n = sms / CL;
      }
      return n;
    }();
    slots = max_clusters;
  }
  const int64_t groups = std::max<int64_t>(1, std::min<int64_t>(slots, valid));
  cfg.gridDim = dim3((unsigned)(groups * CL));
  count_launch();
  return cudaLaunchKernelEx(&cfg, kern, k.map_a, k.map_b, k.map_c, k.C, k.ldc, k.M, k.N, k.nk,
                            k.diag, k.total, k.idesc, k.status, k.err, k.wait_ns,
                            k.use_tma_store, k.vec_ok, k.kbs, k.bstripe);
}


// ------------------------------------------------ tensor-pipe peak loop
// One CTA per SM issues back-to-back dense MMAs M = 128, N = 256 on
// K-major tiles already in shared memory (zeros: the rate does not depend on
// the values), accumulating into one TMEM accumulator, and waits (bounded)
// for their completion.  kind 0: kind::f16 with BF16 operands, 1: kind::f16
// with FP16 operands (K = 16 per instruction), 2: kind::tf32 (K = 8).  Each
// 128-byte row step of the tiles is one instruction's K.
constexpr uint32_t PEAK_A = BM * 128, PEAK_B = BN * 128;  // one 128-byte K step each
constexpr size_t PEAK_SMEM = PEAK_A + PEAK_B + 1024;

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
      : "memory");
}

__global__ void __launch_bounds__(128, 1)
    tc_peak_kernel(int kind, int iters, uint32_t idesc, long long wait_ns, int *err) {
  extern __shared__ __align__(1024) unsigned char peak_raw[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_done;
  __shared__ int s_abort;
  const uint32_t base = (smem_u32(peak_raw) + 1023u) & ~1023u;
  unsigned char *gen = peak_raw + (base - smem_u32(peak_raw));
  for (uint32_t i = threadIdx.x * 16; i < PEAK_A + PEAK_B; i += 128 * 16)
    *reinterpret_cast<uint4 *>(gen + i) = make_uint4(0, 0, 0, 0);
  if (threadIdx.x == 0) {
    mbar_init(&s_done, 1);
    s_abort = 0;
  }
  fence_proxy_async_smem();  // the zeros are read by the tensor pipe
  if (threadIdx.x < 32) tmem_alloc<1>(&s_tmem, 256);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  if (threadIdx.x == 0) {
    const uint32_t a0 = base, b0 = base + PEAK_A;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t da = sw128_desc(a0 + kk * 32), db = sw128_desc(b0 + kk * 32);
        const uint32_t acc = (it | kk) != 0;
        if (kind == 2) mma_tf32(tmem, da, db, idesc, acc);
        else mma_f16<1>(tmem, da, db, idesc, acc);
      }
    }
    mma_commit(&s_done);
  }
  __syncwarp();
  mbar_wait(&s_done, 0, (unsigned long long)wait_ns, err, &s_abort);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (threadIdx.x < 32) tmem_dealloc<1>(tmem, 256);
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

cudaError_t launch_pack16(const float *X, int64_t ldx, int64_t rows, int64_t K, void *out,
                          int64_t ldo, bool f16, cudaStream_t st) {
  if (rows <= 0 || K <= 0) return cudaSuccess;
  const int one[1] = {0};
  const uint32_t code = code_of(one, 1);
  const int64_t Kp = round_up(K, BK);
  if (ldo < Kp) return cudaErrorInvalidValue;
  if (f16)
    launch_pack_rows<__half>(X, ldx, rows, K, Kp, 1, code, reinterpret_cast<__half *>(out), ldo, st);
  else
    launch_pack_rows<__nv_bfloat16>(X, ldx, rows, K, Kp, 1, code,
                                    reinterpret_cast<__nv_bfloat16 *>(out), ldo, st);
  return cudaGetLastError();
}

size_t tc_pack_bytes(int64_t M, int64_t N, int64_t K, bool nn, int split) {
  const int64_t Kp = round_up(std::max<int64_t>(K, 1), BK);
  (void)nn;
  return (size_t)(round_up(M, 8) + round_up(N, 8)) * (size_t)(Kp * split_terms(split)) * 2 + 256;
}

cudaError_t launch_update_tc(const TcUpdateArgs &a, cudaStream_t st) {
  if (a.M <= 0 || a.N <= 0 || a.K <= 0) return cudaSuccess;
  int dev = 0;
  cudaGetDevice(&dev);
  if (!tc_supported(dev)) return cudaErrorNotSupported;
  if (a.M > INT32_MAX - BM || a.N > INT32_MAX - BN) return cudaErrorInvalidValue;
  if (a.split == 3 && a.f16) return cudaErrorNotSupported;
  const int terms = split_terms(a.split);
  const int64_t Kp = round_up(a.K, BK), Ke = Kp * terms;
  if (Ke / BK > INT32_MAX) return cudaErrorInvalidValue;
  const void *xp, *yp;
  int64_t xstride = Ke, ystride = Ke;
  uint32_t bstripe = 0x543210u;  // B's term t from its own stripe t
  if (a.xpack) {
    // operands already resident as 16-bit rows (one plane, K a multiple of
    // 64, rows 16-byte aligned): no packing
    if (terms != 1 || a.K % BK != 0 || !a.ypack) return cudaErrorInvalidValue;
    if ((reinterpret_cast<uintptr_t>(a.xpack) & 15) || (reinterpret_cast<uintptr_t>(a.ypack) & 15) ||
        (a.ldxp & 7) || (a.ldyp & 7) || a.ldxp < a.K || a.ldyp < a.K)
      return cudaErrorInvalidValue;
    xp = a.xpack;
    yp = a.ypack;
    xstride = a.ldxp;
    ystride = a.ldyp;
  } else {
    if (tc_pack_bytes(a.M, a.N, a.K, a.nn, a.split) > a.pack_bytes) return cudaErrorInvalidValue;
    // Y's rows are the first N rows of X (the Cholesky updates: the same
    // panel, the trailing columns a prefix of the trailing rows): X's packed
    // rows serve as Y's too -- with three planes through the stripe table,
    // since X's stripes hold the planes in another order than Y's
    const bool same = !a.nn && a.X == a.Y && a.ldx == a.ldy && a.N <= a.M;
    if (same && terms > 1) bstripe = stripes_of_y_in_x();
    uint8_t *base = reinterpret_cast<uint8_t *>(a.pack);
    void *xw = base;
    void *yw = same ? base : base + (size_t)round_up(a.M, 8) * Ke * 2;
    cudaError_t e = a.f16 ? pack_operands<__half>(a, Kp, terms, (__half *)xw, (__half *)yw, same, st)
                          : pack_operands<__nv_bfloat16>(a, Kp, terms, (__nv_bfloat16 *)xw,
                                                         (__nv_bfloat16 *)yw, same, st);
    if (e != cudaSuccess) return e;
    xp = xw;
    yp = yw;
  }
  CUtensorMap map_a, map_b, map_c;
  memset(&map_c, 0, sizeof map_c);
  const int use_tma_store = make_c_map(&map_c, a.C, a.ldc, a.M, a.N) ? 1 : 0;
  const int vec_ok = ((reinterpret_cast<uintptr_t>(a.C) & 15) == 0 && (a.ldc & 3) == 0) ? 1 : 0;
  // a tile takes microseconds; one second bounds every single wait
  const long long wait_ns = std::min<long long>((long long)a.spin_limit * 100LL, 1000000000LL);
  // persistent grid: one CTA (cluster) per SM (pair of SMs), at most one per
  // valid tile (pair of vertically adjacent tiles)
  const int CL = a.cluster == 2 ? 2 : 1;
  // instruction descriptor: FP32 accumulator, A/B = BF16 (1) or FP16 (0),
  // both K-major, N >> 3 at bit 17, M >> 4 at bit 24 (M = 256 for a pair)
  const uint32_t ab = a.f16 ? 0u : 1u;
  const uint32_t idesc = (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(BN >> 3) << 17) |
                         ((uint32_t)((BM * CL) >> 4) << 24);
  const int64_t nbi = (a.M + BM - 1) / BM, nbj = (a.N + BN - 1) / BN;
  const int64_t nbg = (nbi + CL - 1) / CL;
  int64_t valid = 0;
  for (int64_t bg = 0; bg < nbg; ++bg) {
    if (!a.lower) {
      valid += nbj;
      continue;
    }
    // largest column index on/below the diagonal in the group's lowest tile
    const int64_t last = bg * CL * BM + CL * BM - 1 + a.diag;
    if (last >= 0) valid += std::min<int64_t>(nbj, last / BN + 1);
  }
  if (a.packed) cudaEventRecord(a.packed, st);
  if (valid == 0) return cudaSuccess;
  if (!make_operand_map(&map_a, xp, a.M, Ke, BM, a.f16, xstride) ||
      !make_operand_map(&map_b, yp, a.N, Ke, BN / CL, a.f16, ystride))
    return cudaErrorInvalidValue;
  const TcKernelArgs k{map_a, map_b, map_c, a.C, a.ldc, a.M, a.N, (int)(Ke / BK), a.diag,
                       valid, idesc, a.status, a.err, wait_ns, use_tma_store, vec_ok,
                       (int)(Kp / BK), bstripe};
  cudaError_t e;
  if (a.lower)
    e = CL == 2 ? launch_kernel<true, 2>(k, valid, dev, st) : launch_kernel<true, 1>(k, valid, dev, st);
  else
    e = CL == 2 ? launch_kernel<false, 2>(k, valid, dev, st)
                : launch_kernel<false, 1>(k, valid, dev, st);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// Tensor-pipe throughput (see tc_peak_kernel): flop/s over every SM.
cudaError_t measure_tc_peak(int kind, int sm_count, double *flops_per_s) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (!tc_supported(dev)) return cudaErrorNotSupported;
  if (kind < 0 || kind > 2) return cudaErrorInvalidValue;
  static const cudaError_t attr = cudaFuncSetAttribute(
      tc_peak_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PEAK_SMEM);
  if (attr != cudaSuccess) return attr;
  // A and B formats: BF16 1, FP16 0 (kind::f16), TF32 2 (kind::tf32)
  const uint32_t ab = kind == 0 ? 1u : (kind == 1 ? 0u : 2u);
  const uint32_t idesc = (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(BN >> 3) << 17) |
                         ((uint32_t)(BM >> 4) << 24);
  const int iters = kind == 2 ? 10000 : 20000;
  const double k_instr = kind == 2 ? 8.0 : 16.0;
  int *err = nullptr;
  if ((e = cudaMalloc(&err, sizeof(int))) != cudaSuccess) return e;
  cudaEvent_t a = nullptr, b = nullptr;
  float ms = 0.f;
  int herr = 0;
  const long long wait_ns = 1000000000LL;  // 1 s: the loop takes ~10 ms
  if ((e = cudaMemset(err, 0, sizeof(int))) == cudaSuccess &&
      (e = cudaEventCreate(&a)) == cudaSuccess && (e = cudaEventCreate(&b)) == cudaSuccess) {
    tc_peak_kernel<<<sm_count, 128, PEAK_SMEM>>>(kind, iters / 20, idesc, wait_ns, err);  // warm-up
    count_launch();
    cudaEventRecord(a);
    tc_peak_kernel<<<sm_count, 128, PEAK_SMEM>>>(kind, iters, idesc, wait_ns, err);
    count_launch();
    cudaEventRecord(b);
    if ((e = cudaEventSynchronize(b)) == cudaSuccess && (e = cudaGetLastError()) == cudaSuccess &&
        (e = cudaEventElapsedTime(&ms, a, b)) == cudaSuccess)
      e = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(err);
  if (e != cudaSuccess) return e;
  if (herr) return cudaErrorLaunchTimeout;
  const double flops = (double)sm_count * iters * 4.0 * 2.0 * BM * BN * k_instr;
  *flops_per_s = flops / (ms * 1e-3);
  return cudaSuccess;
}

}  // namespace gb
