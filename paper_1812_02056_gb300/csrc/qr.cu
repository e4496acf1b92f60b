// Algorithm 3 (fast QR with step s, arXiv:1812.02056 Sec. 2) on the CUDA
// cores.  The working matrix M lives in the caller's Q buffer: column c of
// M is turned into column c of Q in place (M's column c is not read again
// once Q's column c exists).
//
//  * qr_panel_kernel -- the column steps of an inner block of bb columns:
//    v := column c of M; v := v - u (u^T v) for the columns u of the block
//    already done, one after the other; v := v / ||v||.  One cluster of 8
//    CTAs (4 warps each, one per SM sub-partition) holds the block, rows
//    split over the CTAs, in shared memory; every dot product is a
//    cluster-wide sum: shuffle trees in each warp, a 4-lane tree over the
//    warps, the 8 CTA sums written into every CTA's shared memory
//    (distributed shared memory), one cluster barrier and an 8-lane shuffle
//    tree in every warp.  The trees are fixed, so every thread of every CTA
//    gets the same bits.  Few warps and trees keep the number of FP64
//    instructions per sum small: on this GPU an FP64 warp instruction
//    occupies its sub-partition's FP64 unit for many cycles.
//  * gemm_tn_kernel -- C := X^T Y for the block projections of Algorithm 3,
//    C = B_Q^T B_M (X = B_Q, Y = B_M, both read along rows of row-major
//    matrices), and for R := Q^T A (upper triangle, zeros below).  Skinny
//    products split K over several CTAs into a workspace and a second
//    kernel adds the slices in a fixed order (deterministic).
//  * S := B_Q C and M -= S use the register-tiled update kernel of
//    Algorithms 1 and 2 (update_simt.cu) in its K x N operand form.
#include <math.h>

#include <algorithm>

#include "gb_internal.cuh"

namespace gb {
namespace {

constexpr int QR_CL = 8;    // CTAs per cluster (portable size)
constexpr int QR_NT = 128;  // threads per CTA: one warp per SM sub-partition
constexpr int QR_NW = QR_NT / 32;

__device__ __forceinline__ uint32_t qr_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void qr_cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t qr_cluster_addr(const void *p, uint32_t rank) {
  uint32_t remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
               : "=r"(remote)
               : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
  return remote;
}
__device__ __forceinline__ void qr_st_cluster(uint32_t addr, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}
__device__ __forceinline__ void qr_st_cluster(uint32_t addr, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}

// Sum of `part` over all threads of the cluster, the same bits in every
// thread: every tree below adds the same two values in every lane (a + b or
// b + a), so all lanes, warps and CTAs end with identical sums.  `slots`
// (2 x QR_CL per CTA) alternates between two halves so that one cluster
// barrier per sum suffices: a CTA writes half p of the others' slots for sum
// k only after every CTA passed the barrier of sum k - 1, by which time all
// reads of half p (sum k - 2) are done.
template <typename T>
__device__ T cluster_sum(T part, T *wsum, T *slots, int &parity, uint32_t rank) {
  static_assert(QR_NW == 4 && QR_CL == 8, "tree shapes below");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if (lane == 0) wsum[warp] = part;
  __syncthreads();
  if (warp == 0) {
    T x = lane < QR_NW ? wsum[lane] : T(0);
    x += __shfl_xor_sync(0xffffffffu, x, 2);
    x += __shfl_xor_sync(0xffffffffu, x, 1);
    x = __shfl_sync(0xffffffffu, x, 0);
    if (lane < QR_CL) qr_st_cluster(qr_cluster_addr(&slots[parity * QR_CL + rank], lane), x);
  }
  qr_cluster_sync();
  T y = lane < QR_CL ? slots[parity * QR_CL + lane] : T(0);
  y += __shfl_xor_sync(0xffffffffu, y, 4);
  y += __shfl_xor_sync(0xffffffffu, y, 2);
  y += __shfl_xor_sync(0xffffffffu, y, 1);
  parity ^= 1;
  return __shfl_sync(0xffffffffu, y, 0);
}

template <typename T>
__device__ __forceinline__ T qr_sqrt(T x);
template <>
__device__ __forceinline__ double qr_sqrt<double>(double x) {
  return sqrt(x);
}
template <>
__device__ __forceinline__ float qr_sqrt<float>(float x) {
  return sqrtf(x);
}

// Column steps of columns [col0, col0 + bb) of the n x n working matrix Qm
// (row-major, ldq).  One cluster; CTA `rank` owns rows
// [rank * rows_per, (rank + 1) * rows_per) and keeps them, column by column,
// in P[j * rows_per + i].  On a zero or NaN norm at column c the kernel
// writes c + 1 to *status and stops (every CTA sees the same norm).
template <typename T>
__global__ void __launch_bounds__(QR_NT, 1)
    qr_panel_kernel(T *__restrict__ Qm, int64_t ldq, int64_t n, int64_t col0, int bb,
                    int64_t rows_per, int *status) {
  extern __shared__ __align__(16) unsigned char qr_smem[];
  T *P = reinterpret_cast<T *>(qr_smem);
  __shared__ T wsum[QR_NW];
  __shared__ T slots[2 * QR_CL];
  // every kernel before this one on the stream has finished: all CTAs read
  // the same value
  if (*reinterpret_cast<const volatile int *>(status) != 0) return;
  const uint32_t rank = qr_ctarank();
  const int tid = threadIdx.x;
  const int64_t r0 = (int64_t)rank * rows_per;
  const int64_t rc = max((int64_t)0, min(rows_per, n - r0));
  // load: consecutive threads take consecutive elements of a row of the block
  for (int64_t e = tid; e < rc * bb; e += QR_NT) {
    const int64_t i = e / bb, j = e % bb;
    P[j * rows_per + i] = Qm[(r0 + i) * ldq + col0 + j];
  }
  __syncthreads();
  int parity = 0;
  for (int c = 0; c < bb; ++c) {
    T *v = P + (int64_t)c * rows_per;
    for (int j = 0; j < c; ++j) {  // v := v - u (u^T v), u = column j of Q
      const T *u = P + (int64_t)j * rows_per;
      T part = T(0);
      for (int64_t i = tid; i < rc; i += QR_NT) part += u[i] * v[i];
      const T d = cluster_sum(part, wsum, slots, parity, rank);
      for (int64_t i = tid; i < rc; i += QR_NT) v[i] = v[i] - u[i] * d;
    }
    T part = T(0);
    for (int64_t i = tid; i < rc; i += QR_NT) part += v[i] * v[i];
    const T nrm = qr_sqrt(cluster_sum(part, wsum, slots, parity, rank));
    if (!(nrm > T(0))) {
      if (rank == 0 && tid == 0) *status = (int)(col0 + c + 1);
      return;  // all CTAs of the cluster leave here
    }
    for (int64_t i = tid; i < rc; i += QR_NT) v[i] = v[i] / nrm;
  }
  __syncthreads();
  for (int64_t e = tid; e < rc * bb; e += QR_NT) {
    const int64_t i = e / bb, j = e % bb;
    Qm[(r0 + i) * ldq + col0 + j] = P[j * rows_per + i];
  }
}

// ------------------------------------------------------------ C := X^T Y
template <typename T>
struct TnCfg;
template <>
struct TnCfg<float> {
  static constexpr int BM = 128, BN = 128, BK = 8, TM = 8, TN = 8;
};
template <>
struct TnCfg<double> {
  static constexpr int BM = 64, BN = 64, BK = 8, TM = 4, TN = 4;
};
template <typename T>
struct TnVec;
template <>
struct TnVec<float> {
  using type = float4;
};
template <>
struct TnVec<double> {
  using type = double2;
};

// C[i][j] = sum_{k in slice} X[k][i] Y[k][j]: X is K x M (ldx), Y is K x N
// (ldy), both row-major.  blockIdx.z selects a K slice of `kslice` rows;
// with several slices the result goes to C + z * slice_stride.
// UPPER: only j >= i is computed; below the diagonal C receives zeros.
template <typename T, bool UPPER>
__global__ void __launch_bounds__(256)
    gemm_tn_kernel(T *__restrict__ C, int64_t ldc, int64_t slice_stride, const T *__restrict__ X,
                   int64_t ldx, const T *__restrict__ Y, int64_t ldy, int64_t M, int64_t N,
                   int64_t K, int64_t kslice, const int *status) {
  constexpr int BM = TnCfg<T>::BM, BN = TnCfg<T>::BN, BK = TnCfg<T>::BK;
  constexpr int TM = TnCfg<T>::TM, TN = TnCfg<T>::TN;
  constexpr int HM = TM / 2, HN = TN / 2;
  constexpr int NT = 256;
  constexpr int PADM = BM + 16 / (int)sizeof(T);
  constexpr int PADN = BN + 16 / (int)sizeof(T);
  constexpr int LA = BM * BK / NT, LB = BN * BK / NT;
  static_assert((BM / TM) * (BN / TN) == NT, "thread layout");
  using V = typename TnVec<T>::type;

  if (*reinterpret_cast<const volatile int *>(status) != 0) return;
  const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);
  T *Cz = C + (int64_t)blockIdx.z * slice_stride;
  if (UPPER && m0 > n0 + BN - 1) {  // tile strictly below the diagonal: zeros
    for (int e = tid; e < BM * BN; e += NT) {
      const int64_t gi = m0 + e / BN, gj = n0 + e % BN;
      if (gi < M && gj < N) Cz[gi * ldc + gj] = T(0);
    }
    return;
  }
  const int64_t kb = (int64_t)blockIdx.z * kslice, ke = min(K, kb + kslice);

  __shared__ __align__(16) T As[2][BK][PADM];
  __shared__ __align__(16) T Bs[2][BK][PADN];
  T ra[LA], rb[LB];
  auto load_global = [&](int64_t k0) {
#pragma unroll
    for (int r = 0; r < LA; ++r) {
      const int e = tid + NT * r;
      const int kk = e / BM, row = e % BM;
      const int64_t gi = m0 + row, gk = k0 + kk;
      ra[r] = (gi < M && gk < ke) ? X[gk * ldx + gi] : T(0);
    }
#pragma unroll
    for (int r = 0; r < LB; ++r) {
      const int e = tid + NT * r;
      const int kk = e / BN, col = e % BN;
      const int64_t gj = n0 + col, gk = k0 + kk;
      rb[r] = (gj < N && gk < ke) ? Y[gk * ldy + gj] : T(0);
    }
  };
  auto store_smem = [&](int buf) {
#pragma unroll
    for (int r = 0; r < LA; ++r) {
      const int e = tid + NT * r;
      As[buf][e / BM][e % BM] = ra[r];
    }
#pragma unroll
    for (int r = 0; r < LB; ++r) {
      const int e = tid + NT * r;
      Bs[buf][e / BN][e % BN] = rb[r];
    }
  };
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

  load_global(kb);
  store_smem(0);
  __syncthreads();
  int buf = 0;
  for (int64_t k0 = kb; k0 < ke; k0 += BK) {
    const bool more = k0 + BK < ke;
    if (more) load_global(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
      *reinterpret_cast<V *>(&a[0]) = *reinterpret_cast<const V *>(&As[buf][kk][ty * HM]);
      *reinterpret_cast<V *>(&a[HM]) =
          *reinterpret_cast<const V *>(&As[buf][kk][BM / 2 + ty * HM]);
      *reinterpret_cast<V *>(&b[0]) = *reinterpret_cast<const V *>(&Bs[buf][kk][tx * HN]);
      *reinterpret_cast<V *>(&b[HN]) =
          *reinterpret_cast<const V *>(&Bs[buf][kk][BN / 2 + tx * HN]);
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] += a[i] * b[j];
    }
    if (more) store_smem(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int64_t gi = m0 + (i < HM ? ty * HM + i : BM / 2 + ty * HM + (i - HM));
    if (gi >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int64_t gj = n0 + (j < HN ? tx * HN + j : BN / 2 + tx * HN + (j - HN));
      if (gj >= N) continue;
      Cz[gi * ldc + gj] = (UPPER && gj < gi) ? T(0) : acc[i][j];
    }
  }
}

// C[i][j] = sum_z W[z][i][j], z ascending (the K slices of gemm_tn_kernel)
template <typename T>
__global__ void sum_slices_kernel(T *__restrict__ C, int64_t ldc, const T *__restrict__ W,
                                  int64_t M, int64_t N, int slices, const int *status) {
  if (*reinterpret_cast<const volatile int *>(status) != 0) return;
  const int64_t total = M * N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    T acc = W[e];
    for (int z = 1; z < slices; ++z) acc += W[(int64_t)z * total + e];
    C[(e / N) * ldc + e % N] = acc;
  }
}

}  // namespace

int64_t qr_panel_max_cols(int64_t n, size_t esz) {
  const int64_t rows_per = std::max<int64_t>(1, (n + QR_CL - 1) / QR_CL);
  return std::max<int64_t>(0, (int64_t)(200 * 1024) / (rows_per * (int64_t)esz));
}

template <typename T>
cudaError_t launch_qr_panel(T *Qm, int64_t ldq, int64_t n, int64_t col0, int bb, int *status,
                            cudaStream_t st) {
  if (n <= 0 || bb <= 0) return cudaSuccess;
  const int64_t rows_per = (n + QR_CL - 1) / QR_CL;
  const size_t smem = (size_t)rows_per * bb * sizeof(T);
  if ((int64_t)bb > qr_panel_max_cols(n, sizeof(T))) return cudaErrorInvalidValue;
  static const cudaError_t attr = cudaFuncSetAttribute(
      qr_panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (attr != cudaSuccess) return attr;
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = QR_CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(QR_CL);
  cfg.blockDim = dim3(QR_NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  count_launch();
  return cudaLaunchKernelEx(&cfg, qr_panel_kernel<T>, Qm, ldq, n, col0, bb, rows_per, status);
}

size_t gemm_tn_work_bytes(size_t esz, int sm_count) {
  // K is split only when the result has fewer tiles than want = 2 * SMs, into
  // at most ceil(want / tiles) slices: slices * M * N < 2 * want * tile
  const size_t tile = esz == 8 ? (size_t)TnCfg<double>::BM * TnCfg<double>::BN
                               : (size_t)TnCfg<float>::BM * TnCfg<float>::BN;
  return 2 * (size_t)(2 * std::max(1, sm_count)) * tile * esz + 256;
}

template <typename T>
cudaError_t launch_gemm_tn(T *C, int64_t ldc, const T *X, int64_t ldx, const T *Y, int64_t ldy,
                           int64_t M, int64_t N, int64_t K, bool upper, const int *status,
                           void *work, size_t work_bytes, int sm_count, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  constexpr int BM = TnCfg<T>::BM, BN = TnCfg<T>::BN, BK = TnCfg<T>::BK;
  const int64_t gy = (M + BM - 1) / BM, gx = (N + BN - 1) / BN;
  if (gy > 65535) return cudaErrorInvalidConfiguration;
  // split K when the tiles alone cannot fill the GPU (skinny results)
  int64_t slices = 1;
  const int64_t tiles = gx * gy, want = 2 * (int64_t)sm_count;
  if (!upper && tiles < want && K >= 4 * 64) {
    slices = std::min<int64_t>((want + tiles - 1) / tiles, K / 64);
    const size_t need = (size_t)slices * (size_t)M * (size_t)N * sizeof(T);
    if (!work || need > work_bytes) slices = 1;
  }
  const int64_t kslice = slices == 1 ? std::max<int64_t>(K, 1)
                                     : ((K + slices - 1) / slices + BK - 1) / BK * BK;
  slices = (K + kslice - 1) / kslice;
  if (K <= 0) slices = 1;
  dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)slices);
  if (slices == 1) {
    if (upper)
      gemm_tn_kernel<T, true><<<grid, 256, 0, st>>>(C, ldc, 0, X, ldx, Y, ldy, M, N, K, kslice,
                                                     status);
    else
      gemm_tn_kernel<T, false><<<grid, 256, 0, st>>>(C, ldc, 0, X, ldx, Y, ldy, M, N, K, kslice,
                                                      status);
    count_launch();
    return cudaGetLastError();
  }
  T *W = reinterpret_cast<T *>(work);
  gemm_tn_kernel<T, false><<<grid, 256, 0, st>>>(W, N, M * N, X, ldx, Y, ldy, M, N, K, kslice,
                                                  status);
  const int64_t total = M * N;
  const unsigned g2 = (unsigned)std::min<int64_t>((total + 255) / 256, 4096);
  sum_slices_kernel<T><<<g2, 256, 0, st>>>(C, ldc, W, M, N, (int)slices, status);
  count_launch(2);
  return cudaGetLastError();
}

template cudaError_t launch_qr_panel<double>(double *, int64_t, int64_t, int64_t, int, int *,
                                             cudaStream_t);
template cudaError_t launch_qr_panel<float>(float *, int64_t, int64_t, int64_t, int, int *,
                                            cudaStream_t);
template cudaError_t launch_gemm_tn<double>(double *, int64_t, const double *, int64_t,
                                            const double *, int64_t, int64_t, int64_t, int64_t,
                                            bool, const int *, void *, size_t, int,
                                            cudaStream_t);
template cudaError_t launch_gemm_tn<float>(float *, int64_t, const float *, int64_t,
                                           const float *, int64_t, int64_t, int64_t, int64_t, bool,
                                           const int *, void *, size_t, int, cudaStream_t);

}  // namespace gb
