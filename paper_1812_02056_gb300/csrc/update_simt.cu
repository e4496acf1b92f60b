// Delayed rank-s update of Algorithms 1 and 2 (arXiv:1812.02056, Sec. 2) on
// the CUDA cores:  C -= X Y  with
//   Cholesky  C = A[c.., c..] (lower triangle), X = Y^T = R = L[c.., z..c-1]
//   LU        C = A[c.., c..] (full square),   X = R_L, Y = R_U.
// The paper forms S = R R^T "using a fast rectangular matrix multiplication"
// and subtracts it; here the product of each output tile is accumulated in
// registers (classical multiplication, k ascending within the tile loop) and
// subtracted from C in the epilogue, so S is never stored.
//
// Register-blocked tile kernel: BM x BN tile per CTA of 256 threads, each
// thread owning a TM x TN sub-tile split into two halves BM/2 (BN/2) apart so
// that 16-byte shared-memory reads by a warp are contiguous; BK-deep k slabs
// double-buffered in shared memory with a register prefetch of the next slab.
// FP32 uses 128x128x8 tiles (8x8 per thread), FP64 64x64x8 (4x4 per thread).
#include "gb_internal.cuh"

namespace gb {
namespace {

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
};
template <>
struct Vec16<double> {
  using type = double2;
};

template <typename T>
struct Cfg;
template <>
struct Cfg<float> {
  static constexpr int BM = 128, BN = 128, BK = 8, TM = 8, TN = 8;
};
template <>
struct Cfg<double> {
  static constexpr int BM = 64, BN = 64, BK = 8, TM = 4, TN = 4;
};

template <typename T, bool NN>
__global__ void __launch_bounds__(256)
    update_kernel(T *__restrict__ C, int64_t ldc, const T *__restrict__ X, int64_t ldx,
                  const T *__restrict__ Y, int64_t ldy, int64_t M, int64_t N, int64_t K,
                  int lower, int64_t diag, const int *status) {
  constexpr int BM = Cfg<T>::BM, BN = Cfg<T>::BN, BK = Cfg<T>::BK;
  constexpr int TM = Cfg<T>::TM, TN = Cfg<T>::TN;
  constexpr int HM = TM / 2, HN = TN / 2;  // 16 bytes each
  constexpr int NT = 256;
  constexpr int PADM = BM + 16 / (int)sizeof(T);
  constexpr int PADN = BN + 16 / (int)sizeof(T);
  constexpr int LA = BM * BK / NT, LB = BN * BK / NT;
  static_assert((BM / TM) * (BN / TN) == NT, "thread layout");
  static_assert(HM * sizeof(T) == 16 && HN * sizeof(T) == 16, "16-byte halves");
  using V = typename Vec16<T>::type;

  const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
  if (lower && m0 + BM - 1 + diag < n0) return;  // tile strictly above the diagonal
  if (*reinterpret_cast<const volatile int *>(status) != 0) return;

  __shared__ __align__(16) T As[2][BK][PADM];
  __shared__ __align__(16) T Bs[2][BK][PADN];

  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);

  T ra[LA], rb[LB];
  auto load_global = [&](int64_t k0) {
#pragma unroll
    for (int r = 0; r < LA; ++r) {
      const int e = tid + NT * r;
      const int row = e / BK, kk = e % BK;
      const int64_t gi = m0 + row, gk = k0 + kk;
      ra[r] = (gi < M && gk < K) ? X[gi * ldx + gk] : T(0);
    }
#pragma unroll
    for (int r = 0; r < LB; ++r) {
      const int e = tid + NT * r;
      if (NN) {
        const int kk = e / BN, col = e % BN;
        const int64_t gj = n0 + col, gk = k0 + kk;
        rb[r] = (gj < N && gk < K) ? Y[gk * ldy + gj] : T(0);
      } else {
        const int col = e / BK, kk = e % BK;
        const int64_t gj = n0 + col, gk = k0 + kk;
        rb[r] = (gj < N && gk < K) ? Y[gj * ldy + gk] : T(0);
      }
    }
  };
  auto store_smem = [&](int buf) {
#pragma unroll
    for (int r = 0; r < LA; ++r) {
      const int e = tid + NT * r;
      As[buf][e % BK][e / BK] = ra[r];
    }
#pragma unroll
    for (int r = 0; r < LB; ++r) {
      const int e = tid + NT * r;
      if (NN)
        Bs[buf][e / BN][e % BN] = rb[r];
      else
        Bs[buf][e % BK][e / BK] = rb[r];
    }
  };

  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

  load_global(0);
  store_smem(0);
  __syncthreads();
  int buf = 0;
  for (int64_t k0 = 0; k0 < K; k0 += BK) {
    const bool more = k0 + BK < K;
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

  // epilogue: C -= acc on the elements this thread owns
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int64_t gi = m0 + (i < HM ? ty * HM + i : BM / 2 + ty * HM + (i - HM));
    if (gi >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int64_t gj = n0 + (j < HN ? tx * HN + j : BN / 2 + tx * HN + (j - HN));
      if (gj >= N) continue;
      if (lower && gi + diag < gj) continue;
      T *p = C + gi * ldc + gj;
      *p = *p - acc[i][j];
    }
  }
}

}  // namespace

template <typename T>
cudaError_t launch_update_simt(T *C, int64_t ldc, const T *X, int64_t ldx, const T *Y,
                               int64_t ldy, int64_t M, int64_t N, int64_t K, bool nn, bool lower,
                               int64_t diag, const int *status, cudaStream_t st) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  constexpr int BM = Cfg<T>::BM, BN = Cfg<T>::BN;
  const int64_t gy = (M + BM - 1) / BM, gx = (N + BN - 1) / BN;
  if (gy > 65535) return cudaErrorInvalidConfiguration;
  dim3 grid((unsigned)gx, (unsigned)gy);
  if (nn)
    update_kernel<T, true><<<grid, 256, 0, st>>>(C, ldc, X, ldx, Y, ldy, M, N, K, lower ? 1 : 0,
                                                 diag, status);
  else
    update_kernel<T, false><<<grid, 256, 0, st>>>(C, ldc, X, ldx, Y, ldy, M, N, K, lower ? 1 : 0,
                                                  diag, status);
  count_launch();
  return cudaGetLastError();
}

template cudaError_t launch_update_simt<float>(float *, int64_t, const float *, int64_t,
                                               const float *, int64_t, int64_t, int64_t, int64_t,
                                               bool, bool, int64_t, const int *, cudaStream_t);
template cudaError_t launch_update_simt<double>(double *, int64_t, const double *, int64_t,
                                                const double *, int64_t, int64_t, int64_t,
                                                int64_t, bool, bool, int64_t, const int *,
                                                cudaStream_t);

}  // namespace gb
