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
//    cluster-wide sum: a shuffle tree in each warp, whose result every warp
//    stores into every CTA's shared memory with st.async (distributed shared
//    memory), each store completing bytes on the receiving CTA's mbarrier;
//    a CTA waits on its own mbarrier for the 32 warp sums and adds them with
//    a fixed 32-lane tree, so every thread of every CTA gets the same bits.
//    No CTA-wide or cluster-wide barrier per sum; few warps and trees keep
//    the number of FP64 instructions per sum small (on this GPU an FP64 warp
//    instruction occupies its sub-partition's FP64 unit for many cycles).
//    Every wait is bounded (%globaltimer); on expiry the kernel raises the
//    error word, writes info = -1 and stops.
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
__device__ __forceinline__ uint32_t qr_smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint32_t qr_cluster_addr(const void *p, uint32_t rank) {
  uint32_t remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(qr_smem_u32(p)), "r"(rank));
  return remote;
}
// Store v at the shared::cluster address `addr` and complete its bytes on the
// mbarrier at the shared::cluster address `bar` (both in the same CTA).
__device__ __forceinline__ void qr_st_async(uint32_t addr, double v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];" ::"r"(addr),
               "l"(__double_as_longlong(v)), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void qr_st_async(uint32_t addr, float v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(addr),
               "r"(__float_as_uint(v)), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void qr_mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(qr_smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void qr_mbar_expect(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(qr_smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool qr_mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(qr_smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long qr_now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Cluster-wide sum state of one CTA: 2 x 32 slots (one per warp of the
// cluster) and one mbarrier per half; sum k uses half k & 1, and that
// half's barrier completes its phase (k >> 1) once the 32 warp sums landed.
// A warp stores into half h for sum k + 2 only after its CTA's sum k + 1
// completed, which needs every warp's sum k + 1, which each warp sends only
// after it read sum k's slots: no slot is overwritten before it is read.
template <typename T>
struct ClusterSum {
  T *slots;         // [2][QR_CL * QR_NW]
  uint64_t *bars;   // [2]
  uint32_t rank;
  int k;
  unsigned long long wait_ns;
  bool failed;
};

template <typename T>
__device__ T cluster_sum(T part, ClusterSum<T> &cs) {
  static_assert(QR_NW * QR_CL == 32, "one slot per lane");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int h = cs.k & 1;
  const uint32_t parity = (uint32_t)(cs.k >> 1) & 1u;
  ++cs.k;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if (cs.failed) return part;  // after an expired wait: no more traffic, finish quickly
  T *half = cs.slots + h * 32;
  if (threadIdx.x == 0) qr_mbar_expect(&cs.bars[h], 32u * (uint32_t)sizeof(T));
  if (lane < QR_CL)
    qr_st_async(qr_cluster_addr(&half[cs.rank * QR_NW + warp], lane), part,
                qr_cluster_addr(&cs.bars[h], lane));
  // every lane waits (acquire) for itself; the decisions to go on or to
  // give up are warp votes, so the warp stays converged for its shuffles
  bool ok = qr_mbar_try_wait(&cs.bars[h], parity);
  if (!__all_sync(0xffffffffu, ok)) {
    const unsigned long long until = qr_now_ns() + cs.wait_ns;
    for (;;) {
      ok = ok || qr_mbar_try_wait(&cs.bars[h], parity);
      if (__all_sync(0xffffffffu, ok)) break;
      if (__any_sync(0xffffffffu, qr_now_ns() > until)) {
        cs.failed = true;
        return part;
      }
    }
  }
  T y = half[lane];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
  return y;
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
                    int64_t rows_per, int *status, int *err, long long wait_ns) {
  extern __shared__ __align__(16) unsigned char qr_smem[];
  T *P = reinterpret_cast<T *>(qr_smem);
  __shared__ __align__(16) T slots[2 * 32];
  __shared__ __align__(8) uint64_t bars[2];
  // every kernel before this one on the stream has finished: all CTAs read
  // the same value
  if (*reinterpret_cast<const volatile int *>(status) != 0) return;
  const uint32_t rank = qr_ctarank();
  const int tid = threadIdx.x;
  if (tid == 0) {
    qr_mbar_init(&bars[0], 1);
    qr_mbar_init(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const int64_t r0 = (int64_t)rank * rows_per;
  const int64_t rc = max((int64_t)0, min(rows_per, n - r0));
  // load: consecutive threads take consecutive elements of a row of the block
  for (int64_t e = tid; e < rc * bb; e += QR_NT) {
    const int64_t i = e / bb, j = e % bb;
    P[j * rows_per + i] = Qm[(r0 + i) * ldq + col0 + j];
  }
  qr_cluster_sync();  // barriers initialised in every CTA, block loaded
  ClusterSum<T> cs{slots, bars, rank, 0, (unsigned long long)wait_ns, false};
  int broke = 0;
  for (int c = 0; c < bb && !cs.failed; ++c) {
    T *v = P + (int64_t)c * rows_per;
    for (int j = 0; j < c; ++j) {  // v := v - u (u^T v), u = column j of Q
      const T *u = P + (int64_t)j * rows_per;
      T part = T(0);
      for (int64_t i = tid; i < rc; i += QR_NT) part += u[i] * v[i];
      const T d = cluster_sum(part, cs);
      for (int64_t i = tid; i < rc; i += QR_NT) v[i] = v[i] - u[i] * d;
    }
    T part = T(0);
    for (int64_t i = tid; i < rc; i += QR_NT) part += v[i] * v[i];
    const T nrm = qr_sqrt(cluster_sum(part, cs));
    if (cs.failed) break;
    if (!(nrm > T(0))) {  // every CTA sees the same norm
      broke = c + 1;
      break;
    }
    for (int64_t i = tid; i < rc; i += QR_NT) v[i] = v[i] / nrm;
  }
  // a wait that expired in one thread ends the block for every thread of
  // the CTA; other CTAs find their own waits expiring
  const int any_failed = __syncthreads_or(cs.failed ? 1 : 0);
  if (any_failed) {
    if (tid == 0) {
      atomicOr(err, DEV_ERR_TIMEOUT);
      *status = -1;
    }
  } else if (broke) {
    if (rank == 0 && tid == 0) *status = (int)(col0 + broke);
  } else {
    for (int64_t e = tid; e < rc * bb; e += QR_NT) {
      const int64_t i = e / bb, j = e % bb;
      Qm[(r0 + i) * ldq + col0 + j] = P[j * rows_per + i];
    }
  }
  qr_cluster_sync();  // no CTA leaves while another may still store into it
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

// The same product for a skinny result (M <= 32 rows, M * N <= 4096): one
// CTA per K slice computes all M x N outputs of its slice without padding
// (the tiled kernel would spend a 64-row tile's multiply-adds on M rows);
// KC-row chunks of X and Y are staged in shared memory.
constexpr int SK_KC = 16, SK_RMAX = 16, SK_NT = 256;
template <typename T>
__global__ void __launch_bounds__(SK_NT)
    gemm_tn_skinny_kernel(T *__restrict__ W, int64_t slice_stride, const T *__restrict__ X,
                          int64_t ldx, const T *__restrict__ Y, int64_t ldy, int M, int N,
                          int64_t K, int64_t kslice, const int *status) {
  extern __shared__ __align__(16) unsigned char sk_smem[];
  if (*reinterpret_cast<const volatile int *>(status) != 0) return;
  T *Xs = reinterpret_cast<T *>(sk_smem);
  T *Ys = Xs + SK_KC * M;
  const int tid = threadIdx.x;
  const int64_t kb = (int64_t)blockIdx.x * kslice, ke = min(K, kb + kslice);
  const int nout = M * N;
  T acc[SK_RMAX];
#pragma unroll
  for (int r = 0; r < SK_RMAX; ++r) acc[r] = T(0);
  for (int64_t k0 = kb; k0 < ke; k0 += SK_KC) {
    const int kc = (int)min((int64_t)SK_KC, ke - k0);
    for (int e = tid; e < SK_KC * M; e += SK_NT) {
      const int kk = e / M, i = e % M;
      Xs[e] = kk < kc ? X[(k0 + kk) * ldx + i] : T(0);
    }
    for (int e = tid; e < SK_KC * N; e += SK_NT) {
      const int kk = e / N, j = e % N;
      Ys[e] = kk < kc ? Y[(k0 + kk) * ldy + j] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < SK_RMAX; ++r) {
      const int o = tid + SK_NT * r;
      if (o < nout) {
        const int i = o / N, j = o % N;
        T a = acc[r];
#pragma unroll
        for (int kk = 0; kk < SK_KC; ++kk) a += Xs[kk * M + i] * Ys[kk * N + j];
        acc[r] = a;
      }
    }
    __syncthreads();
  }
  T *Wz = W + (int64_t)blockIdx.x * slice_stride;
#pragma unroll
  for (int r = 0; r < SK_RMAX; ++r) {
    const int o = tid + SK_NT * r;
    if (o < nout) Wz[o] = acc[r];
  }
}

// C[i][j] = sum_z W[z][i][j] over the K slices of the gemm_tn kernels: one
// warp per element, lane l adding slices l, l + 32, ... in ascending order,
// then a fixed shuffle tree (deterministic: the same bits on every run).
template <typename T>
__global__ void sum_slices_kernel(T *__restrict__ C, int64_t ldc, const T *__restrict__ W,
                                  int64_t M, int64_t N, int slices, const int *status) {
  if (*reinterpret_cast<const volatile int *>(status) != 0) return;
  const int64_t total = M * N;
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < total; e += warps) {
    T acc = T(0);
    for (int z = lane; z < slices; z += 32) acc += W[(int64_t)z * total + e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) C[(e / N) * ldc + e % N] = acc;
  }
}

}  // namespace

int64_t qr_panel_max_cols(int64_t n, size_t esz) {
  const int64_t rows_per = std::max<int64_t>(1, (n + QR_CL - 1) / QR_CL);
  return std::max<int64_t>(0, (int64_t)(200 * 1024) / (rows_per * (int64_t)esz));
}

template <typename T>
cudaError_t launch_qr_panel(T *Qm, int64_t ldq, int64_t n, int64_t col0, int bb, int *status,
                            int *err, int64_t spin_limit, cudaStream_t st) {
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
  // A sum takes about a microsecond; one second bounds every single wait.
  // The floor of 10 ms keeps a small spin limit from cutting off sums that
  // are merely in flight: the give-up path is for a wait that cannot end.
  const long long wait_ns = std::max<long long>(
      10000000LL, std::min<long long>((long long)spin_limit * 100LL, 1000000000LL));
  count_launch();
  return cudaLaunchKernelEx(&cfg, qr_panel_kernel<T>, Qm, ldq, n, col0, bb, rows_per, status, err,
                            wait_ns);
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
  if (!upper && M <= 32 && M * N <= SK_NT * SK_RMAX && K >= 1 &&
      (size_t)SK_KC * (size_t)(M + N) * sizeof(T) <= 48 * 1024) {
    // skinny result: K slices of at least SK_KC rows over up to 2 waves of CTAs
    int64_t slices = std::min<int64_t>(2 * (int64_t)sm_count, (K + SK_KC - 1) / SK_KC);
    while (slices > 1 && (size_t)slices * (size_t)M * (size_t)N * sizeof(T) > work_bytes) slices /= 2;
    if (work && slices >= 1 && (size_t)slices * (size_t)M * (size_t)N * sizeof(T) <= work_bytes) {
      const int64_t kslice = ((K + slices - 1) / slices + SK_KC - 1) / SK_KC * SK_KC;
      slices = (K + kslice - 1) / kslice;
      const size_t smem = (size_t)SK_KC * (size_t)(M + N) * sizeof(T);
      T *W = reinterpret_cast<T *>(work);
      gemm_tn_skinny_kernel<T><<<(unsigned)slices, SK_NT, smem, st>>>(
          W, M * N, X, ldx, Y, ldy, (int)M, (int)N, K, kslice, status);
      const int64_t total = M * N;
      const unsigned g2 = (unsigned)std::min<int64_t>((total * 32 + 255) / 256, 8192);
      sum_slices_kernel<T><<<g2, 256, 0, st>>>(C, ldc, W, M, N, (int)slices, status);
      count_launch(2);
      return cudaGetLastError();
    }
  }
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
  const unsigned g2 = (unsigned)std::min<int64_t>((total * 32 + 255) / 256, 8192);
  sum_slices_kernel<T><<<g2, 256, 0, st>>>(C, ldc, W, M, N, (int)slices, status);
  count_launch(2);
  return cudaGetLastError();
}

template cudaError_t launch_qr_panel<double>(double *, int64_t, int64_t, int64_t, int, int *,
                                             int *, int64_t, cudaStream_t);
template cudaError_t launch_qr_panel<float>(float *, int64_t, int64_t, int64_t, int, int *, int *,
                                            int64_t, cudaStream_t);
template cudaError_t launch_gemm_tn<double>(double *, int64_t, const double *, int64_t,
                                            const double *, int64_t, int64_t, int64_t, int64_t,
                                            bool, const int *, void *, size_t, int,
                                            cudaStream_t);
template cudaError_t launch_gemm_tn<float>(float *, int64_t, const float *, int64_t,
                                           const float *, int64_t, int64_t, int64_t, int64_t, bool,
                                           const int *, void *, size_t, int, cudaStream_t);

}  // namespace gb
