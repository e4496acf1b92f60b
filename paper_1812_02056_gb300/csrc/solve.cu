// Solves with the factors of Algorithms 1 and 2 (arXiv:1812.02056), the
// FP64 residual of iterative refinement, and the FP64 backward error.
//
// Triangular solve: one launch per solve.  The n rows are cut into blocks
// of TB rows; CTAs take block rows in dependence order from an atomic ticket
// (so a CTA only ever waits on blocks already owned by running CTAs), apply
// every finished block's contribution as soon as its flag is published, then
// substitute within their own diagonal block and publish.  Every wait is
// bounded by a %globaltimer deadline; on expiry the kernel raises
// DEV_ERR_TIMEOUT in the error word, every other waiter sees it and returns,
// and the host reports GB_ERR_TIMEOUT.
#include <math.h>

#include "gb_internal.cuh"

namespace gb {
namespace {

constexpr int TB = 32;       // rows per block
constexpr int NRC = 32;      // right-hand sides per chunk
constexpr int TRSM_THREADS = 256;
constexpr int TRSM_MAX_GROUPS = 4;  // right-hand-side groups of 16 per trsm_inv launch

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(int *p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Element (i, k) of op(F) for the three solve kinds.
template <typename Tf>
__device__ __forceinline__ Tf op_elem(const Tf *F, int64_t ldf, int kind, int64_t i, int64_t k) {
  return kind == TRSM_LOWER_T ? F[k * ldf + i] : F[i * ldf + k];
}

template <typename Tf, typename Tc>
__global__ void __launch_bounds__(TRSM_THREADS)
    trsm_kernel(const Tf *__restrict__ F, int64_t ldf, double *B, int64_t ldb, int64_t n,
                int64_t nrhs, int kind, int *ticket, int *flags, unsigned epoch, int *err,
                long long wait_ns) {
  __shared__ Tc Fs[TB][TB + 1];
  __shared__ Tc Xs[TB][NRC + 1];
  __shared__ Tc Acc[TB][NRC + 1];
  __shared__ int s_ib, s_abort;
  const int tid = threadIdx.x;
  const int nb = (int)((n + TB - 1) / TB);
  const bool fwd = (kind == TRSM_LOWER);
  if (tid == 0) {
    const int t = atomicAdd(ticket, 1);
    s_ib = fwd ? t : nb - 1 - t;
    s_abort = 0;
  }
  __syncthreads();
  const int ib = s_ib;
  if (ib < 0 || ib >= nb) return;
  const int64_t r0 = (int64_t)ib * TB;
  const int rows = (int)min64(TB, n - r0);
  // thread -> (row, 4 columns) of the chunk
  const int tr = tid / (NRC / 4), tc = (tid % (NRC / 4)) * 4;

  for (int64_t c0 = 0; c0 < nrhs; c0 += NRC) {
    const int cols = (int)min64(NRC, nrhs - c0);
    Tc acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      acc[q] = (tr < rows && tc + q < cols) ? (Tc)B[(r0 + tr) * ldb + c0 + tc + q] : Tc(0);
    // contributions of the finished blocks, in dependence order
    for (int step = 0; step < (fwd ? ib : nb - 1 - ib); ++step) {
      const int jb = fwd ? step : nb - 1 - step;
      if (tid == 0) {
        const long long t0 = (long long)globaltimer_ns();
        while (ld_acquire(&flags[jb]) != (int)epoch) {
          if (ld_acquire(err) & DEV_ERR_TIMEOUT) {
            s_abort = 1;
            break;
          }
          if ((long long)globaltimer_ns() - t0 > wait_ns) {
            atomicOr(err, DEV_ERR_TIMEOUT);
            s_abort = 1;
            break;
          }
          __nanosleep(64);
        }
      }
      __syncthreads();
      if (s_abort) return;
      const int64_t k0 = (int64_t)jb * TB;
      const int kr = (int)min64(TB, n - k0);
      for (int idx = tid; idx < TB * TB; idx += TRSM_THREADS) {
        const int i = idx / TB, k = idx % TB;
        Fs[i][k] = (i < rows && k < kr) ? (Tc)op_elem(F, ldf, kind, r0 + i, k0 + k) : Tc(0);
      }
      for (int idx = tid; idx < TB * NRC; idx += TRSM_THREADS) {
        const int k = idx / NRC, c = idx % NRC;
        Xs[k][c] = (k < kr && c < cols) ? (Tc)__ldcg(&B[(k0 + k) * ldb + c0 + c]) : Tc(0);
      }
      __syncthreads();
#pragma unroll 8
      for (int k = 0; k < TB; ++k) {
        const Tc f = Fs[tr][k];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = acc[q] - f * Xs[k][tc + q];
      }
      __syncthreads();
    }
    // substitution inside the diagonal block
    for (int idx = tid; idx < TB * TB; idx += TRSM_THREADS) {
      const int i = idx / TB, k = idx % TB;
      Fs[i][k] = (i < rows && k < rows) ? (Tc)op_elem(F, ldf, kind, r0 + i, r0 + k) : Tc(0);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) Acc[tr][tc + q] = acc[q];
    __syncthreads();
    if (tid < NRC) {
      const int c = tid;
      if (fwd) {
        for (int i = 0; i < rows; ++i) {
          Tc v = Acc[i][c];
          for (int k = 0; k < i; ++k) v = v - Fs[i][k] * Acc[k][c];
          Acc[i][c] = v / Fs[i][i];
        }
      } else {
        for (int i = rows - 1; i >= 0; --i) {
          Tc v = Acc[i][c];
          for (int k = i + 1; k < rows; ++k) v = v - Fs[i][k] * Acc[k][c];
          Acc[i][c] = (kind == TRSM_UNIT_UPPER) ? v : v / Fs[i][i];
        }
      }
    }
    __syncthreads();
    for (int idx = tid; idx < TB * NRC; idx += TRSM_THREADS) {
      const int i = idx / NRC, c = idx % NRC;
      if (i < rows && c < cols) B[(r0 + i) * ldb + c0 + c] = (double)Acc[i][c];
    }
    __syncthreads();
  }
  if (tid == 0) {
    __threadfence();
    st_release(&flags[ib], (int)epoch);
  }
}

// ---------------------------------------- solve with inverted diagonal blocks
// Pre-pass: Dinv[b] = inverse of the b-th BS x BS diagonal block of op(F),
// one CTA of BS threads per block, thread j computing column j of the
// inverse by substitution.  The solve below then finishes a block with the
// small product X_b = Dinv[b] * (b - contributions): no dependent chain of
// length BS on the critical path.  BS = 64 for FP32 factors (half the
// sequential blocks of a sweep), 32 for FP64 (whose multiply-adds on the
// critical path are slow on this GPU).
template <typename Tc>
constexpr int inv_block() {
  return sizeof(Tc) == 4 ? 64 : 32;
}

template <typename Tf, typename Tc>
__global__ void __launch_bounds__(inv_block<Tc>())
    diag_inv_kernel(const Tf *__restrict__ F, int64_t ldf, int64_t n, int kind,
                    Tc *__restrict__ Dinv) {
  constexpr int TB = inv_block<Tc>();
  // Bs: the block, Ys: column j of the inverse, built by thread j ([TB][TB + 1] each)
  extern __shared__ __align__(16) unsigned char inv_smem[];
  Tc (*Bs)[TB + 1] = reinterpret_cast<Tc (*)[TB + 1]>(inv_smem);
  Tc (*Ys)[TB + 1] = Bs + TB;
  const int b = blockIdx.x, j = threadIdx.x;
  const int64_t r0 = (int64_t)b * TB;
  const int rows = (int)min64(TB, n - r0);
  for (int i = 0; i < TB; ++i) {
    Bs[i][j] = (i < rows && j < rows) ? (Tc)op_elem(F, ldf, kind, r0 + i, r0 + j) : Tc(0);
    Ys[i][j] = Tc(0);
  }
  __syncthreads();
  if (j < rows) {
    if (kind == TRSM_LOWER) {  // lower, non-unit: forward substitution on e_j
      for (int i = j; i < rows; ++i) {
        Tc v = (i == j) ? Tc(1) : Tc(0);
        for (int k = j; k < i; ++k) v = v - Bs[i][k] * Ys[k][j];
        Ys[i][j] = v / Bs[i][i];
      }
    } else {  // upper (L^T, or unit U): back substitution on e_j
      const bool unit = (kind == TRSM_UNIT_UPPER);
      for (int i = j; i >= 0; --i) {
        Tc v = (i == j) ? Tc(1) : Tc(0);
        for (int k = i + 1; k <= j; ++k) v = v - Bs[i][k] * Ys[k][j];
        Ys[i][j] = unit ? v : v / Bs[i][i];
      }
    }
  }
  Tc *D = Dinv + (int64_t)b * TB * TB;
  for (int i = 0; i < TB; ++i) D[i * TB + j] = (i < rows && j < rows) ? Ys[i][j] : Tc(0);
}

// Coupling blocks of the solve: for position p >= 1 (block b, previous
// position's block bp), M_p = Dinv[b] op(F)[b rows, bp columns], so that
// X_b = Dinv[b] (B_b - sum over earlier positions) - M_p X_bp puts a single
// BS x BS product on the dependence chain.
template <typename Tc>
__global__ void __launch_bounds__(TRSM_THREADS)
    coupling_kernel(const Tc *__restrict__ F, int64_t ldf, const Tc *__restrict__ Dinv, int64_t n,
                    int kind, Tc *__restrict__ M) {
  constexpr int BS = inv_block<Tc>();
  extern __shared__ __align__(16) unsigned char cpl_smem[];  // Ds, Os: [BS][BS + 1] each
  Tc (*Ds)[BS + 1] = reinterpret_cast<Tc (*)[BS + 1]>(cpl_smem);
  Tc (*Os)[BS + 1] = Ds + BS;
  const int nb = (int)((n + BS - 1) / BS);
  const int p = blockIdx.x + 1;
  if (p >= nb) return;
  const bool fwd = (kind == TRSM_LOWER);
  const int b = fwd ? p : nb - 1 - p, bp = fwd ? p - 1 : nb - p;
  const int64_t r0 = (int64_t)b * BS, c0 = (int64_t)bp * BS;
  const int rows = (int)min64(BS, n - r0), cw = (int)min64(BS, n - c0);
  const Tc *D = Dinv + (int64_t)b * BS * BS;
  for (int idx = threadIdx.x; idx < BS * BS; idx += TRSM_THREADS) {
    const int i = idx / BS, k = idx % BS;
    Ds[i][k] = D[idx];
    Os[i][k] = (i < rows && k < cw) ? op_elem(F, ldf, kind, r0 + i, c0 + k) : Tc(0);
  }
  __syncthreads();
  Tc *Mo = M + (int64_t)p * BS * BS;
  for (int idx = threadIdx.x; idx < BS * BS; idx += TRSM_THREADS) {
    const int i = idx / BS, k = idx % BS;
    Tc v = Tc(0);
    for (int j = 0; j < BS; ++j) v = v + Ds[i][j] * Os[j][k];
    Mo[idx] = v;
  }
}

// Solve with inverted diagonal blocks.  CTAs take block rows (BS rows) in
// dependence order from a ticket (position t: block t forward, block
// nb - 1 - t backward).  `progress` counts the finished positions; blocks
// finish in order, so progress = p means positions 0 .. p - 1 are solved.  A
// CTA walks its row panel, except the previous position's block, in chunks
// of up to KC columns: the op(F) part of a chunk is loaded once, before any
// wait (it does not depend on X), as is the CTA's Dinv block; then each wait
// applies as many of the chunk's blocks as are finished when it looks (all
// of them far behind the wavefront, one per wait when caught up), so a CTA
// that trails the wavefront re-reads neither op(F) nor X.  Then
// Y = Dinv[b] (B_b - contributions) before the previous position is waited
// for, and after it X_b = Y - M_t X_prev with the coupling block M_t
// (coupling_kernel), stored and published.  Every wait is bounded by a
// %globaltimer deadline; on expiry the kernel raises DEV_ERR_TIMEOUT in the
// error word, every other waiter sees it and returns, and the host reports
// GB_ERR_TIMEOUT.
template <typename Tc>
struct TrsmCfg {
  static constexpr int BS = inv_block<Tc>();
  static constexpr int KC = sizeof(Tc) == 4 ? 256 : 64;  // columns per chunk
  static constexpr int NRC = 16;                         // right-hand sides per pass
  static constexpr int TPR = TRSM_THREADS / BS;          // threads per row
  static constexpr int OPT = NRC / TPR;                  // outputs per thread
  static constexpr size_t SMEM =
      sizeof(Tc) * ((size_t)BS * (KC + 1) + (size_t)KC * (NRC + 1) + (size_t)BS * (BS + 1));
};

// One group of at most NRC right-hand sides: the same steps as
// trsm_inv_kernel with TRSM_GROUPS = 1, in the form that keeps the register
// count low (40 instead of 109 for FP32), which measured faster for the
// common solve with 16 right-hand sides.
template <typename Tf, typename Tc>
__global__ void __launch_bounds__(TRSM_THREADS)
    trsm_inv1_kernel(const Tf *__restrict__ F, int64_t ldf, const Tc *__restrict__ Dinv,
                    const Tc *__restrict__ Mc, double *B, int64_t ldb, int64_t n, int64_t nrhs,
                    int kind, int *ticket, int *progress, int *err, long long wait_ns,
                    int withhold) {
  using C = TrsmCfg<Tc>;
  constexpr int BS = C::BS, KC = C::KC, NRC = C::NRC, OPT = C::OPT;
  static_assert(KC % BS == 0 && C::TPR * OPT == NRC, "layout");
  extern __shared__ __align__(16) unsigned char trsm_smem[];
  Tc *Fs = reinterpret_cast<Tc *>(trsm_smem);   // [BS][KC + 1]
  Tc *Xs = Fs + (size_t)BS * (KC + 1);           // [KC][NRC + 1]
  Tc *Ds = Xs + (size_t)KC * (NRC + 1);          // [BS][BS + 1]
  __shared__ int s_t, s_avail, s_abort;
  const int tid = threadIdx.x;
  const int nb = (int)((n + BS - 1) / BS);
  const bool fwd = (kind == TRSM_LOWER);
  if (tid == 0) {
    s_t = atomicAdd(ticket, 1);
    s_abort = 0;
  }
  __syncthreads();
  const int t = s_t;
  if (t < 0 || t >= nb) return;
  const int ib = fwd ? t : nb - 1 - t;
  const int64_t r0 = (int64_t)ib * BS;
  const int rows = (int)min64(BS, n - r0);
  const int tr = tid / C::TPR, tc = (tid % C::TPR) * OPT;
  {
    const Tc *D = Dinv + (int64_t)ib * BS * BS;
    for (int idx = tid; idx < BS * BS; idx += TRSM_THREADS) Ds[(idx / BS) * (BS + 1) + idx % BS] = D[idx];
  }

  // columns of op(F) for positions [p0, p0 + w): forward blocks p0 .. p0+w-1,
  // backward blocks nb-p0-w .. nb-p0-1 (both as one ascending column range)
  auto col_range = [&](int p0, int w, int64_t &c0, int64_t &c1) {
    const int64_t b0 = fwd ? p0 : nb - p0 - w;
    c0 = b0 * BS;
    c1 = min64((b0 + w) * BS, n);
  };

  // every thread: wait until position p is finished; the number of finished
  // positions, or -1 once a wait has expired (here or in another CTA)
  auto wait_pos = [&](int p) {
    if (tid == 0) {
      int spins = 0, avail = ld_acquire(progress);
      const long long t0 = (long long)globaltimer_ns();
      while (avail <= p) {
        if ((++spins & 255) == 0) {
          if (ld_acquire(err) & DEV_ERR_TIMEOUT) {
            s_abort = 1;
            break;
          }
          if ((long long)globaltimer_ns() - t0 > wait_ns) {
            atomicOr(err, DEV_ERR_TIMEOUT);
            s_abort = 1;
            break;
          }
        }
        avail = ld_acquire(progress);
      }
      s_avail = avail;
    }
    __syncthreads();
    return s_abort ? -1 : s_avail;
  };

  // positions 0 .. t - 2 go through the chunks; the previous position t - 1
  // enters through the coupling block M_t = Dinv[b] op(F)[b, previous block]
  const int tmain = t > 0 ? t - 1 : 0;
  for (int64_t rc0 = 0; rc0 < nrhs; rc0 += NRC) {
    const int cols = (int)min64(NRC, nrhs - rc0);
    if (rc0 > 0 && t > 0) {  // the previous group left M_t in Ds
      const Tc *D = Dinv + (int64_t)ib * BS * BS;
      for (int idx = tid; idx < BS * BS; idx += TRSM_THREADS) Ds[(idx / BS) * (BS + 1) + idx % BS] = D[idx];
    }
    Tc acc[OPT];
#pragma unroll
    for (int q = 0; q < OPT; ++q)
      acc[q] = (tr < rows && tc + q < cols) ? (Tc)B[(r0 + tr) * ldb + rc0 + tc + q] : Tc(0);
    int done = 0;
    while (done < tmain) {
      // op(F) for the next chunk of positions, loaded once, before waiting
      // for any of its X
      const int wmax = min(KC / BS, tmain - done);
      int64_t f0, f1;
      col_range(done, wmax, f0, f1);
      const int fw = (int)(f1 - f0);
      for (int idx = tid; idx < BS * KC; idx += TRSM_THREADS) {
        const int i = idx / KC, k = idx % KC;
        Fs[i * (KC + 1) + k] = (i < rows && k < fw) ? (Tc)op_elem(F, ldf, kind, r0 + i, f0 + k) : Tc(0);
      }
      int applied = 0;  // positions of this chunk applied so far
      while (applied < wmax) {
        const int p0 = done + applied;
        const int avail = wait_pos(p0);
        if (avail < 0) return;
        // the finished positions p0 .. p0 + w - 1 of this chunk
        const int w = min(wmax - applied, avail - p0);
        int64_t c0, c1;
        col_range(p0, w, c0, c1);
        const int kw = (int)(c1 - c0);
        // only the kw rows the products below read
        for (int idx = tid; idx < kw * NRC; idx += TRSM_THREADS) {
          const int k = idx / NRC, c = idx % NRC;
          Xs[k * (NRC + 1) + c] = c < cols ? (Tc)__ldcg(&B[(c0 + k) * ldb + rc0 + c]) : Tc(0);
        }
        __syncthreads();
        // blocks in position order (backward: descending), columns ascending
        // inside a block: the same order for any chunking, so results do not
        // depend on how far the other blocks had got
        for (int pb = 0; pb < w; ++pb) {
          const int64_t b0 = fwd ? (int64_t)(p0 + pb) : (int64_t)(nb - 1 - p0 - pb);
          const int64_t bc0 = b0 * BS;
          const int bw = (int)min64(BS, n - bc0);
          const Tc *Fr = Fs + tr * (KC + 1) + (bc0 - f0);
          const Tc *Xb = Xs + (bc0 - c0) * (NRC + 1) + tc;
          for (int k = 0; k < bw; ++k) {
            const Tc f = Fr[k];
            const Tc *xk = Xb + k * (NRC + 1);
#pragma unroll
            for (int q = 0; q < OPT; ++q) acc[q] = acc[q] - f * xk[q];
          }
        }
        __syncthreads();
        applied += w;
      }
      done += wmax;
    }
    // Y = Dinv[b] * acc, before the previous position is waited for
#pragma unroll
    for (int q = 0; q < OPT; ++q) Xs[tr * (NRC + 1) + tc + q] = acc[q];
    __syncthreads();
    Tc out[OPT];
#pragma unroll
    for (int q = 0; q < OPT; ++q) out[q] = Tc(0);
#pragma unroll 8
    for (int k = 0; k < BS; ++k) {
      const Tc d = Ds[tr * (BS + 1) + k];
#pragma unroll
      for (int q = 0; q < OPT; ++q) out[q] = out[q] + d * Xs[k * (NRC + 1) + tc + q];
    }
    if (t > 0) {
      // X_b = Y - M_t X_{t-1}: one product on the dependence chain
      __syncthreads();  // Ds and Xs are read
      const Tc *M = Mc + (int64_t)t * BS * BS;
      for (int idx = tid; idx < BS * BS; idx += TRSM_THREADS) Ds[(idx / BS) * (BS + 1) + idx % BS] = M[idx];
      if (wait_pos(t - 1) < 0) return;
      int64_t c0, c1;
      col_range(t - 1, 1, c0, c1);
      const int kw = (int)(c1 - c0);
      for (int idx = tid; idx < kw * NRC; idx += TRSM_THREADS) {
        const int k = idx / NRC, c = idx % NRC;
        Xs[k * (NRC + 1) + c] = c < cols ? (Tc)__ldcg(&B[(c0 + k) * ldb + rc0 + c]) : Tc(0);
      }
      __syncthreads();
#pragma unroll 8
      for (int k = 0; k < kw; ++k) {
        const Tc m = Ds[tr * (BS + 1) + k];
#pragma unroll
        for (int q = 0; q < OPT; ++q) out[q] = out[q] - m * Xs[k * (NRC + 1) + tc + q];
      }
    }
#pragma unroll
    for (int q = 0; q < OPT; ++q)
      if (tr < rows && tc + q < cols) B[(r0 + tr) * ldb + rc0 + tc + q] = (double)out[q];
    __syncthreads();
  }
  if (tid == 0 && t != withhold) {  // (test hook: see trsm_inv_kernel)
    __threadfence();
    st_release(progress, t + 1);  // every position before t is finished: progress was t
  }
}

// Resident CTAs per SM the registers must allow: FP64 blocks with one group
// keep six resident (their shared memory allows it); FP32 with one group is
// left to the compiler (its shared memory holds it to two CTAs anyway); more
// groups need two.
template <typename Tc, int G>
constexpr int trsm_min_blocks() {
  return G == 1 ? (sizeof(Tc) == 8 ? 6 : 1) : 2;
}

template <typename Tf, typename Tc, int TRSM_GROUPS>
__global__ void __launch_bounds__(TRSM_THREADS, trsm_min_blocks<Tc, TRSM_GROUPS>())
    trsm_inv_kernel(const Tf *__restrict__ F, int64_t ldf, const Tc *__restrict__ Dinv,
                    const Tc *__restrict__ Mc, double *B, int64_t ldb, int64_t n, int64_t nrhs,
                    int kind, int *ticket, int *progress, int *err, long long wait_ns,
                    int withhold) {
  using C = TrsmCfg<Tc>;
  constexpr int BS = C::BS, KC = C::KC, NRC = C::NRC, OPT = C::OPT;
  static_assert(KC % BS == 0 && C::TPR * OPT == NRC, "layout");
  extern __shared__ __align__(16) unsigned char trsm_smem[];
  Tc *Fs = reinterpret_cast<Tc *>(trsm_smem);   // [BS][KC + 1]
  Tc *Xs = Fs + (size_t)BS * (KC + 1);           // [KC][NRC + 1]
  Tc *Ds = Xs + (size_t)KC * (NRC + 1);          // [BS][BS + 1]
  __shared__ int s_t, s_avail, s_abort;
  const int tid = threadIdx.x;
  const int nb = (int)((n + BS - 1) / BS);
  const bool fwd = (kind == TRSM_LOWER);
  if (tid == 0) {
    s_t = atomicAdd(ticket, 1);
    s_abort = 0;
  }
  __syncthreads();
  const int t = s_t;
  if (t < 0 || t >= nb) return;
  const int ib = fwd ? t : nb - 1 - t;
  const int64_t r0 = (int64_t)ib * BS;
  const int rows = (int)min64(BS, n - r0);
  const int tr = tid / C::TPR, tc = (tid % C::TPR) * OPT;
  {
    const Tc *D = Dinv + (int64_t)ib * BS * BS;
    for (int idx = tid; idx < BS * BS; idx += TRSM_THREADS) Ds[(idx / BS) * (BS + 1) + idx % BS] = D[idx];
  }

  // columns of op(F) for positions [p0, p0 + w): forward blocks p0 .. p0+w-1,
  // backward blocks nb-p0-w .. nb-p0-1 (both as one ascending column range)
  auto col_range = [&](int p0, int w, int64_t &c0, int64_t &c1) {
    const int64_t b0 = fwd ? p0 : nb - p0 - w;
    c0 = b0 * BS;
    c1 = min64((b0 + w) * BS, n);
  };

  // every thread: wait until position p is finished; the number of finished
  // positions, or -1 once a wait has expired (here or in another CTA)
  auto wait_pos = [&](int p) {
    if (tid == 0) {
      int spins = 0, avail = ld_acquire(progress);
      const long long t0 = (long long)globaltimer_ns();
      while (avail <= p) {
        if ((++spins & 255) == 0) {
          if (ld_acquire(err) & DEV_ERR_TIMEOUT) {
            s_abort = 1;
            break;
          }
          if ((long long)globaltimer_ns() - t0 > wait_ns) {
            atomicOr(err, DEV_ERR_TIMEOUT);
            s_abort = 1;
            break;
          }
        }
        avail = ld_acquire(progress);
      }
      s_avail = avail;
    }
    __syncthreads();
    return s_abort ? -1 : s_avail;
  };

  // positions 0 .. t - 2 go through the chunks; the previous position t - 1
  // enters through the coupling block M_t = Dinv[b] op(F)[b, previous block].
  // All right-hand-side groups (NRC columns each, at most TRSM_GROUPS) are
  // carried together: each chunk of finished positions is applied to every
  // group before the next wait, so only one pass over the row panel lies on
  // the chain between this position and the next.
  const int tmain = t > 0 ? t - 1 : 0;
  const int ng = (int)((nrhs + NRC - 1) / NRC);  // <= TRSM_GROUPS (the launcher slices)
  Tc acc[TRSM_GROUPS][OPT];
#pragma unroll
  for (int g = 0; g < TRSM_GROUPS; ++g)
#pragma unroll
    for (int q = 0; q < OPT; ++q) {
      const int64_t c = (int64_t)g * NRC + tc + q;
      acc[g][q] = (g < ng && tr < rows && c < nrhs) ? (Tc)B[(r0 + tr) * ldb + c] : Tc(0);
    }
  // X rows [c0, c0 + kw) of group g into Xs
  auto load_x = [&](int g, int64_t c0, int kw) {
    const int64_t cb = (int64_t)g * NRC;
    for (int idx = tid; idx < kw * NRC; idx += TRSM_THREADS) {
      const int k = idx / NRC, c = idx % NRC;
      Xs[k * (NRC + 1) + c] = cb + c < nrhs ? (Tc)__ldcg(&B[(c0 + k) * ldb + cb + c]) : Tc(0);
    }
  };
  int done = 0;
  while (done < tmain) {
    // op(F) for the next chunk of positions, loaded once, before waiting
    // for any of its X
    const int wmax = min(KC / BS, tmain - done);
    int64_t f0, f1;
    col_range(done, wmax, f0, f1);
    const int fw = (int)(f1 - f0);
    for (int idx = tid; idx < BS * KC; idx += TRSM_THREADS) {
      const int i = idx / KC, k = idx % KC;
      Fs[i * (KC + 1) + k] = (i < rows && k < fw) ? (Tc)op_elem(F, ldf, kind, r0 + i, f0 + k) : Tc(0);
    }
    int applied = 0;  // positions of this chunk applied so far
    while (applied < wmax) {
      const int p0 = done + applied;
      const int avail = wait_pos(p0);
      if (avail < 0) return;
      // the finished positions p0 .. p0 + w - 1 of this chunk
      const int w = min(wmax - applied, avail - p0);
      int64_t c0, c1;
      col_range(p0, w, c0, c1);
      const int kw = (int)(c1 - c0);
#pragma unroll
      for (int g = 0; g < TRSM_GROUPS; ++g) {
        if (g >= ng) continue;  // uniform
        load_x(g, c0, kw);  // only the kw rows the products below read
        __syncthreads();
        // blocks in position order (backward: descending), columns ascending
        // inside a block: the same order for any chunking, so results do not
        // depend on how far the other blocks had got
        for (int pb = 0; pb < w; ++pb) {
          const int64_t b0 = fwd ? (int64_t)(p0 + pb) : (int64_t)(nb - 1 - p0 - pb);
          const int64_t bc0 = b0 * BS;
          const int bw = (int)min64(BS, n - bc0);
          const Tc *Fr = Fs + tr * (KC + 1) + (bc0 - f0);
          const Tc *Xb = Xs + (bc0 - c0) * (NRC + 1) + tc;
          for (int k = 0; k < bw; ++k) {
            const Tc f = Fr[k];
            const Tc *xk = Xb + k * (NRC + 1);
#pragma unroll
            for (int q = 0; q < OPT; ++q) acc[g][q] = acc[g][q] - f * xk[q];
          }
        }
        __syncthreads();
      }
      applied += w;
    }
    done += wmax;
  }
  // Y = Dinv[b] * acc per group, before the previous position is waited for
  Tc out[TRSM_GROUPS][OPT];
#pragma unroll
  for (int g = 0; g < TRSM_GROUPS; ++g) {
#pragma unroll
    for (int q = 0; q < OPT; ++q) out[g][q] = Tc(0);
    if (g >= ng) continue;  // uniform
#pragma unroll
    for (int q = 0; q < OPT; ++q) Xs[tr * (NRC + 1) + tc + q] = acc[g][q];
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < BS; ++k) {
      const Tc d = Ds[tr * (BS + 1) + k];
#pragma unroll
      for (int q = 0; q < OPT; ++q) out[g][q] = out[g][q] + d * Xs[k * (NRC + 1) + tc + q];
    }
    __syncthreads();  // Xs is rewritten by the next group
  }
  if (t > 0) {
    // X_b = Y - M_t X_{t-1}: one product per group on the dependence chain
    const Tc *M = Mc + (int64_t)t * BS * BS;
    for (int idx = tid; idx < BS * BS; idx += TRSM_THREADS) Ds[(idx / BS) * (BS + 1) + idx % BS] = M[idx];
    if (wait_pos(t - 1) < 0) return;
    int64_t c0, c1;
    col_range(t - 1, 1, c0, c1);
    const int kw = (int)(c1 - c0);
#pragma unroll
    for (int g = 0; g < TRSM_GROUPS; ++g) {
      if (g >= ng) continue;  // uniform
      load_x(g, c0, kw);
      __syncthreads();
#pragma unroll 8
      for (int k = 0; k < kw; ++k) {
        const Tc m = Ds[tr * (BS + 1) + k];
#pragma unroll
        for (int q = 0; q < OPT; ++q) out[g][q] = out[g][q] - m * Xs[k * (NRC + 1) + tc + q];
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int g = 0; g < TRSM_GROUPS; ++g)
#pragma unroll
    for (int q = 0; q < OPT; ++q) {
      const int64_t c = (int64_t)g * NRC + tc + q;
      if (g < ng && tr < rows && c < nrhs) B[(r0 + tr) * ldb + c] = (double)out[g][q];
    }
  __syncthreads();  // every row of X_b is stored before thread 0 publishes it
  // (test hook: position `withhold` never publishes, so the waits for it
  // run out; -1 in every normal call)
  if (tid == 0 && t != withhold) {
    __threadfence();
    st_release(progress, t + 1);  // every position before t is finished: progress was t
  }
}

// ------------------------------------------------------------- residual
// R = B - A X in FP64: a tiled product.  A CTA of RES_THREADS threads owns
// RES_ROWS rows and RES_NC right-hand sides; k-chunks of A (rows x RES_KC, padded to
// an odd stride) and of X (RES_KC x RES_NC) are staged in shared memory with
// coalesced loads; thread (r, g) accumulates row r against columns
// 4g .. 4g + 3 over k in ascending order.  Each element of A is read once;
// the kernel is bound by the FP64 units (16 multiply-adds per element).
constexpr int RES_ROWS = 16;  // n / 16 CTAs: even load over the SMs
constexpr int RES_KC = 64;
constexpr int RES_NC = 16;
constexpr int RES_THREADS = RES_ROWS * RES_NC / 4;  // 64

__device__ __forceinline__ double finite_abs(double v) {
  const double a = fabs(v);
  return a <= 1.7976931348623157e308 ? a : __longlong_as_double(0x7ff0000000000000LL);
}

__device__ __forceinline__ void atomic_max_nonneg(double *addr, double v) {
  // non-negative doubles order like their bit patterns as signed integers
  atomicMax(reinterpret_cast<long long *>(addr), __double_as_longlong(v));
}

// With `P` (gridDim.y K slices of `kslice` columns): slice blockIdx.y writes
// its partial products P[slice][i][c] instead; residual_finish_kernel sums
// the slices in order.  Small orders use slices so that the grid still
// fills every SM.
__global__ void __launch_bounds__(RES_THREADS)
    residual_kernel(const double *__restrict__ A, int64_t lda, const double *__restrict__ X,
                    int64_t ldx, const double *__restrict__ B, int64_t ldb, double *__restrict__ R,
                    int64_t ldr, int64_t n, int64_t nrhs, double *norms, int64_t kslice,
                    double *__restrict__ P) {
  __shared__ double As[RES_ROWS][RES_KC + 1];
  __shared__ __align__(16) double Xs[RES_KC][RES_NC];
  const int tid = threadIdx.x;
  const int r = tid >> 2, g = tid & 3;  // row, group of 4 columns
  const int64_t i0 = (int64_t)blockIdx.x * RES_ROWS;
  const int64_t kb = (int64_t)blockIdx.y * kslice, ke = min64(n, kb + kslice);
  for (int64_t c0 = 0; c0 < nrhs; c0 += RES_NC) {
    const int cols = (int)min64(RES_NC, nrhs - c0);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t k0 = kb; k0 < ke; k0 += RES_KC) {
      const int kr = (int)min64(RES_KC, ke - k0);
      __syncthreads();
      for (int idx = tid; idx < RES_ROWS * RES_KC; idx += RES_THREADS) {
        const int ii = idx / RES_KC, k = idx % RES_KC;
        const int64_t i = i0 + ii;
        As[ii][k] = (i < n && k < kr) ? A[i * lda + k0 + k] : 0.0;
      }
      for (int idx = tid; idx < RES_KC * RES_NC; idx += RES_THREADS) {
        const int k = idx / RES_NC, c = idx % RES_NC;
        Xs[k][c] = (k < kr && c < cols) ? X[(k0 + k) * ldx + c0 + c] : 0.0;
      }
      __syncthreads();
#pragma unroll 8
      for (int k = 0; k < RES_KC; ++k) {
        const double av = As[r][k];
        const double2 x01 = *reinterpret_cast<const double2 *>(&Xs[k][4 * g]);
        const double2 x23 = *reinterpret_cast<const double2 *>(&Xs[k][4 * g + 2]);
        acc[0] = fma(av, x01.x, acc[0]);
        acc[1] = fma(av, x01.y, acc[1]);
        acc[2] = fma(av, x23.x, acc[2]);
        acc[3] = fma(av, x23.y, acc[3]);
      }
    }
    const int64_t i = i0 + r;
    if (P) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = 4 * g + q;
        if (i < n && c < cols) P[((int64_t)blockIdx.y * n + i) * nrhs + c0 + c] = acc[q];
      }
      continue;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = 4 * g + q;
      if (i < n && c < cols) {
        const double rv = B[i * ldb + c0 + c] - acc[q];
        R[i * ldr + c0 + c] = rv;
        if (norms) {  // a non-finite value counts as +inf in every norm
          atomic_max_nonneg(&norms[c0 + c], finite_abs(rv));                          // ||r||_inf
          atomic_max_nonneg(&norms[nrhs + c0 + c], finite_abs(X[i * ldx + c0 + c]));  // ||x||_inf
          atomic_max_nonneg(&norms[2 * nrhs + c0 + c], finite_abs(B[i * ldb + c0 + c]));
        }
      }
    }
  }
}

// One warp per row; with `vec` (A 16-byte aligned, lda even) each lane reads
// 16 bytes per load with four loads in flight.
__global__ void inf_norm_rows_kernel(const double *__restrict__ A, int64_t lda, int64_t n,
                                     double *out, int vec) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (i >= n) return;
  const double *row = A + i * lda;
  double s = 0.0;
  int64_t k = 0;
  if (vec) {
    for (; k + 256 <= n; k += 256) {
      double2 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = *reinterpret_cast<const double2 *>(row + k + u * 64 + 2 * lane);
#pragma unroll
      for (int u = 0; u < 4; ++u) s += fabs(v[u].x) + fabs(v[u].y);
    }
  }
  for (k += lane; k < n; k += 32) s += fabs(row[k]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) atomic_max_nonneg(out, finite_abs(s));
}

__global__ void axpy_cols_kernel(double *X, int64_t ldx, const double *D, int64_t ldd, int64_t n,
                                 int64_t nrhs) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * nrhs) return;
  const int64_t i = idx / nrhs, c = idx % nrhs;
  X[i * ldx + c] += D[i * ldd + c];
}

// ------------------------------------------------------- backward error
// acc[0] += sum (A - P)^2, acc[1] += sum A^2 over the full square, with
// P = F F^T (Cholesky) or L U (LU compact, unit U).  32 x 32 output tiles.
template <typename Tf>
__global__ void __launch_bounds__(256)
    backward_error_kernel(int is_lu, const double *__restrict__ A, int64_t lda,
                          const Tf *__restrict__ F, int64_t ldf, int64_t n, double *acc_out) {
  __shared__ double Ls[32][33];
  __shared__ double Rs[32][33];
  __shared__ double red[2][8];
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int64_t i0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;
  double p[4] = {0, 0, 0, 0};
  const int64_t kend = min64(n, min64(i0, j0) + 32);
  for (int64_t k0 = 0; k0 < kend; k0 += 32) {
    for (int idx = tid; idx < 32 * 32; idx += 256) {
      const int r = idx / 32, k = idx % 32;
      const int64_t gi = i0 + r, gk = k0 + k, gj = j0 + r;
      double lv = 0.0, rv = 0.0;
      if (gi < n && gk < n && gk <= gi) lv = (double)F[gi * ldf + gk];
      if (!is_lu) {
        if (gj < n && gk < n && gk <= gj) rv = (double)F[gj * ldf + gk];
      } else {
        // Rs[r][k] = U_{k0+k, j0+r}
        if (gj < n && gk < n) rv = (gk == gj) ? 1.0 : (gk < gj ? (double)F[gk * ldf + gj] : 0.0);
      }
      Ls[r][k] = lv;
      Rs[r][k] = rv;
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < 32; ++k) {
      const double rv = Rs[tx][k];
#pragma unroll
      for (int a = 0; a < 4; ++a) p[a] = fma(Ls[ty + 8 * a][k], rv, p[a]);
    }
    __syncthreads();
  }
  double num = 0.0, den = 0.0;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t gi = i0 + ty + 8 * a, gj = j0 + tx;
    if (gi < n && gj < n) {
      const double av = A[gi * lda + gj];
      const double d = av - p[a];
      num += d * d;
      den += av * av;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_xor_sync(0xffffffffu, num, o);
    den += __shfl_xor_sync(0xffffffffu, den, o);
  }
  if (tx == 0) {
    red[0][ty] = num;
    red[1][ty] = den;
  }
  __syncthreads();
  if (tid == 0) {
    double a = 0, b = 0;
    for (int w = 0; w < 8; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    atomicAdd(&acc_out[0], a);
    atomicAdd(&acc_out[1], b);
  }
}

template <typename Tf>
__global__ void check_diag_kernel(const Tf *F, int64_t ldf, int64_t n, int *flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double d = (double)F[i * ldf + i];
  if (!(fabs(d) > 0.0) || !isfinite(d)) atomicOr(flag, 1);
}

}  // namespace

template <typename Tf, typename Tc>
cudaError_t launch_trsm(const Tf *F, int64_t ldf, double *B, int64_t ldb, int64_t n,
                        int64_t nrhs, int kind, int *sync, unsigned epoch, int *err,
                        int64_t spin_limit, cudaStream_t st) {
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  const int64_t nb = (n + TB - 1) / TB;
  if (nb + 1 > SYNC_WORDS) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(sync, 0, sizeof(int), st);  // ticket
  if (e != cudaSuccess) return e;
  const long long wait_ns = (long long)spin_limit * 100LL;  // spin_limit in units of 100 ns
  trsm_kernel<Tf, Tc><<<(unsigned)nb, TRSM_THREADS, 0, st>>>(F, ldf, B, ldb, n, nrhs, kind, sync,
                                                             sync + 1, epoch, err, wait_ns);
  count_launch();
  return cudaGetLastError();
}

size_t trsm_inv_bytes(int64_t n, size_t esz) {
  const int64_t bs = esz == 4 ? inv_block<float>() : inv_block<double>();
  const int64_t nb = (n + bs - 1) / bs;
  return (size_t)nb * bs * bs * esz;
}

template <typename Tf>
cudaError_t launch_diag_inv(const Tf *F, int64_t ldf, int64_t n, int kind, Tf *Dinv,
                            cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  constexpr int BS = inv_block<Tf>();
  constexpr size_t smem = 2 * sizeof(Tf) * BS * (BS + 1);
  static const cudaError_t attr = cudaFuncSetAttribute(
      diag_inv_kernel<Tf, Tf>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (attr != cudaSuccess) return attr;
  const int64_t nb = (n + BS - 1) / BS;
  diag_inv_kernel<Tf, Tf><<<(unsigned)nb, BS, smem, st>>>(F, ldf, n, kind, Dinv);
  count_launch();
  return cudaGetLastError();
}

template <typename Tf>
cudaError_t launch_coupling(const Tf *F, int64_t ldf, const Tf *Dinv, int64_t n, int kind, Tf *M,
                            cudaStream_t st) {
  const int64_t bs = inv_block<Tf>(), nb = (n + bs - 1) / bs;
  if (nb <= 1) return cudaSuccess;
  constexpr size_t smem = 2 * sizeof(Tf) * inv_block<Tf>() * (inv_block<Tf>() + 1);
  static const cudaError_t attr = cudaFuncSetAttribute(
      coupling_kernel<Tf>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (attr != cudaSuccess) return attr;
  coupling_kernel<Tf><<<(unsigned)(nb - 1), TRSM_THREADS, smem, st>>>(F, ldf, Dinv, n, kind, M);
  count_launch();
  return cudaGetLastError();
}

template <typename Tf>
cudaError_t launch_trsm_inv(const Tf *F, int64_t ldf, const Tf *Dinv, const Tf *M, double *B,
                            int64_t ldb, int64_t n, int64_t nrhs, int kind, int *sync,
                            unsigned epoch, int *err, int64_t spin_limit, cudaStream_t st,
                            int withhold) {
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  using C = TrsmCfg<Tf>;
  const int64_t nb = (n + C::BS - 1) / C::BS;
  (void)epoch;
  static const cudaError_t attr = [] {
    cudaError_t a = cudaFuncSetAttribute(trsm_inv1_kernel<Tf, Tf>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (a == cudaSuccess)
      a = cudaFuncSetAttribute(trsm_inv_kernel<Tf, Tf, 2>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (a == cudaSuccess)
      a = cudaFuncSetAttribute(trsm_inv_kernel<Tf, Tf, TRSM_MAX_GROUPS>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    return a;
  }();
  if (attr != cudaSuccess) return attr;
  const long long wait_ns = (long long)spin_limit * 100LL;
  // one launch per slab of up to TRSM_GROUPS * NRC right-hand sides, each a
  // complete sweep with fresh sync words (stream order separates the slabs)
  constexpr int64_t SLAB = (int64_t)TRSM_MAX_GROUPS * C::NRC;
  for (int64_t c0 = 0; c0 < nrhs; c0 += SLAB) {
    cudaError_t e = cudaMemsetAsync(sync, 0, 2 * sizeof(int), st);  // ticket, progress
    if (e != cudaSuccess) return e;
    const int64_t w = min64(SLAB, nrhs - c0);
    const int hold = withhold < nb ? withhold : -1;
    if (w <= C::NRC)
      trsm_inv1_kernel<Tf, Tf><<<(unsigned)nb, TRSM_THREADS, C::SMEM, st>>>(
          F, ldf, Dinv, M, B + c0, ldb, n, w, kind, sync, sync + 1, err, wait_ns, hold);
    else if (w <= 2 * C::NRC)
      trsm_inv_kernel<Tf, Tf, 2><<<(unsigned)nb, TRSM_THREADS, C::SMEM, st>>>(
          F, ldf, Dinv, M, B + c0, ldb, n, w, kind, sync, sync + 1, err, wait_ns, hold);
    else
      trsm_inv_kernel<Tf, Tf, TRSM_MAX_GROUPS><<<(unsigned)nb, TRSM_THREADS, C::SMEM, st>>>(
          F, ldf, Dinv, M, B + c0, ldb, n, w, kind, sync, sync + 1, err, wait_ns, hold);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// r = b - (P[0] + P[1] + ... ) with the slices summed in order; the norms as
// in residual_kernel.
__global__ void residual_finish_kernel(const double *__restrict__ P, int slices,
                                       const double *__restrict__ X, int64_t ldx,
                                       const double *__restrict__ B, int64_t ldb,
                                       double *__restrict__ R, int64_t ldr, int64_t n,
                                       int64_t nrhs, double *norms) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * nrhs) return;
  const int64_t i = e / nrhs, c = e % nrhs;
  double acc = P[e];
  for (int sl = 1; sl < slices; ++sl) acc += P[(int64_t)sl * n * nrhs + e];
  const double rv = B[i * ldb + c] - acc;
  R[i * ldr + c] = rv;
  if (norms) {
    atomic_max_nonneg(&norms[c], finite_abs(rv));
    atomic_max_nonneg(&norms[nrhs + c], finite_abs(X[i * ldx + c]));
    atomic_max_nonneg(&norms[2 * nrhs + c], finite_abs(B[i * ldb + c]));
  }
}

int residual_slices(int64_t n, int sm_count) {
  const int64_t blocks = ceil_div(n, RES_ROWS);
  const int64_t want = 4 * (int64_t)sm_count;  // about eight warps per SM
  if (blocks >= want || n < 4 * RES_KC) return 1;
  return (int)std::min<int64_t>(8, std::min<int64_t>(ceil_div(want, blocks), n / (2 * RES_KC)));
}

size_t residual_work_bytes(int64_t n, int64_t nrhs, int sm_count) {
  const int sl = residual_slices(n, sm_count);
  return sl > 1 ? (size_t)sl * n * nrhs * sizeof(double) : 0;
}

cudaError_t launch_residual(const double *A, int64_t lda, const double *X, int64_t ldx,
                            const double *B, int64_t ldb, double *R, int64_t ldr, int64_t n,
                            int64_t nrhs, double *norms, double *work, size_t work_bytes,
                            int sm_count, cudaStream_t st) {
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  if (norms) {
    cudaError_t e = cudaMemsetAsync(norms, 0, sizeof(double) * 3 * nrhs, st);
    if (e != cudaSuccess) return e;
  }
  int sl = residual_slices(n, sm_count);
  if (sl > 1 && (!work || work_bytes < residual_work_bytes(n, nrhs, sm_count))) sl = 1;
  if (sl == 1) {
    residual_kernel<<<(unsigned)ceil_div(n, RES_ROWS), RES_THREADS, 0, st>>>(
        A, lda, X, ldx, B, ldb, R, ldr, n, nrhs, norms, n, nullptr);
    count_launch();
    return cudaGetLastError();
  }
  // K slices: whole 64-column chunks, the last slice possibly shorter
  const int64_t kslice = ceil_div(ceil_div(n, sl), RES_KC) * RES_KC;
  sl = (int)ceil_div(n, kslice);
  residual_kernel<<<dim3((unsigned)ceil_div(n, RES_ROWS), (unsigned)sl), RES_THREADS, 0, st>>>(
      A, lda, X, ldx, B, ldb, R, ldr, n, nrhs, nullptr, kslice, work);
  count_launch();
  const int64_t total = n * nrhs;
  residual_finish_kernel<<<(unsigned)ceil_div(total, 256), 256, 0, st>>>(work, sl, X, ldx, B, ldb,
                                                                         R, ldr, n, nrhs, norms);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_inf_norm_rows(const double *A, int64_t lda, int64_t n, double *out,
                                 cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), st);
  if (e != cudaSuccess || n <= 0) return e;
  const int vec = ((reinterpret_cast<uintptr_t>(A) & 15) == 0 && (lda & 1) == 0) ? 1 : 0;
  inf_norm_rows_kernel<<<(unsigned)ceil_div(n, 8), 256, 0, st>>>(A, lda, n, out, vec);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_axpy_cols(double *X, int64_t ldx, const double *D, int64_t ldd, int64_t n,
                             int64_t nrhs, cudaStream_t st) {
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  axpy_cols_kernel<<<(unsigned)ceil_div(n * nrhs, 256), 256, 0, st>>>(X, ldx, D, ldd, n, nrhs);
  count_launch();
  return cudaGetLastError();
}

template <typename Tf>
cudaError_t launch_backward_error(int is_lu, const double *A, int64_t lda, const Tf *F,
                                  int64_t ldf, int64_t n, double *acc, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(acc, 0, 2 * sizeof(double), st);
  if (e != cudaSuccess || n <= 0) return e;
  const int64_t g = (n + 31) / 32;
  if (g > 65535) return cudaErrorInvalidConfiguration;
  backward_error_kernel<Tf><<<dim3((unsigned)g, (unsigned)g), 256, 0, st>>>(is_lu, A, lda, F, ldf,
                                                                          n, acc);
  count_launch();
  return cudaGetLastError();
}

template <typename Tf>
cudaError_t launch_check_diag(const Tf *F, int64_t ldf, int64_t n, int *flag, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), st);
  if (e != cudaSuccess || n <= 0) return e;
  check_diag_kernel<Tf><<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(F, ldf, n, flag);
  count_launch();
  return cudaGetLastError();
}

template cudaError_t launch_trsm<double, double>(const double *, int64_t, double *, int64_t,
                                                 int64_t, int64_t, int, int *, unsigned, int *,
                                                 int64_t, cudaStream_t);
template cudaError_t launch_trsm<float, float>(const float *, int64_t, double *, int64_t, int64_t,
                                               int64_t, int, int *, unsigned, int *, int64_t,
                                               cudaStream_t);
template cudaError_t launch_diag_inv<double>(const double *, int64_t, int64_t, int, double *,
                                             cudaStream_t);
template cudaError_t launch_diag_inv<float>(const float *, int64_t, int64_t, int, float *,
                                            cudaStream_t);
template cudaError_t launch_coupling<double>(const double *, int64_t, const double *, int64_t, int,
                                             double *, cudaStream_t);
template cudaError_t launch_coupling<float>(const float *, int64_t, const float *, int64_t, int,
                                            float *, cudaStream_t);
template cudaError_t launch_trsm_inv<double>(const double *, int64_t, const double *, const double *,
                                             double *, int64_t, int64_t, int64_t, int, int *,
                                             unsigned, int *, int64_t, cudaStream_t, int);
template cudaError_t launch_trsm_inv<float>(const float *, int64_t, const float *, const float *,
                                            double *, int64_t, int64_t, int64_t, int, int *, unsigned,
                                            int *, int64_t, cudaStream_t, int);
template cudaError_t launch_backward_error<double>(int, const double *, int64_t, const double *,
                                                   int64_t, int64_t, double *, cudaStream_t);
template cudaError_t launch_backward_error<float>(int, const double *, int64_t, const float *,
                                                  int64_t, int64_t, double *, cudaStream_t);
template cudaError_t launch_check_diag<double>(const double *, int64_t, int64_t, int *,
                                               cudaStream_t);
template cudaError_t launch_check_diag<float>(const float *, int64_t, int64_t, int *,
                                              cudaStream_t);

}  // namespace gb
