// Batched Algorithm 1 (arXiv:1812.02056, Sec. 2): thousands of independent
// SPD matrices of uneven orders factored in ONE persistent launch.
//
// The host sorts the matrices longest first (n^3, LPT order) and uploads a
// plan; each CTA takes the next matrix from an atomic ticket and factors it
// in place with step s:
//   * small matrices (the packed lower triangle fits in shared memory): the
//     whole of Algorithm 1 in shared memory -- column steps left-looking over
//     the columns since the checkpoint z, and every s columns the delayed
//     update A[c.., c..] -= S with S_ij formed first and then subtracted;
//   * larger matrices: the s-wide panel L[z.., z..z+sb) lives in shared
//     memory for its column steps, and the delayed update is applied to the
//     trailing lower triangle in global memory (L2-resident for n <= 1024).
// Every sum runs in ascending k, one product at a time.  With `exact` set the
// kernel uses separately rounded multiply and subtract (no FMA), so its FP64
// result is the same bits as the oracle's literal mode.
//
// Batched Algorithm 2 (pivot-free Crout LU, L lower, U unit upper, stored
// compactly) follows the same plan: the whole matrix in shared memory when
// it fits, else an L panel (rows [z, n) x the block's columns) and a U panel
// (the block's rows x columns [z, n)) in shared memory and the delayed
// update of the trailing square in place in the output.
#include <math.h>

#include <algorithm>

#include "gb_internal.cuh"

namespace gb {
namespace {

constexpr int BT = 256;  // threads per CTA

template <typename T>
__device__ __forceinline__ T msub(T acc, T a, T b, bool exact);
template <>
__device__ __forceinline__ double msub<double>(double acc, double a, double b, bool exact) {
  return exact ? __dsub_rn(acc, __dmul_rn(a, b)) : fma(-a, b, acc);
}
template <>
__device__ __forceinline__ float msub<float>(float acc, float a, float b, bool exact) {
  return exact ? __fsub_rn(acc, __fmul_rn(a, b)) : fmaf(-a, b, acc);
}
template <typename T>
__device__ __forceinline__ T madd(T acc, T a, T b, bool exact);
template <>
__device__ __forceinline__ double madd<double>(double acc, double a, double b, bool exact) {
  return exact ? __dadd_rn(acc, __dmul_rn(a, b)) : fma(a, b, acc);
}
template <>
__device__ __forceinline__ float madd<float>(float acc, float a, float b, bool exact) {
  return exact ? __fadd_rn(acc, __fmul_rn(a, b)) : fmaf(a, b, acc);
}
template <typename T>
__device__ __forceinline__ T dsqrt(T x);
template <>
__device__ __forceinline__ double dsqrt<double>(double x) {
  return __dsqrt_rn(x);
}
template <>
__device__ __forceinline__ float dsqrt<float>(float x) {
  return __fsqrt_rn(x);
}
template <typename T>
__device__ __forceinline__ T ddiv(T a, T b);
template <>
__device__ __forceinline__ double ddiv<double>(double a, double b) {
  return __ddiv_rn(a, b);
}
template <>
__device__ __forceinline__ float ddiv<float>(float a, float b) {
  return __fdiv_rn(a, b);
}

__device__ __forceinline__ int64_t tri(int64_t i) { return i * (i + 1) / 2; }

// The delayed update of an m x nc block: out(i, j) -= sum_{k < kn} X(i, k) Y(j, k),
// for every (i, j) (LOWER: j <= i).  The 256 threads form a 16 x 16 grid; in
// each (16 TR) x (16 TR) block tile a thread owns TR consecutive rows and TR
// columns 16 apart (so the 16 threads of a row group read 16 consecutive
// rows of Y: distinct banks), held as a TR x TR register tile.  A k step
// costs 2 TR shared-memory loads for TR^2 multiply-adds (a dot product per
// element would cost two loads per multiply-add).  Each element's sum still
// runs over k in ascending order from zero and is subtracted once, so exact
// mode keeps the oracle's rounding sequence.
template <typename T, bool EXACT, bool LOWER, int TR, typename FX, typename FY, typename FO>
__device__ __forceinline__ void tiled_update(int m, int nc, int kn, FX X, FY Y, FO out) {
  constexpr int TB = 16 * TR;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int nti = (m + TB - 1) / TB, ntj = (nc + TB - 1) / TB;
  for (int t = 0; t < nti * ntj; ++t) {
    const int ti = t / ntj, tj = t % ntj;
    if (LOWER && tj > ti) continue;  // block tile strictly above the diagonal (TB square tiles)
    const int i0 = ti * TB + ty * TR, j0 = tj * TB + tx;
    if (i0 >= m || j0 >= nc) continue;
    if (LOWER && j0 > i0 + TR - 1) continue;  // every element of this thread above the diagonal
    int ii[TR], jj[TR];
#pragma unroll
    for (int a = 0; a < TR; ++a) {
      ii[a] = min(i0 + a, m - 1);
      jj[a] = min(j0 + 16 * a, nc - 1);
    }
    // the outputs are read before the products (global memory on the panel
    // path: the load latency overlaps the k loop); nothing else writes them
    T acc[TR][TR], cv[TR][TR];
#pragma unroll
    for (int a = 0; a < TR; ++a)
#pragma unroll
      for (int b = 0; b < TR; ++b) {
        acc[a][b] = T(0);
        const int i = i0 + a, j = j0 + 16 * b;
        cv[a][b] = (i < m && j < nc && (!LOWER || j <= i)) ? *out(i, j) : T(0);
      }
#pragma unroll 4
    for (int k = 0; k < kn; ++k) {
      T xa[TR], yb[TR];
#pragma unroll
      for (int a = 0; a < TR; ++a) {
        xa[a] = X(ii[a], k);
        yb[a] = Y(jj[a], k);
      }
#pragma unroll
      for (int a = 0; a < TR; ++a)
#pragma unroll
        for (int b = 0; b < TR; ++b) acc[a][b] = madd(acc[a][b], xa[a], yb[b], EXACT);
    }
#pragma unroll
    for (int a = 0; a < TR; ++a)
#pragma unroll
      for (int b = 0; b < TR; ++b) {
        const int i = i0 + a, j = j0 + 16 * b;
        if (i < m && j < nc && (!LOWER || j <= i))
          *out(i, j) = cv[a][b] - acc[a][b];  // a lone subtraction is never contracted
      }
  }
}

// One dot product per element (warp w takes rows w, w + 8, ...; its lanes the
// columns): no multiply-add is spent above the diagonal.  FP64 uses it: its
// rate is bound by the FP64 units, not by shared-memory loads.
template <typename T, bool EXACT, bool LOWER, typename FX, typename FY, typename FO>
__device__ __forceinline__ void dot_update(int m, int nc, int kn, FX X, FY Y, FO out) {
  const int tid = threadIdx.x;
  for (int i = tid >> 5; i < m; i += BT / 32) {
    const int jend = LOWER ? min(i + 1, nc) : nc;
    for (int j = tid & 31; j < jend; j += 32) {
      T *p = out(i, j);
      const T cij = *p;  // read before the products: its latency overlaps them
      T sij = T(0);
#pragma unroll 4
      for (int k = 0; k < kn; ++k) sij = madd(sij, X(i, k), Y(j, k), EXACT);
      *p = cij - sij;  // a lone subtraction is never contracted
    }
  }
}

template <typename T, bool EXACT, bool LOWER, typename FX, typename FY, typename FO>
__device__ __forceinline__ void block_update(int m, int nc, int kn, FX X, FY Y, FO out) {
  if (sizeof(T) == 8)
    dot_update<T, EXACT, LOWER>(m, nc, kn, X, Y, out);
  else if (m >= 48 && nc >= 48)
    tiled_update<T, EXACT, LOWER, 4>(m, nc, kn, X, Y, out);
  else
    tiled_update<T, EXACT, LOWER, 2>(m, nc, kn, X, Y, out);
}

// ------------------------------------------------- column steps of one s-block
// Columns [0, sb) of rows [0, R) (R >= sb) of the block since the checkpoint,
// row r's entries at row(r)[0 .. sb): Algorithm 1's column steps, in chunks
// of CCH columns.  Per chunk:
//   (a) warp 0, lane l holding row c0 + l of the chunk: the products of the
//       block's finished columns k < c0 (k ascending), then
//   (b) the chunk's cw x cw diagonal part column by column, the pivot and
//       each column's entries passed between lanes by shuffles;
//   (c) every row below the chunk subtracts the finished columns' products
//       and then the chunk's columns one at a time, dividing by L_cc.
// Two barriers per chunk instead of two per column.  Each entry still
// receives its products in ascending k, one at a time, and one division by
// its pivot -- the same operations in the same order as column by column, so
// exact mode keeps the oracle's rounding sequence.  Returns 0, or the local
// column + 1 of a pivot that is not positive (or NaN).
constexpr int CCH = 16;

template <typename T, bool EXACT, typename ROW>
__device__ int chol_block_columns(int R, int sb, ROW row, int *s_bad) {
  const int tid = threadIdx.x, lane = tid & 31;
  for (int c0 = 0; c0 < sb; c0 += CCH) {
    const int cw = min(CCH, sb - c0);
    if (tid < 32) {  // (a) and (b): lane l < cw holds row c0 + l
      const bool act = lane < cw;
      T *Lr = row(c0 + (act ? lane : 0));
      T va[CCH];
#pragma unroll
      for (int j = 0; j < CCH; ++j) va[j] = (act && j <= lane) ? Lr[c0 + j] : T(0);
      if (act) {
        for (int k = 0; k < c0; ++k) {
          const T a = Lr[k];
#pragma unroll
          for (int j = 0; j < CCH; ++j)
            if (j <= lane) va[j] = msub(va[j], a, row(c0 + j)[k], EXACT);
        }
      }
      int bad = 0;
#pragma unroll
      for (int cc = 0; cc < CCH; ++cc) {
        if (cc < cw && !bad) {
          const T d = __shfl_sync(0xffffffffu, va[cc], cc);
          if (!(d > T(0))) {  // uniform over the warp
            bad = c0 + cc + 1;
          } else {
            const T lcc = dsqrt(d);
            if (lane == cc) va[cc] = lcc;
            else if (lane > cc) va[cc] = ddiv(va[cc], lcc);
#pragma unroll
            for (int cc2 = cc + 1; cc2 < CCH; ++cc2) {
              const T l = __shfl_sync(0xffffffffu, va[cc], cc2);  // L_{c0+cc2, c0+cc}
              if (lane >= cc2) va[cc2] = msub(va[cc2], va[cc], l, EXACT);
            }
          }
        }
      }
      if (lane < cw) {
#pragma unroll
        for (int j = 0; j < CCH; ++j)
          if (j <= lane) Lr[c0 + j] = va[j];
      }
      if (lane == 0) *s_bad = bad;
    }
    __syncthreads();
    const int bad = *s_bad;
    if (bad) return bad;  // uniform
    for (int r = c0 + cw + tid; r < R; r += BT) {  // (c)
      T *Lr = row(r);
      T v[CCH];
#pragma unroll
      for (int j = 0; j < CCH; ++j) v[j] = j < cw ? Lr[c0 + j] : T(0);
      for (int k = 0; k < c0; ++k) {
        const T a = Lr[k];
#pragma unroll
        for (int j = 0; j < CCH; ++j)
          if (j < cw) v[j] = msub(v[j], a, row(c0 + j)[k], EXACT);
      }
#pragma unroll
      for (int cc = 0; cc < CCH; ++cc) {
        if (cc < cw) {
          const T *Lc = row(c0 + cc);
          v[cc] = ddiv(v[cc], Lc[c0 + cc]);
#pragma unroll
          for (int cc2 = cc + 1; cc2 < CCH; ++cc2)
            if (cc2 < cw) v[cc2] = msub(v[cc2], v[cc], row(c0 + cc2)[c0 + cc], EXACT);
        }
      }
#pragma unroll
      for (int j = 0; j < CCH; ++j)
        if (j < cw) Lr[c0 + j] = v[j];
    }
    __syncthreads();
  }
  return 0;
}

// ------------------------------------------------- whole matrix in shared memory
// S holds the packed lower triangle: (i, j), j <= i, at i (i + 1) / 2 + j.
template <typename T, bool EXACT>
__device__ int chol_in_smem(T *S, int n, int s, int *s_bad) {
  for (int z = 0; z < n; z += s) {
    if (z > 0) {
      // delayed update of the previous block [z - s, z): A[i][j] -= S_ij,
      // S_ij = sum_{k=z-s}^{z-1} L_ik L_jk, z <= j <= i
      const int z0 = z - s, c0 = z;
      block_update<T, EXACT, true>(
          n - c0, n - c0, s, [&](int i, int k) { return S[tri(c0 + i) + z0 + k]; },
          [&](int j, int k) { return S[tri(c0 + j) + z0 + k]; },
          [&](int i, int j) { return &S[tri(c0 + i) + c0 + j]; });
      __syncthreads();
    }
    const int sb = min(s, n - z);
    const int bad = chol_block_columns<T, EXACT>(
        n - z, sb, [&](int r) { return S + tri(z + r) + z; }, s_bad);
    if (bad) return z + bad;
  }
  return 0;
}

// ------------------------------------------------- panel in shared memory
// P: rows [z, n) x columns [z, z + sb) of the working matrix, row-major with
// leading dimension ldp >= s (odd when it fits: rows then fall in different
// shared-memory banks).  Once the trailing matrix's lower triangle fits in
// the `smem_elems` elements of P's buffer, it moves there and the rest of
// the factorization runs as the whole-matrix path (same steps, same order).
template <typename T, bool EXACT>
__device__ int chol_panel_path(T *A, int64_t lda, int n, int s, T *P, int ldp, int *s_bad,
                               int64_t smem_elems) {
  const int tid = threadIdx.x;
  for (int z = 0; z < n; z += s) {
    if (z > 0 && tri(n - z) <= smem_elems) {
      const int m = n - z;
      T *S = P;
      for (int r = tid >> 5; r < m; r += BT / 32)
        for (int q = tid & 31; q <= r; q += 32) S[tri(r) + q] = A[(int64_t)(z + r) * lda + z + q];
      __syncthreads();
      const int bad = chol_in_smem<T, EXACT>(S, m, s, s_bad);
      __syncthreads();
      for (int r = tid >> 5; r < m; r += BT / 32)
        for (int q = tid & 31; q <= r; q += 32) A[(int64_t)(z + r) * lda + z + q] = S[tri(r) + q];
      __syncthreads();
      return bad ? z + bad : 0;
    }
    const int sb = min(s, n - z);
    const int rows = n - z;
    for (int r = tid >> 5; r < rows; r += BT / 32)
      for (int q = tid & 31; q < sb; q += 32) P[(int64_t)r * ldp + q] = A[(int64_t)(z + r) * lda + z + q];
    __syncthreads();
    const int bad = chol_block_columns<T, EXACT>(
        rows, sb, [&](int r) { return P + (int64_t)r * ldp; }, s_bad);
    if (bad) return z + bad;
    for (int r = tid >> 5; r < rows; r += BT / 32)
      for (int q = tid & 31; q < sb; q += 32)
        if (q <= r) A[(int64_t)(z + r) * lda + z + q] = P[(int64_t)r * ldp + q];
    // delayed update of the trailing lower triangle: rows/cols [z+sb, n)
    const int m = n - z - sb;
    const int64_t base = (int64_t)(z + sb) * lda + z + sb;
    block_update<T, EXACT, true>(
        m, m, sb, [&](int r, int k) { return P[(int64_t)(sb + r) * ldp + k]; },
        [&](int q, int k) { return P[(int64_t)(sb + q) * ldp + k]; },
        [&](int r, int q) { return A + base + (int64_t)r * lda + q; });
    __syncthreads();  // global writes of this CTA are visible to it after the barrier
  }
  return 0;
}


// ------------------------------------------------- Algorithm 2, whole matrix in shared memory
// W: n x n working matrix, leading dimension ld.  L_ic (i >= c) overwrites
// W[i][c], U_ci (i > c) overwrites W[c][i]; U's unit diagonal is implied.
template <typename T, bool EXACT>
__device__ int lu_in_smem(T *W, int n, int ld, int s) {
  constexpr bool exact = EXACT;
  const int tid = threadIdx.x;
  int z = 0;
  for (int c = 0; c < n; ++c) {
    if (c == z + s) {
      // delayed update of the trailing square: W_ij -= S_ij, S_ij = sum_k L_ik U_kj
      const int z0 = z, c0 = c;
      block_update<T, EXACT, false>(
          n - c, n - c, c - z, [&](int i, int k) { return W[(int64_t)(c0 + i) * ld + z0 + k]; },
          [&](int j, int k) { return W[(int64_t)(z0 + k) * ld + c0 + j]; },
          [&](int i, int j) { return &W[(int64_t)(c0 + i) * ld + c0 + j]; });
      z = c;
      __syncthreads();
    }
    // column c of L (rows i >= c) and the numerators of row c of U (j > c)
    const int m = n - c;
    for (int t = tid; t < 2 * m - 1; t += BT) {
      if (t < m) {
        const int i = c + t;
        const T *Li = W + (int64_t)i * ld;
        T v = Li[c];
#pragma unroll 4
        for (int k = z; k < c; ++k) v = msub(v, Li[k], W[(int64_t)k * ld + c], exact);
        W[(int64_t)i * ld + c] = v;
      } else {
        const int j = c + 1 + (t - m);
        const T *Lc = W + (int64_t)c * ld;
        T u = Lc[j];
#pragma unroll 4
        for (int k = z; k < c; ++k) u = msub(u, Lc[k], W[(int64_t)k * ld + j], exact);
        W[(int64_t)c * ld + j] = u;
      }
    }
    __syncthreads();
    const T lcc = W[(int64_t)c * ld + c];
    if (lcc == T(0) || lcc != lcc) return c + 1;  // uniform: every thread read the same lcc
    for (int j = c + 1 + tid; j < n; j += BT) W[(int64_t)c * ld + j] = ddiv(W[(int64_t)c * ld + j], lcc);
    __syncthreads();
  }
  return 0;
}

// ------------------------------------------------- Algorithm 2, panels in shared memory
// A: the n x n working matrix in global memory (the output), in place.
// PL: rows [z, n) x columns [z, z + sb), leading dimension s (L panel);
// PU: rows [z, z + sb) x columns [z, n), leading dimension n (U panel).
// Inside the diagonal block, L is read from PL (on and below the diagonal)
// and U from PU (above it).
template <typename T, bool EXACT>
__device__ int lu_panel_path(T *A, int64_t lda, int n, int s, T *PL, int ldp, T *PU) {
  constexpr bool exact = EXACT;
  const int tid = threadIdx.x;
  for (int z = 0; z < n; z += s) {
    const int sb = min(s, n - z);
    const int rows = n - z;
    for (int r = tid >> 5; r < rows; r += BT / 32)
      for (int q = tid & 31; q < sb; q += 32) PL[(int64_t)r * ldp + q] = A[(int64_t)(z + r) * lda + z + q];
    for (int r = tid >> 5; r < sb; r += BT / 32)
      for (int q = tid & 31; q < rows; q += 32) PU[(int64_t)r * n + q] = A[(int64_t)(z + r) * lda + z + q];
    __syncthreads();
    for (int c = 0; c < sb; ++c) {  // column z + c, local index c
      const int m = rows - c;
      for (int t = tid; t < 2 * m - 1; t += BT) {
        if (t < m) {
          const int r = c + t;
          T *Pr = PL + (int64_t)r * ldp;
          T v = Pr[c];
#pragma unroll 4
          for (int k = 0; k < c; ++k) v = msub(v, Pr[k], PU[(int64_t)k * n + c], exact);
          Pr[c] = v;
        } else {
          const int q = c + 1 + (t - m);
          const T *Pc = PL + (int64_t)c * ldp;
          T u = PU[(int64_t)c * n + q];
#pragma unroll 4
          for (int k = 0; k < c; ++k) u = msub(u, Pc[k], PU[(int64_t)k * n + q], exact);
          PU[(int64_t)c * n + q] = u;
        }
      }
      __syncthreads();
      const T lcc = PL[(int64_t)c * ldp + c];
      if (lcc == T(0) || lcc != lcc) return z + c + 1;
      for (int q = c + 1 + tid; q < rows; q += BT) PU[(int64_t)c * n + q] = ddiv(PU[(int64_t)c * n + q], lcc);
      __syncthreads();
    }
    for (int r = tid >> 5; r < rows; r += BT / 32)
      for (int q = tid & 31; q < sb; q += 32)
        if (q <= r) A[(int64_t)(z + r) * lda + z + q] = PL[(int64_t)r * ldp + q];
    for (int r = tid >> 5; r < sb; r += BT / 32)
      for (int q = r + 1 + (tid & 31); q < rows; q += 32) A[(int64_t)(z + r) * lda + z + q] = PU[(int64_t)r * n + q];
    // delayed update of the trailing square: rows/cols [z+sb, n)
    const int mt = n - z - sb;
    const int64_t base = (int64_t)(z + sb) * lda + z + sb;
    block_update<T, EXACT, false>(
        mt, mt, sb, [&](int r, int k) { return PL[(int64_t)(sb + r) * ldp + k]; },
        [&](int q, int k) { return PU[(int64_t)k * n + sb + q]; },
        [&](int r, int q) { return A + base + (int64_t)r * lda + q; });
    __syncthreads();
  }
  return 0;
}

struct Plan {
  int count;
  const int *order;
  const int *n;
  const int *step;
  void *const *A;       // inputs (lower triangle read)
  const int64_t *lda;
  void *const *L;       // outputs (may alias the inputs)
  const int64_t *ldl;
  int *info;
  int *ticket;
};

template <typename T, bool EXACT>
__global__ void __launch_bounds__(BT, 2) batched_chol_kernel(Plan plan, int64_t smem_elems) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *buf = reinterpret_cast<T *>(smem_raw);
  __shared__ int s_bad;
  __shared__ int s_idx;
  for (;;) {
    if (threadIdx.x == 0) {
      const int t = atomicAdd(plan.ticket, 1);
      s_idx = t < plan.count ? plan.order[t] : -1;
    }
    __syncthreads();
    const int idx = s_idx;
    if (idx < 0) break;
    const int n = plan.n[idx];
    const int s = max(1, plan.step[idx]);
    const T *A = reinterpret_cast<const T *>(plan.A[idx]);
    const int64_t lda = plan.lda[idx];
    T *L = reinterpret_cast<T *>(plan.L[idx]);
    const int64_t ldl = plan.ldl[idx];
    int info = 0;
    if (n > 0) {
      if (tri(n) <= smem_elems) {
        for (int r = threadIdx.x >> 5; r < n; r += BT / 32)
          for (int q = threadIdx.x & 31; q <= r; q += 32) buf[tri(r) + q] = A[(int64_t)r * lda + q];
        __syncthreads();
        info = chol_in_smem<T, EXACT>(buf, n, min(s, n), &s_bad);
        __syncthreads();
        for (int r = threadIdx.x >> 5; r < n; r += BT / 32)
          for (int q = threadIdx.x & 31; q < n; q += 32)
            L[(int64_t)r * ldl + q] = q <= r ? buf[tri(r) + q] : T(0);
      } else {
        // the panel path works in place in L: copy A's lower triangle first
        for (int r = threadIdx.x >> 5; r < n; r += BT / 32)
          for (int q = threadIdx.x & 31; q < n; q += 32)
            L[(int64_t)r * ldl + q] = q <= r ? A[(int64_t)r * lda + q] : T(0);
        __syncthreads();
        const int sp = max(1, (int)min64(s, smem_elems / n));  // panel width that fits
        const int ldp = (int64_t)n * (sp | 1) <= smem_elems ? (sp | 1) : sp;
        info = chol_panel_path<T, EXACT>(L, ldl, n, sp, buf, ldp, &s_bad, smem_elems);
        __syncthreads();
      }
    }
    if (threadIdx.x == 0) plan.info[idx] = info;
    __syncthreads();  // s_idx is rewritten next iteration
  }
}


// Leading dimension of a matrix held whole in shared memory: odd, so that
// threads walking down a column hit different banks.
__device__ __host__ inline int64_t lu_smem_ld(int n) { return (n & 1) ? n : n + 1; }

template <typename T, bool EXACT>
__global__ void __launch_bounds__(BT, 2) batched_lu_kernel(Plan plan, int64_t smem_elems) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *buf = reinterpret_cast<T *>(smem_raw);
  __shared__ int s_idx;
  for (;;) {
    if (threadIdx.x == 0) {
      const int t = atomicAdd(plan.ticket, 1);
      s_idx = t < plan.count ? plan.order[t] : -1;
    }
    __syncthreads();
    const int idx = s_idx;
    if (idx < 0) break;
    const int n = plan.n[idx];
    const int s = max(1, plan.step[idx]);
    const T *A = reinterpret_cast<const T *>(plan.A[idx]);
    const int64_t lda = plan.lda[idx];
    T *LU = reinterpret_cast<T *>(plan.L[idx]);
    const int64_t ldo = plan.ldl[idx];
    int info = 0;
    if (n > 0) {
      const int64_t ld = lu_smem_ld(n);
      if ((int64_t)n * ld <= smem_elems) {
        for (int r = threadIdx.x >> 5; r < n; r += BT / 32)
          for (int q = threadIdx.x & 31; q < n; q += 32) buf[r * ld + q] = A[(int64_t)r * lda + q];
        __syncthreads();
        info = lu_in_smem<T, EXACT>(buf, n, (int)ld, min(s, n));
        __syncthreads();
        for (int r = threadIdx.x >> 5; r < n; r += BT / 32)
          for (int q = threadIdx.x & 31; q < n; q += 32) LU[(int64_t)r * ldo + q] = buf[r * ld + q];
      } else {
        // the panel path works in place in the output: copy A first
        if (LU != A)
          for (int r = threadIdx.x >> 5; r < n; r += BT / 32)
            for (int q = threadIdx.x & 31; q < n; q += 32) LU[(int64_t)r * ldo + q] = A[(int64_t)r * lda + q];
        __syncthreads();
        const int sp = max(1, (int)min64(s, smem_elems / (2 * (int64_t)n)));  // both panels fit
        const int ldp = (int64_t)n * ((sp | 1) + sp) <= smem_elems ? (sp | 1) : sp;
        T *PL = buf;
        T *PU = buf + (int64_t)n * ldp;
        info = lu_panel_path<T, EXACT>(LU, ldo, n, sp, PL, ldp, PU);
        __syncthreads();
      }
    }
    if (threadIdx.x == 0) plan.info[idx] = info;
    __syncthreads();  // s_idx is rewritten next iteration
  }
}

// A = n I + ones: symmetric positive definite, exact in every precision.
template <typename T>
__global__ void fill_spd_kernel(T *base, int64_t stride, int count, int n) {
  const int64_t total = (int64_t)count * n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = e / ((int64_t)n * n), r = (e / n) % n, q = e % n;
    base[m * stride + r * n + q] = (r == q) ? (T)(n + 1) : T(1);
  }
}

}  // namespace

template <typename T>
cudaError_t launch_fill_spd(T *base, int64_t stride, int count, int n, cudaStream_t st) {
  fill_spd_kernel<T><<<1024, 256, 0, st>>>(base, stride, count, n);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t launch_fill_spd<double>(double *, int64_t, int, int, cudaStream_t);
template cudaError_t launch_fill_spd<float>(float *, int64_t, int, int, cudaStream_t);

size_t batched_smem_bytes() { return 110 * 1024; }  // two CTAs per SM

template <typename T>
cudaError_t launch_chol_batched_plan(int count, const int *order, const int *n, const int *step,
                                     void *const *A, const int64_t *lda, void *const *L,
                                     const int64_t *ldl, int *info, int *ticket, int sm_count,
                                     int exact, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const size_t smem = batched_smem_bytes();
  static cudaError_t attr0 = cudaFuncSetAttribute(
      batched_chol_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  static cudaError_t attr1 = cudaFuncSetAttribute(
      batched_chol_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (attr0 != cudaSuccess) return attr0;
  if (attr1 != cudaSuccess) return attr1;
  cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  Plan p{count, order, n, step, A, lda, L, ldl, info, ticket};
  const int grid = std::min(count, 2 * sm_count);
  if (exact)
    batched_chol_kernel<T, true><<<grid, BT, smem, st>>>(p, (int64_t)(smem / sizeof(T)));
  else
    batched_chol_kernel<T, false><<<grid, BT, smem, st>>>(p, (int64_t)(smem / sizeof(T)));
  count_launch();
  return cudaGetLastError();
}

template cudaError_t launch_chol_batched_plan<double>(int, const int *, const int *, const int *,
                                                      void *const *, const int64_t *, void *const *,
                                                      const int64_t *, int *, int *, int, int,
                                                      cudaStream_t);
template cudaError_t launch_chol_batched_plan<float>(int, const int *, const int *, const int *,
                                                     void *const *, const int64_t *, void *const *,
                                                     const int64_t *, int *, int *, int, int,
                                                     cudaStream_t);

template <typename T>
cudaError_t launch_lu_batched_plan(int count, const int *order, const int *n, const int *step,
                                   void *const *A, const int64_t *lda, void *const *LU,
                                   const int64_t *ldlu, int *info, int *ticket, int sm_count,
                                   int exact, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const size_t smem = batched_smem_bytes();
  static cudaError_t attr0 = cudaFuncSetAttribute(
      batched_lu_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  static cudaError_t attr1 = cudaFuncSetAttribute(
      batched_lu_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (attr0 != cudaSuccess) return attr0;
  if (attr1 != cudaSuccess) return attr1;
  cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  Plan p{count, order, n, step, A, lda, LU, ldlu, info, ticket};
  const int grid = std::min(count, 2 * sm_count);
  if (exact)
    batched_lu_kernel<T, true><<<grid, BT, smem, st>>>(p, (int64_t)(smem / sizeof(T)));
  else
    batched_lu_kernel<T, false><<<grid, BT, smem, st>>>(p, (int64_t)(smem / sizeof(T)));
  count_launch();
  return cudaGetLastError();
}

template cudaError_t launch_lu_batched_plan<double>(int, const int *, const int *, const int *,
                                                    void *const *, const int64_t *, void *const *,
                                                    const int64_t *, int *, int *, int, int,
                                                    cudaStream_t);
template cudaError_t launch_lu_batched_plan<float>(int, const int *, const int *, const int *,
                                                   void *const *, const int64_t *, void *const *,
                                                   const int64_t *, int *, int *, int, int,
                                                   cudaStream_t);

}  // namespace gb
