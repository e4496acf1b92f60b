// Column steps of Algorithms 1 and 2 (arXiv:1812.02056, Sec. 2) for one
// block of at most 64 columns [j0, j0+bw) of the working matrix W.
//
// Every entry that the paper's column step produces,
//   Cholesky  L_cc = sqrt(A_cc - sum_{k=z}^{c-1} L_ck^2)
//             L_ic = (A_ic - sum_{k=z}^{c-1} L_ik L_ck) / L_cc      (i > c)
//   LU        L_ic = A_ic - sum_{k=z}^{c-1} L_ik U_kc               (i >= c)
//             U_ci = (A_ci - sum_{k=z}^{c-1} L_ck U_ki) / L_cc      (i > c)
// is formed here with its sum taken in ascending k, one product at a time, as
// the paper writes it.  The work is split by dependence, not reordered:
//   the bw x bw diagonal block, whose columns depend on one another (one
//     CTA, shared memory, bw dependent steps): chol_panel_kernel's first
//     part (every CTA for FP32 data; one PANEL_DIAG launch for FP64),
//     lu_diag_kernel;
//   the rows below the block: each row is an independent forward
//     substitution against the finished diagonal block (chol_panel_kernel's
//     second part, lu_rows_kernel);
//   lu_cols_kernel: columns of U right of the block, likewise independent.
// W already holds A minus every delayed update applied before this block.
#include <math.h>

#include <algorithm>

#include "gb_internal.cuh"

namespace gb {
namespace {

__device__ __forceinline__ int load_status(const int *status) {
  return *reinterpret_cast<const volatile int *>(status);
}

// Global -> shared copy of one element (4 or 8 bytes) that completes
// asynchronously (zero-filled when `valid` is false); waited for with
// cp_async_wait_all by the same thread.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T *dst, const T *src, bool valid) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "element size");
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(d), "l"(src),
               "n"((int)sizeof(T)), "r"(valid ? (int)sizeof(T) : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

constexpr int DIAG_THREADS = 256;  // 16 x 16 threads, 4 x 4 elements each

constexpr int ROWS_PER_CTA = 64;  // one row per thread; small CTAs spread rows over all SMs

// ------------------------------------------------ fused column-step kernel
// One launch per inner block: every CTA factors the bw x bw diagonal block
// itself and then solves its rows below the block against it.  Work is cut
// into 16-column chunks: the products of the columns already finished are
// subtracted by short runtime loops (small loop bodies, reused across
// iterations), then the chunk's own columns are finished one at a time.
// Every entry still receives its products in ascending k, one at a time.
// One barrier per column: at the start of a chunk each diagonal entry's
// running value is published, and every thread keeps its own copy of the
// chunk's diagonal, updated with the same products (L_jc * L_jc, in the same
// order) as the row that owns it, so that each thread forms the pivot
// itself; a breakdown is seen by every thread at once.
// The rows below the block are fetched into shared memory with asynchronous
// copies issued before the diagonal block is factored.
// The factored block is written back by the last CTA to have loaded it:
// each CTA bumps an arrival counter after loading; the CTA that arrives as
// number grid - 1 knows every other CTA already holds its own copy, writes
// the block, and resets the counter to zero for the next launch (ordered
// after this one on the stream).  No CTA waits.
// Inside the diagonal block the column below L_cc is scaled by 1 / L_cc
// (one reciprocal per column, as LAPACK's unblocked Cholesky does); the rows
// below the block divide by L_cc as the paper writes.
// The pivot's square root and reciprocal are IEEE round-to-nearest
// operations in T.  For FP32 data they give the same bits as the FP64
// operations rounded to FP32: double rounding is innocuous for the square
// root and for division when the wider format carries at least 2p + 2
// significand bits (53 >= 2 * 24 + 2; S. A. Figueroa, "When is double
// rounding innocuous?", 1995), so the mixed dtypes' FP64 pivots cost no FP64
// instruction.  MODE: PANEL_FUSED, PANEL_DIAG (one CTA: factor and write the
// block), PANEL_ROWS_ONLY (read the finished block, then the rows).
enum { PANEL_FUSED = 0, PANEL_DIAG = 1, PANEL_ROWS_ONLY = 2 };
constexpr int PB = 64;   // inner block width bound
constexpr int CH = 16;   // chunk width

// 16 consecutive elements of a 16-byte aligned shared-memory row.
__device__ __forceinline__ void load_row16(float (&o)[16], const float *p) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float4 w = reinterpret_cast<const float4 *>(p)[q];
    o[4 * q] = w.x;
    o[4 * q + 1] = w.y;
    o[4 * q + 2] = w.z;
    o[4 * q + 3] = w.w;
  }
}
__device__ __forceinline__ void load_row16(double (&o)[16], const double *p) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const double2 w = reinterpret_cast<const double2 *>(p)[q];
    o[2 * q] = w.x;
    o[2 * q + 1] = w.y;
  }
}

template <typename T>
struct PanelSmem {
  static constexpr int PADT = PB + 16 / (int)sizeof(T);  // 16-byte aligned rows
  static constexpr size_t bytes(int rows) {
    return sizeof(T) * ((size_t)PB * (PB + 1) + (size_t)PB * PADT + (size_t)PB * rows);
  }
};

template <typename T, int MODE, int ROWS>
__global__ void __launch_bounds__(ROWS)
    chol_panel_kernel(T *__restrict__ W, int64_t ld, int64_t j0, int bw, int64_t row0,
                      int64_t nrows, int *status, unsigned long long *arrivals) {
  constexpr int PADT = PanelSmem<T>::PADT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T(*Ld)[PB + 1] = reinterpret_cast<T(*)[PB + 1]>(smem_raw);  // Ld[i][k] = L_ik, k <= i
  T(*LdT)[PADT] = reinterpret_cast<T(*)[PADT]>(smem_raw + sizeof(T) * PB * (PB + 1));  // LdT[k][i] = L_ik
  T(*Ys)[ROWS] = reinterpret_cast<T(*)[ROWS]>(smem_raw + sizeof(T) * (PB * (PB + 1) + PB * PADT));
  __shared__ int s_last, s_bad;
  __shared__ T s_piv;
  if (load_status(status) != 0) return;
  const int tid = threadIdx.x;
  T *D = W + j0 * ld + j0;

  // this thread's row below the block, copied into its column of Ys while
  // the diagonal block is factored
  const int64_t r = row0 + (int64_t)blockIdx.x * ROWS + tid;
  const bool has_row = MODE != PANEL_DIAG && r < row0 + nrows;
  T *row = has_row ? W + r * ld + j0 : D;  // D: a valid address for the zero-filled copies
  if (MODE != PANEL_DIAG) {
#pragma unroll 16
    for (int u = 0; u < PB; ++u) cp_async_elem<T>(&Ys[u][tid], row + (u < bw ? u : 0), has_row && u < bw);
  }

  // all loads of the block in flight at once: registers first, then shared memory
  constexpr int PER = PB * PB / ROWS;
  T blk[PER];
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int idx = tid + u * ROWS, i = idx / PB, k = idx % PB;
    blk[u] = (i < bw && k <= i) ? D[(int64_t)i * ld + k] : T(0);
  }
  if (MODE == PANEL_ROWS_ONLY) {
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int idx = tid + u * ROWS, i = idx / PB, k = idx % PB;
      LdT[k][i] = blk[u];
    }
    __syncthreads();
  } else {
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int idx = tid + u * ROWS, i = idx / PB, k = idx % PB;
      Ld[i][k] = blk[u];
      LdT[k][i] = T(0);
    }
    __syncthreads();
    if (tid == 0) s_bad = 0;
    if (MODE == PANEL_DIAG) {
      if (tid == 0) s_last = 1;
    } else if (tid == ROWS - 1) {  // the last warp: warp 0 starts the block at once
      __threadfence();
      const unsigned long long a = atomicAdd(arrivals, 1ULL);
      s_last = (a == (unsigned long long)gridDim.x - 1) ? 1 : 0;
      if (s_last) atomicExch(arrivals, 0ULL);  // every CTA has arrived
    }
    if constexpr (sizeof(T) == 8) {
      // FP64 data: GB300 issues FP64 arithmetic at a small fraction of the
      // FP32 rate per scheduler, so the block's column updates stay spread
      // over the rows' threads (two warps): thread i < bw holds row i's
      // chunk columns; per column, the owner of the diagonal forms the pivot
      // and one barrier publishes it, a second the scaled column.
      for (int c0 = 0; c0 < bw; c0 += CH) {
        const bool mine = tid >= c0 && tid < bw;
        const int cw = min(CH, bw - c0);
        T v[CH];
#pragma unroll
        for (int j = 0; j < CH; ++j) v[j] = (mine && j < cw && c0 + j <= tid) ? Ld[tid][c0 + j] : T(0);
        if (mine) {  // products of the finished columns k < c0
          for (int k = 0; k < c0; ++k) {
            const T lik = Ld[tid][k];
#pragma unroll
            for (int j = 0; j < CH; ++j) v[j] = v[j] - lik * LdT[k][c0 + j];
          }
        }
#pragma unroll
        for (int cc = 0; cc < CH; ++cc) {  // the chunk's columns, one at a time
          if (cc < cw) {
            const int c = c0 + cc;
            if (tid == c) {
              const T d = v[cc];
              s_bad = (d > T(0)) ? 0 : c + 1;  // not positive, or NaN: breakdown
              const T piv = sqrt(d);
              s_piv = T(1) / piv;  // the column is scaled by 1 / L_cc
              v[cc] = piv;
              LdT[c][c] = piv;
            }
            __syncthreads();
            if (s_bad) {  // uniform
              if (blockIdx.x == 0 && tid == 0) atomicCAS(status, 0, (int)(j0 + s_bad));
              if (MODE != PANEL_DIAG) cp_async_wait_all();
              return;
            }
            if (tid > c && tid < bw) {
              v[cc] = v[cc] * s_piv;
              LdT[c][tid] = v[cc];
            }
            __syncthreads();
            if (tid > c && tid < bw) {
              const T lic = v[cc];
#pragma unroll
              for (int cc2 = cc + 1; cc2 < CH; ++cc2)
                if (c0 + cc2 <= tid) v[cc2] = v[cc2] - lic * LdT[c][c0 + cc2];
            }
          }
        }
        if (mine) {
#pragma unroll
          for (int j = 0; j < CH; ++j)
            if (j < cw && c0 + j <= tid) Ld[tid][c0 + j] = v[j];
        }
        __syncthreads();
      }
    } else {
      // Per 16-column chunk: every row i in [c0, bw) first receives the
      // products of the finished columns k < c0 (thread i, its row in
      // registers); then warp 0 finishes the chunk's columns one at a time,
      // lane l holding rows c0 + l and c0 + 32 + l, with the pivot and the
      // column's entries passed between lanes by shuffles (no barrier inside
      // the chunk).
      const int lane = tid & 31;
      for (int c0 = 0; c0 < bw; c0 += CH) {
        const int cw = min(CH, bw - c0);
        if (tid >= c0 && tid < bw) {  // products of the finished columns k < c0
          T v[CH];
#pragma unroll
          for (int j = 0; j < CH; ++j) v[j] = Ld[tid][c0 + j];
          for (int k0 = 0; k0 < c0; k0 += 4) {  // c0 is a multiple of 16
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const T lik = Ld[tid][k0 + u];
              T lk[CH];
              load_row16(lk, &LdT[k0 + u][c0]);
#pragma unroll
              for (int j = 0; j < CH; ++j) v[j] = v[j] - lik * lk[j];
            }
          }
#pragma unroll
          for (int j = 0; j < CH; ++j) Ld[tid][c0 + j] = v[j];
        }
        __syncthreads();
        if (tid < 32) {
          const int ra = c0 + lane, rb = c0 + 32 + lane;  // rb > every column of the chunk
          T va[CH], vb[CH];
#pragma unroll
          for (int j = 0; j < CH; ++j) {
            va[j] = ra < bw ? Ld[ra][c0 + j] : T(0);
            vb[j] = rb < bw ? Ld[rb][c0 + j] : T(0);
          }
          int bad = 0;
#pragma unroll
          for (int cc = 0; cc < CH; ++cc) {  // the chunk's columns, one at a time
            if (cc < cw && !bad) {
              const T d = __shfl_sync(0xffffffffu, va[cc], cc);  // row c's running diagonal
              if (!(d > T(0))) {  // not positive, or NaN: breakdown (uniform over the warp)
                bad = c0 + cc + 1;
              } else {
                const T piv = sqrt(d);
                const T rpiv = T(1) / piv;  // the column is scaled by 1 / L_cc
                va[cc] = lane == cc ? piv : va[cc] * rpiv;
                vb[cc] = vb[cc] * rpiv;
#pragma unroll
                for (int cc2 = cc + 1; cc2 < CH; ++cc2) {
                  const T l = __shfl_sync(0xffffffffu, va[cc], cc2);  // L_{c0+cc2, c}
                  va[cc2] = va[cc2] - va[cc] * l;
                  vb[cc2] = vb[cc2] - vb[cc] * l;
                }
              }
            }
          }
          // the chunk's columns of rows >= c0 (entries on or below the diagonal)
#pragma unroll
          for (int j = 0; j < CH; ++j) {
            if (j < cw && ra < bw && c0 + j <= ra) {
              Ld[ra][c0 + j] = va[j];
              LdT[c0 + j][ra] = va[j];
            }
            if (j < cw && rb < bw) {
              Ld[rb][c0 + j] = vb[j];
              LdT[c0 + j][rb] = vb[j];
            }
          }
          if (lane == 0) s_bad = bad;
        }
        __syncthreads();
        if (s_bad) {  // uniform
          if (blockIdx.x == 0 && tid == 0) atomicCAS(status, 0, (int)(j0 + s_bad));
          if (MODE != PANEL_DIAG) cp_async_wait_all();
          return;
        }
      }
    }
    if (s_last) {
      for (int idx = tid; idx < PB * PB; idx += ROWS) {
        const int i = idx / PB, k = idx % PB;
        if (i < bw && k <= i) D[(int64_t)i * ld + k] = Ld[i][k];
      }
    }
  }

  if constexpr (MODE != PANEL_DIAG) {
    // ---- rows below the block: thread t owns row row0 + blockIdx.x * ROWS + t
    cp_async_wait_all();  // this thread's own copies into its column of Ys
    if (!has_row) return;
    for (int c0 = 0; c0 < bw; c0 += CH) {
      const int cw = min(CH, bw - c0);
      T y[CH];
#pragma unroll
      for (int j = 0; j < CH; ++j) y[j] = Ys[c0 + j][tid];
      for (int k0 = 0; k0 < c0; k0 += 4) {  // products of the finished columns
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const T yk = Ys[k0 + u][tid];
          T lk[CH];
          load_row16(lk, &LdT[k0 + u][c0]);
#pragma unroll
          for (int j = 0; j < CH; ++j) y[j] = y[j] - yk * lk[j];
        }
      }
#pragma unroll
      for (int j = 0; j < CH; ++j) {  // the chunk's columns, one at a time
        if (j < cw) {
          const T yj = y[j] / LdT[c0 + j][c0 + j];
          y[j] = yj;
#pragma unroll
          for (int j2 = j + 1; j2 < CH; ++j2) y[j2] = y[j2] - yj * LdT[c0 + j][c0 + j2];
        }
      }
#pragma unroll
      for (int j = 0; j < CH; ++j)
        if (j < cw) {
          Ys[c0 + j][tid] = y[j];
          row[c0 + j] = y[j];
        }
    }
  }
}

// ---------------------------------------------------------------------- LU
template <typename T, typename Tc>
__global__ void __launch_bounds__(DIAG_THREADS)
    lu_diag_kernel(T *__restrict__ W, int64_t ld, int64_t j0, int bw, int *status) {
  __shared__ Tc S[64][65];
  if (load_status(status) != 0) return;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  T *D = W + j0 * ld + j0;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = ty + 16 * a, j = tx + 16 * b;
      S[i][j] = (i < bw && j < bw) ? (Tc)D[(int64_t)i * ld + j] : Tc(0);
    }
  __syncthreads();
  for (int c = 0; c < bw; ++c) {
    const Tc p = S[c][c];  // L_cc = A_cc - sum_{k<c} L_ck U_kc
    if (p == Tc(0) || p != p) {
      if (tid == 0) atomicCAS(status, 0, (int)(j0 + c + 1));
      return;
    }
    if (tid > c && tid < bw) S[c][tid] = S[c][tid] / p;  // U_ci
    __syncthreads();
    const int m = bw - c - 1;  // trailing m x m block, enumerated densely
    for (int e = tid; e < m * m; e += DIAG_THREADS) {
      const int i = c + 1 + e / m, j = c + 1 + e % m;
      S[i][j] = S[i][j] - S[i][c] * S[c][j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = ty + 16 * a, j = tx + 16 * b;
      if (i < bw && j < bw) D[(int64_t)i * ld + j] = (T)S[i][j];
    }
}

// Rows of L below the block: x_c = a_c - sum_{k<c} x_k U_kc (no division,
// U is unitriangular).
template <typename T, int B>
__global__ void __launch_bounds__(ROWS_PER_CTA)
    lu_rows_kernel(T *__restrict__ W, int64_t ld, int64_t row0, int64_t nrows, int64_t j0,
                   int bw, const int *status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T(*UT)[B + 1] = reinterpret_cast<T(*)[B + 1]>(smem_raw);  // UT[c][k] = U_kc, k < c
  T(*X)[B + 1] = reinterpret_cast<T(*)[B + 1]>(smem_raw + sizeof(T) * B * (B + 1));
  if (load_status(status) != 0) return;
  const int tid = threadIdx.x;
  const int64_t rbase = row0 + (int64_t)blockIdx.x * ROWS_PER_CTA;
  const int rows_here = (int)min64(ROWS_PER_CTA, row0 + nrows - rbase);
  for (int idx = tid; idx < B * B; idx += ROWS_PER_CTA) {
    const int k = idx / B, c = idx % B;
    UT[c][k] = (k < bw && c < bw && k < c) ? W[(j0 + k) * ld + j0 + c] : T(0);
  }
  for (int idx = tid; idx < ROWS_PER_CTA * B; idx += ROWS_PER_CTA) {
    const int r = idx / B, j = idx % B;
    X[r][j] = (r < rows_here && j < bw) ? W[(rbase + r) * ld + j0 + j] : T(0);
  }
  __syncthreads();
  if (tid < rows_here) {
    T x[B];
#pragma unroll
    for (int c = 0; c < B; ++c) x[c] = X[tid][c];
#pragma unroll
    for (int c = 0; c < B; ++c) {
      if (c < bw) {
        const T xc = x[c];
#pragma unroll
        for (int c2 = c + 1; c2 < B; ++c2) x[c2] = x[c2] - xc * UT[c2][c];
      }
    }
#pragma unroll
    for (int c = 0; c < B; ++c) X[tid][c] = x[c];
  }
  __syncthreads();
  for (int idx = tid; idx < ROWS_PER_CTA * B; idx += ROWS_PER_CTA) {
    const int r = idx / B, j = idx % B;
    if (r < rows_here && j < bw) W[(rbase + r) * ld + j0 + j] = X[r][j];
  }
}

// Columns of U right of the block: y_c = (a_c - sum_{k<c} L_ck y_k) / L_cc.
// One thread per column; loads along a row are coalesced across threads.
template <typename T, int B>
__global__ void __launch_bounds__(ROWS_PER_CTA)
    lu_cols_kernel(T *__restrict__ W, int64_t ld, int64_t col0, int64_t ncols, int64_t j0,
                   int bw, const int *status) {
  __shared__ T LD[B][B + 1];
  if (load_status(status) != 0) return;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < B * B; idx += ROWS_PER_CTA) {
    const int i = idx / B, j = idx % B;
    LD[i][j] = (i < bw && j <= i) ? W[(j0 + i) * ld + j0 + j] : T(0);
  }
  __syncthreads();
  const int64_t q = col0 + (int64_t)blockIdx.x * ROWS_PER_CTA + tid;
  if (q >= col0 + ncols) return;
  T y[B];
#pragma unroll
  for (int c = 0; c < B; ++c) y[c] = (c < bw) ? W[(j0 + c) * ld + q] : T(0);
#pragma unroll
  for (int c = 0; c < B; ++c) {
    if (c < bw) {
      const T yc = y[c] / LD[c][c];
      y[c] = yc;
#pragma unroll
      for (int c2 = c + 1; c2 < B; ++c2) y[c2] = y[c2] - LD[c2][c] * yc;
    }
  }
#pragma unroll
  for (int c = 0; c < B; ++c)
    if (c < bw) W[(j0 + c) * ld + q] = y[c];
}

// ------------------------------------------------------------------- copies
template <typename Tin, typename Tout>
__global__ void copy_matrix_kernel(const Tin *__restrict__ A, int64_t lda, Tout *__restrict__ W,
                                   int64_t ldw, int64_t n, int lower_only) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  for (int64_t i = blockIdx.y; i < n; i += gridDim.y) {
    Tout v = (!lower_only || j <= i) ? (Tout)A[i * lda + j] : Tout(0);
    W[i * ldw + j] = v;
  }
}

// rows x cols block of A into W, cast; with lower_only the entries above the
// block's own diagonal (j > i) are zero
template <typename Tin, typename Tout>
__global__ void copy_slab_kernel(const Tin *__restrict__ A, int64_t lda, Tout *__restrict__ W,
                                 int64_t ldw, int64_t rows, int64_t cols, int lower_only) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  for (int64_t i = blockIdx.y; i < rows; i += gridDim.y) {
    Tout v = (!lower_only || j <= i) ? (Tout)A[i * lda + j] : Tout(0);
    W[i * ldw + j] = v;
  }
}

}  // namespace

// ------------------------------------------------------------------ launchers
template <typename T, int B>
constexpr size_t rows_smem_bytes() {
  return sizeof(T) * (size_t)(B + ROWS_PER_CTA) * (B + 1);
}

// Opt a kernel into more than 48 KB of dynamic shared memory (once per
// instantiation; a repeated call is harmless).
template <typename K>
cudaError_t allow_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, int B>
cudaError_t lu_rows_b(T *W, int64_t ld, int64_t row0, int64_t nrows, int64_t j0, int bw,
                      int *status, cudaStream_t st) {
  constexpr size_t smem = rows_smem_bytes<T, B>();
  static cudaError_t attr = allow_smem(lu_rows_kernel<T, B>, smem);
  if (attr != cudaSuccess) return attr;
  const unsigned grid = (unsigned)ceil_div(nrows, ROWS_PER_CTA);
  lu_rows_kernel<T, B><<<grid, ROWS_PER_CTA, smem, st>>>(W, ld, row0, nrows, j0, bw, status);
  count_launch();
  return cudaGetLastError();
}

template <typename T, int MODE, int ROWS>
cudaError_t panel_launch(unsigned grid, T *W, int64_t ld, int64_t j0, int bw, int64_t nrows,
                         int *status, unsigned long long *arrivals, cudaStream_t st) {
  constexpr size_t smem = PanelSmem<T>::bytes(ROWS);
  static cudaError_t attr = allow_smem(chol_panel_kernel<T, MODE, ROWS>, smem);
  if (attr != cudaSuccess) return attr;
  chol_panel_kernel<T, MODE, ROWS><<<grid, ROWS, smem, st>>>(W, ld, j0, bw, j0 + bw, nrows,
                                                           status, arrivals);
  count_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_chol_panel(T *W, int64_t ld, int64_t j0, int bw, int64_t nrows, int *status,
                              unsigned long long *arrivals, cudaStream_t st) {
  if (bw < 1 || bw > PB) return cudaErrorInvalidValue;
  if (sizeof(T) == 8) {
    // FP64: the block's DFMA work once (one CTA), then the rows over every SM
    cudaError_t e = panel_launch<T, PANEL_DIAG, 64>(1, W, ld, j0, bw, 0, status, arrivals, st);
    if (e != cudaSuccess || nrows <= 0) return e;
    return panel_launch<T, PANEL_ROWS_ONLY, 64>((unsigned)((nrows + 63) / 64), W, ld, j0, bw,
                                                 nrows, status, arrivals, st);
  }
  const int64_t grid = std::max<int64_t>(1, (nrows + 127) / 128);
  return panel_launch<T, PANEL_FUSED, 128>((unsigned)grid, W, ld, j0, bw, nrows, status, arrivals,
                                            st);
}

template <typename T, typename Tc>
cudaError_t launch_lu_diag(T *W, int64_t ld, int64_t j0, int bw, int *status, cudaStream_t st) {
  if (bw < 1 || bw > 64) return cudaErrorInvalidValue;
  lu_diag_kernel<T, Tc><<<1, DIAG_THREADS, 0, st>>>(W, ld, j0, bw, status);
  count_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_lu_rows(T *W, int64_t ld, int64_t row0, int64_t nrows, int64_t j0, int bw,
                           int *status, cudaStream_t st) {
  if (nrows <= 0) return cudaSuccess;
  if (bw < 1 || bw > 64) return cudaErrorInvalidValue;
  if (bw <= 32) return lu_rows_b<T, 32>(W, ld, row0, nrows, j0, bw, status, st);
  return lu_rows_b<T, 64>(W, ld, row0, nrows, j0, bw, status, st);
}

template <typename T>
cudaError_t launch_lu_cols(T *W, int64_t ld, int64_t col0, int64_t ncols, int64_t j0, int bw,
                           int *status, cudaStream_t st) {
  if (ncols <= 0) return cudaSuccess;
  if (bw < 1 || bw > 64) return cudaErrorInvalidValue;
  const unsigned grid = (unsigned)ceil_div(ncols, ROWS_PER_CTA);
  if (bw <= 32)
    lu_cols_kernel<T, 32><<<grid, ROWS_PER_CTA, 0, st>>>(W, ld, col0, ncols, j0, bw, status);
  else
    lu_cols_kernel<T, 64><<<grid, ROWS_PER_CTA, 0, st>>>(W, ld, col0, ncols, j0, bw, status);
  count_launch();
  return cudaGetLastError();
}

template <typename Tin, typename Tout>
cudaError_t launch_copy_matrix(const Tin *A, int64_t lda, Tout *W, int64_t ldw, int64_t n,
                               bool lower_only, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  dim3 block(256), grid((unsigned)ceil_div(n, 256), (unsigned)min64(n, 65535));
  copy_matrix_kernel<Tin, Tout><<<grid, block, 0, st>>>(A, lda, W, ldw, n, lower_only ? 1 : 0);
  count_launch();
  return cudaGetLastError();
}

template <typename Tin, typename Tout>
cudaError_t launch_copy_slab(const Tin *A, int64_t lda, Tout *W, int64_t ldw, int64_t rows,
                             int64_t cols, bool lower_only, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  const dim3 block(256), grid((unsigned)((cols + 255) / 256), (unsigned)std::min<int64_t>(rows, 4096));
  copy_slab_kernel<Tin, Tout><<<grid, block, 0, st>>>(A, lda, W, ldw, rows, cols, lower_only ? 1 : 0);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t launch_copy_slab<double, double>(const double *, int64_t, double *, int64_t,
                                                      int64_t, int64_t, bool, cudaStream_t);
template cudaError_t launch_copy_slab<float, float>(const float *, int64_t, float *, int64_t,
                                                    int64_t, int64_t, bool, cudaStream_t);
template cudaError_t launch_copy_slab<double, float>(const double *, int64_t, float *, int64_t,
                                                     int64_t, int64_t, bool, cudaStream_t);

template cudaError_t launch_chol_panel<double>(double *, int64_t, int64_t, int, int64_t, int *, unsigned long long *, cudaStream_t);
template cudaError_t launch_chol_panel<float>(float *, int64_t, int64_t, int, int64_t, int *, unsigned long long *, cudaStream_t);
template cudaError_t launch_lu_diag<double, double>(double *, int64_t, int64_t, int, int *, cudaStream_t);
template cudaError_t launch_lu_diag<float, float>(float *, int64_t, int64_t, int, int *, cudaStream_t);
template cudaError_t launch_lu_diag<float, double>(float *, int64_t, int64_t, int, int *, cudaStream_t);
template cudaError_t launch_lu_rows<double>(double *, int64_t, int64_t, int64_t, int64_t, int, int *, cudaStream_t);
template cudaError_t launch_lu_rows<float>(float *, int64_t, int64_t, int64_t, int64_t, int, int *, cudaStream_t);
template cudaError_t launch_lu_cols<double>(double *, int64_t, int64_t, int64_t, int64_t, int, int *, cudaStream_t);
template cudaError_t launch_lu_cols<float>(float *, int64_t, int64_t, int64_t, int64_t, int, int *, cudaStream_t);
template cudaError_t launch_copy_matrix<double, double>(const double *, int64_t, double *, int64_t, int64_t, bool, cudaStream_t);
template cudaError_t launch_copy_matrix<float, float>(const float *, int64_t, float *, int64_t, int64_t, bool, cudaStream_t);
template cudaError_t launch_copy_matrix<double, float>(const double *, int64_t, float *, int64_t, int64_t, bool, cudaStream_t);

}  // namespace gb
