// One level of Strassen's multiplication for the delayed update
// C -= X op(Y) (arXiv:1812.02056 Sec. 2: the rectangular product "using a
// fast rectangular matrix multiplication algorithm"; the paper's timings use
// Strassen recursions on the rectangles, after Knight 1995).
//
// With X, Y and C split into 2 x 2 blocks (A = X, B = op(Y)):
//   M1 = (A11 + A22)(B11 + B22)   M5 = (A11 + A12) B22
//   M2 = (A21 + A22) B11          M6 = (A21 - A11)(B11 + B12)
//   M3 = A11 (B12 - B22)          M7 = (A12 - A22)(B21 + B22)
//   M4 = A22 (B21 - B11)
//   C11 -= M1 + M4 - M5 + M7      C12 -= M3 + M5
//   C21 -= M2 + M4                C22 -= M1 - M2 + M3 + M6
// Each product is formed in a workspace P by the classical update kernel
// (P = 0; P -= SA SB, so P = -M_i) and added into the blocks of C.  Odd
// M, N or K leave a last row, column or rank-1 term, applied classically.
#include "gb_internal.cuh"

namespace gb {
namespace {

// out[i][k] = X(i0a + i, k0a + k) + beta * X(i0b + i, k0b + k)
template <typename T>
__global__ void form_a_kernel(T *out, int64_t ldo, const T *X, int64_t ldx, int64_t i0a,
                              int64_t k0a, int64_t i0b, int64_t k0b, T beta, int64_t rows,
                              int64_t cols) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= cols) return;
  for (int64_t i = blockIdx.y; i < rows; i += gridDim.y) {
    T v = X[(i0a + i) * ldx + k0a + k];
    if (beta != T(0)) v = v + beta * X[(i0b + i) * ldx + k0b + k];
    out[i * ldo + k] = v;
  }
}

// out[k][j] = B(k0a + k, j0a + j) + beta * B(k0b + k, j0b + j), B = op(Y):
// nn: B(k, j) = Y[k * ldy + j]; otherwise B(k, j) = Y[j * ldy + k].
template <typename T>
__global__ void form_b_kernel(T *out, int64_t ldo, const T *Y, int64_t ldy, int nn, int64_t k0a,
                              int64_t j0a, int64_t k0b, int64_t j0b, T beta, int64_t rows,
                              int64_t cols) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  for (int64_t k = blockIdx.y; k < rows; k += gridDim.y) {
    T v = nn ? Y[(k0a + k) * ldy + j0a + j] : Y[(j0a + j) * ldy + k0a + k];
    if (beta != T(0)) v = v + beta * (nn ? Y[(k0b + k) * ldy + j0b + j] : Y[(j0b + j) * ldy + k0b + k]);
    out[k * ldo + j] = v;
  }
}

// C[i][j] += sign * P[i][j]
template <typename T>
__global__ void accum_kernel(T *C, int64_t ldc, const T *P, int64_t ldp, T sign, int64_t rows,
                             int64_t cols) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  for (int64_t i = blockIdx.y; i < rows; i += gridDim.y) C[i * ldc + j] += sign * P[i * ldp + j];
}

dim3 grid_for(int64_t rows, int64_t cols) {
  return dim3((unsigned)((cols + 255) / 256), (unsigned)std::min<int64_t>(rows, 65535));
}

}  // namespace

size_t strassen_work_bytes(int64_t M, int64_t N, int64_t K, size_t esz) {
  const int64_t M2 = M / 2, N2 = N / 2, K2 = K / 2;
  return (size_t)(M2 * K2 + K2 * N2 + M2 * N2) * esz + 256;
}

template <typename T>
cudaError_t launch_update_strassen(T *C, int64_t ldc, const T *X, int64_t ldx, const T *Y,
                                   int64_t ldy, int64_t M, int64_t N, int64_t K, bool nn,
                                   const int *status, void *work, size_t work_bytes,
                                   cudaStream_t st) {
  const int64_t M2 = M / 2, N2 = N / 2, K2 = K / 2;
  if (M2 < 1 || N2 < 1 || K2 < 1)
    return launch_update_simt<T>(C, ldc, X, ldx, Y, ldy, M, N, K, nn, false, 0, status, st);
  if (strassen_work_bytes(M, N, K, sizeof(T)) > work_bytes) return cudaErrorInvalidValue;
  T *SA = reinterpret_cast<T *>(work);
  T *SB = SA + M2 * K2;
  T *P = SB + K2 * N2;
  // block (bi, bk) of A and (bk, bj) of B, as element offsets
  auto a_off = [&](int bi, int bk, int64_t &i0, int64_t &k0) {
    i0 = bi * M2;
    k0 = bk * K2;
  };
  auto b_off = [&](int bk, int bj, int64_t &k0, int64_t &j0) {
    k0 = bk * K2;
    j0 = bj * N2;
  };
  struct Term {
    int a1i, a1k, a2i, a2k, asign;  // SA = A(a1) + asign * A(a2); asign 0: A(a1)
    int b1k, b1j, b2k, b2j, bsign;
    int tgt[4][2];                   // C blocks receiving this product
    int sgn[4];                      // sign of -M_i in each (P = -M_i)
    int ntgt;
  };
  const Term terms[7] = {
      {0, 0, 1, 1, 1, 0, 0, 1, 1, 1, {{0, 0}, {1, 1}}, {1, 1}, 2},     // M1
      {1, 0, 1, 1, 1, 0, 0, 0, 0, 0, {{1, 0}, {1, 1}}, {1, -1}, 2},    // M2
      {0, 0, 0, 0, 0, 0, 1, 1, 1, -1, {{0, 1}, {1, 1}}, {1, 1}, 2},    // M3
      {1, 1, 1, 1, 0, 1, 0, 0, 0, -1, {{0, 0}, {1, 0}}, {1, 1}, 2},    // M4
      {0, 0, 0, 1, 1, 1, 1, 1, 1, 0, {{0, 0}, {0, 1}}, {-1, 1}, 2},    // M5
      {1, 0, 0, 0, -1, 0, 0, 0, 1, 1, {{1, 1}}, {1}, 1},               // M6
      {0, 1, 1, 1, -1, 1, 0, 1, 1, 1, {{0, 0}}, {1}, 1},               // M7
  };
  cudaError_t e;
  for (const Term &t : terms) {
    int64_t i1, k1, i2, k2, kb1, j1, kb2, j2;
    a_off(t.a1i, t.a1k, i1, k1);
    a_off(t.a2i, t.a2k, i2, k2);
    form_a_kernel<T><<<grid_for(M2, K2), 256, 0, st>>>(SA, K2, X, ldx, i1, k1, i2, k2, (T)t.asign,
                                                       M2, K2);
    b_off(t.b1k, t.b1j, kb1, j1);
    b_off(t.b2k, t.b2j, kb2, j2);
    form_b_kernel<T><<<grid_for(K2, N2), 256, 0, st>>>(SB, N2, Y, ldy, nn ? 1 : 0, kb1, j1, kb2, j2,
                                                       (T)t.bsign, K2, N2);
    count_launch(2);
    if ((e = cudaMemsetAsync(P, 0, sizeof(T) * M2 * N2, st)) != cudaSuccess) return e;
    if ((e = launch_update_simt<T>(P, N2, SA, K2, SB, N2, M2, N2, K2, true, false, 0, status,
                                   st)) != cudaSuccess)
      return e;
    for (int q = 0; q < t.ntgt; ++q) {
      T *Cb = C + (int64_t)t.tgt[q][0] * M2 * ldc + (int64_t)t.tgt[q][1] * N2;
      accum_kernel<T><<<grid_for(M2, N2), 256, 0, st>>>(Cb, ldc, P, N2, (T)t.sgn[q], M2, N2);
      count_launch();
    }
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // classical remainders
  const T *Yk = nn ? Y + 2 * K2 * ldy : Y + 2 * K2;  // B row 2K2 (odd K)
  if (K % 2)
    if ((e = launch_update_simt<T>(C, ldc, X + 2 * K2, ldx, Yk, ldy, M, N, 1, nn, false, 0, status,
                                   st)) != cudaSuccess)
      return e;
  if (M % 2)
    if ((e = launch_update_simt<T>(C + (M - 1) * ldc, ldc, X + (M - 1) * ldx, ldx, Y, ldy, 1,
                                   2 * N2, 2 * K2, nn, false, 0, status, st)) != cudaSuccess)
      return e;
  if (N % 2) {
    const T *Yn = nn ? Y + (N - 1) : Y + (N - 1) * ldy;  // B column N - 1
    if ((e = launch_update_simt<T>(C + (N - 1), ldc, X, ldx, Yn, ldy, M, 1, 2 * K2, nn, false, 0,
                                   status, st)) != cudaSuccess)
      return e;
  }
  return cudaSuccess;
}

template cudaError_t launch_update_strassen<double>(double *, int64_t, const double *, int64_t,
                                                    const double *, int64_t, int64_t, int64_t,
                                                    int64_t, bool, const int *, void *, size_t,
                                                    cudaStream_t);
template cudaError_t launch_update_strassen<float>(float *, int64_t, const float *, int64_t,
                                                   const float *, int64_t, int64_t, int64_t,
                                                   int64_t, bool, const int *, void *, size_t,
                                                   cudaStream_t);

}  // namespace gb
