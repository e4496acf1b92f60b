// Internal declarations of the gbchol library (not installed, not part of the
// C ABI).  Kernels live in panel.cu (column steps), update_simt.cu (SIMT
// rank-s update), update_tc.cu (tcgen05 rank-s update), solve.cu (triangular
// solves, residual, backward error), batched.cu; the host-side block loop and
// the exported entry points live in abi.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "../../include/gbchol.h"

namespace gb {

// ------------------------------------------------------------------ errors
#define GB_CUDA_TRY(expr)                                  \
  do {                                                     \
    cudaError_t _e = (expr);                               \
    if (_e != cudaSuccess) {                               \
      ::gb::record_cuda_error(_e, #expr, __FILE__, __LINE__); \
      return GB_ERR_CUDA;                                  \
    }                                                      \
  } while (0)

void record_cuda_error(cudaError_t e, const char *what, const char *file, int line);

// Launch counter behind gb_kernel_launches(); every launcher bumps it.
extern std::atomic<uint64_t> g_launches;
inline void count_launch(uint64_t k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }
const char *last_error_message();

// Device error word bits (handle->d_err): set by kernels instead of trapping.
enum : int {
  DEV_ERR_TIMEOUT = 1,   // a bounded spin wait gave up
  DEV_ERR_BOUNDS = 2,    // a self-check found an index out of range
  DEV_ERR_TMEM = 4,      // tensor-memory allocation returned an unusable address
};

// ------------------------------------------------------------------ handle
struct Workspace {
  void *ptr = nullptr;
  size_t bytes = 0;
};

}  // namespace gb

struct gb_handle {
  int device = 0;
  int sm_count = 0;
  int inner_step = 64;
  int use_graphs = 1;
  int tc_update = 2;
  int qr_inner = 16;          // inner step of the QR panel (GB_OPT_QR_INNER_STEP)
  int left_looking = 0;       // GB_OPT_LEFT_LOOKING
  int test_withhold = 0;      // GB_OPT_TEST_WITHHOLD (test hook, 0 = off)
  int inner_cuda_cores = 0;   // GB_OPT_INNER_CUDA_CORES
  int inner_recursive = 2;    // GB_OPT_INNER_RECURSIVE
  int inner_lookahead = 2;    // GB_OPT_INNER_LOOKAHEAD
  int early_rest = 2;         // GB_OPT_EARLY_REST
  int residual = 2;           // GB_OPT_RESIDUAL
  int f64_update = 0;         // GB_OPT_F64_UPDATE
  int digits_reserve = 16;    // SMs the look-ahead stream's digit updates leave free
  cudaStream_t aux2 = nullptr;  // high priority: the inner updates' rest (inner look-ahead)
  cudaEvent_t ev_ip = nullptr, ev_ir = nullptr;  // inner block's columns final / inner rest done
  // device copies of host buffers come from this pool, which keeps its
  // memory between calls (allocating and mapping it again each call costs
  // more than the copies)
  cudaMemPool_t stage_pool = nullptr;
  // steps chosen by gb_tune_step for s = 0: [kind: chol, LU, QR][dtype][floor(log2 n)]
  struct TunedStep {
    int64_t s = 0;
    int b = 0;
  } tuned[3][5][32];
  int64_t spin_limit = 1 << 26;
  int *d_status = nullptr;   // scratch status word for host `info` pointers
  int *d_err = nullptr;      // device error word (DEV_ERR_*)
  int *d_sync = nullptr;     // flags / tickets for single-kernel solves (SYNC_WORDS ints)
  unsigned long long *d_arrivals = nullptr;  // arrival counter of the fused panel kernel
  double *d_scalars = nullptr;  // small FP64 reduction outputs
  unsigned sync_epoch = 0;
  gb::Workspace ws[12];      // named workspaces, see WS_* below
  std::mutex mu;
  // GB_OPT_PROFILE: event pairs recorded around launches, read later
  int profile = 0;
  int lookahead = 1;                  // GB_OPT_LOOKAHEAD
  int strassen = 0;                   // GB_OPT_STRASSEN
  cudaStream_t hi = nullptr;          // high priority: column steps and next-block updates
  cudaStream_t aux = nullptr;         // low priority: the rest of each update
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_next = nullptr;      // next block's columns updated (main stream)
  cudaEvent_t ev_rest = nullptr;      // rest of the update done (aux stream)
  // Host-buffer Cholesky: each finished block column is copied to the host
  // on `cpy` while the factorization goes on (set by factor_common)
  cudaStream_t cpy = nullptr;
  cudaEvent_t ev_cpy = nullptr;
  // Host-input Cholesky: A arrives in column slabs of s columns (rows from
  // the slab's first column down), each cast into W on `cpy`; slab k is
  // ready when ev_in[k] completes (set by factor_common)
  struct CopyIn {
    bool active = false;
    int64_t s = 0;
  } cin;
  std::vector<cudaEvent_t> ev_in;
  struct CopyOut {
    bool active = false;
    void *host = nullptr;
    int64_t ldh = 0;
    const void *dev = nullptr;
    int64_t ldd = 0, n = 0;
    size_t esz = 0;
  } cout;
  struct ProfRec {
    int phase;
    cudaEvent_t start, stop;
    double flops, bytes;
    bool owns_start = true;  // false: start is an earlier record's stop
  };
  std::vector<ProfRec> prof_pending;
  std::vector<cudaEvent_t> prof_pool;
  // batched: step per order bucket (index 0 FP64, 1 FP32), 0 = default rule
  int batched_step[2][32] = {};
  int batched_exact = 0;
  // the uploaded batched plan (device addresses inside ws[WS_MISC])
  struct BatchPlanDev {
    int count = 0;
    int dt = -1;
    const int *order = nullptr, *n = nullptr, *step = nullptr;
    void *const *A = nullptr;
    void *const *L = nullptr;
    const int64_t *lda = nullptr, *ldl = nullptr;
    int *ticket = nullptr;
    int lu = 0;  // 1: Algorithm 2 (LU), 0: Algorithm 1 (Cholesky)
  } plan;
};

namespace gb {

enum { WS_STAGE = 0, WS_PANEL = 1, WS_SOLVE = 2, WS_MISC = 3, WS_DINV = 4, WS_PANEL2 = 5,
       WS_STRAS = 6, WS_STRAS2 = 7, WS_QR = 8, WS_LEFT = 9, WS_INNER = 10,
       WS_SPLIT = 11 };
constexpr int SYNC_WORDS = 1 << 16;

// Make sure workspace `slot` holds >= bytes; waits for `stream` before
// releasing an older, smaller buffer.
gb_status ws_reserve(gb_handle *h, int slot, size_t bytes, cudaStream_t stream);

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }
__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

// ------------------------------------------------------------ kernels (host)
// Column steps of one inner block [j0, j0+bw) of the working matrix W (row
// major, ld), rows j0..n-1, storage T.
// Cholesky: fused column steps of one inner block (diagonal block in every
// CTA, then its rows); `arrivals` is a zeroed counter the kernel leaves zeroed.
template <typename T>
cudaError_t launch_chol_panel(T *W, int64_t ld, int64_t j0, int bw, int64_t nrows, int *status,
                              unsigned long long *arrivals, cudaStream_t st);
template <typename T, typename Tc>
cudaError_t launch_lu_diag(T *W, int64_t ld, int64_t j0, int bw, int *status, cudaStream_t st);
template <typename T>
cudaError_t launch_lu_rows(T *W, int64_t ld, int64_t row0, int64_t nrows, int64_t j0, int bw,
                           int *status, cudaStream_t st);
template <typename T>
cudaError_t launch_lu_cols(T *W, int64_t ld, int64_t col0, int64_t ncols, int64_t j0, int bw,
                           int *status, cudaStream_t st);

// C[i][j] -= sum_k X[i][k] * Y(k, j), 0 <= i < M, 0 <= j < N, 0 <= k < K.
//   nn = false: Y(k, j) = Y[j * ldy + k]   (Cholesky, Y = R)
//   nn = true:  Y(k, j) = Y[k * ldy + j]   (LU, Y = U panel)
//   lower: update only elements with i + diag >= j.
template <typename T>
cudaError_t launch_update_simt(T *C, int64_t ldc, const T *X, int64_t ldx, const T *Y,
                               int64_t ldy, int64_t M, int64_t N, int64_t K, bool nn, bool lower,
                               int64_t diag, const int *status, cudaStream_t st);

// One level of Strassen for C -= X op(Y) (no lower mask); workspace of
// strassen_work_bytes.  Odd sizes leave classical remainders.
size_t strassen_work_bytes(int64_t M, int64_t N, int64_t K, size_t esz);
template <typename T>
cudaError_t launch_update_strassen(T *C, int64_t ldc, const T *X, int64_t ldx, const T *Y,
                                   int64_t ldy, int64_t M, int64_t N, int64_t K, bool nn,
                                   const int *status, void *work, size_t work_bytes,
                                   cudaStream_t st);

// Elementwise copies.  Lower-triangle copy with zeroed strict upper (chol)
// or full copy (lu); Tin -> Tout.
template <typename Tin, typename Tout>
cudaError_t launch_copy_matrix(const Tin *A, int64_t lda, Tout *W, int64_t ldw, int64_t n,
                               bool lower_only, cudaStream_t st);
// rows x cols block (A's and W's pointers at its top-left corner), zero above
// the block's own diagonal with lower_only
template <typename Tin, typename Tout>
cudaError_t launch_copy_slab(const Tin *A, int64_t lda, Tout *W, int64_t ldw, int64_t rows,
                             int64_t cols, bool lower_only, cudaStream_t st);

// tcgen05 mixed update (update_tc.cu).  Packs the panel to 16-bit operands and
// runs the tensor-core kernel.  Returns cudaErrorNotSupported if the device
// cannot run it.
struct TcUpdateArgs {
  float *C;          // working matrix (FP32), rows/cols start at (r0, r0)
  int64_t ldc;
  const float *X;    // panel rows (FP32), X[i * ldx + k]
  int64_t ldx;
  const float *Y;    // nn = false: Y[j * ldy + k]; nn = true: Y[k * ldy + j]
  int64_t ldy;
  int64_t M, N, K;
  bool nn;
  bool lower;
  int64_t diag;
  bool f16;          // FP16 operands instead of BF16
  int split;         // 1: plain 16-bit operands; 3: three-plane BF16 split
                     //    (the six leading plane products, ~FP32 accuracy)
  const int *status;
  int *err;
  int64_t spin_limit;
  void *pack;        // workspace for the packed operands
  size_t pack_bytes;
  int cluster;       // 2: CTA pairs with pair MMAs (256 x 256 tiles); else 1
  // resident operands (optional): 16-bit rows of X and Y, leading dimensions
  // in elements; then X, Y and pack are not used and K must be a multiple of 64
  const void *xpack, *ypack;
  int64_t ldxp, ldyp;
  cudaEvent_t packed; // optional: recorded on the stream between the packing
                      // launches and the tensor-core kernel (profiling)
};
// Round an FP32 rows x K block to 16-bit rows of ldo elements (K rounded up
// to 64 with zeros) -- the resident operand layout of the update.
cudaError_t launch_pack16(const float *X, int64_t ldx, int64_t rows, int64_t K, void *out,
                          int64_t ldo, bool f16, cudaStream_t st);
size_t tc_pack_bytes(int64_t M, int64_t N, int64_t K, bool nn, int split);
cudaError_t launch_update_tc(const TcUpdateArgs &a, cudaStream_t st);
bool tc_supported(int device);
// tensor-pipe peak loop: kind 0 BF16, 1 FP16 (kind::f16), 2 TF32 (kind::tf32)
cudaError_t measure_tc_peak(int kind, int sm_count, double *flops_per_s);

// Solves (solve.cu)
template <typename Tf, typename Tc>
cudaError_t launch_trsm(const Tf *F, int64_t ldf, double *B, int64_t ldb, int64_t n,
                        int64_t nrhs, int kind, int *sync, unsigned epoch, int *err,
                        int64_t spin_limit, cudaStream_t st);
enum { TRSM_LOWER = 0, TRSM_LOWER_T = 1, TRSM_UNIT_UPPER = 2 };
// Solve through inverted diagonal blocks: launch_diag_inv fills Dinv
// (trsm_inv_bytes), launch_coupling the coupling blocks M (trsm_inv_bytes:
// block p couples position p to position p - 1), then launch_trsm_inv
// solves in place like launch_trsm.
size_t trsm_inv_bytes(int64_t n, size_t esz);
template <typename Tf>
cudaError_t launch_diag_inv(const Tf *F, int64_t ldf, int64_t n, int kind, Tf *Dinv,
                            cudaStream_t st);
template <typename Tf>
cudaError_t launch_coupling(const Tf *F, int64_t ldf, const Tf *Dinv, int64_t n, int kind, Tf *M,
                            cudaStream_t st);
template <typename Tf>
cudaError_t launch_trsm_inv(const Tf *F, int64_t ldf, const Tf *Dinv, const Tf *M, double *B,
                            int64_t ldb, int64_t n, int64_t nrhs, int kind, int *sync,
                            unsigned epoch, int *err, int64_t spin_limit, cudaStream_t st,
                            int withhold = -1);
// r = b - A x in FP64 (and the norms of r, x, b per column when `norms`);
// small orders split the columns of A into slices whose partial products go
// to `work` (residual_work_bytes; without it, one slice).
cudaError_t launch_residual(const double *A, int64_t lda, const double *X, int64_t ldx,
                            const double *B, int64_t ldb, double *R, int64_t ldr, int64_t n,
                            int64_t nrhs, double *norms, double *work, size_t work_bytes,
                            int sm_count, cudaStream_t st);
size_t residual_work_bytes(int64_t n, int64_t nrhs, int sm_count);
cudaError_t launch_inf_norm_rows(const double *A, int64_t lda, int64_t n, double *out,
                                 cudaStream_t st);
// The same residual from exact digit products on the tensor cores
// (residual_tc.cu): launch_split_a writes A's digit planes and row scales to
// `work` (split_a_bytes) and ||A||_inf to *anorm; launch_residual_split then
// computes r = b - A x with the norms of r, x and b (as launch_residual),
// using `xwork` (split_x_bytes) for the digits of x and partial sums.
// FP64-accurate delayed update C -= X Y^T (lower, j <= i) from exact digit
// products on the tensor cores (update_digits.cu); `work` of
// update_digits_bytes (same: Y is X's first N rows).  At most `max_ctas`
// persistent CTAs (one per SM): fewer leave SMs to concurrent column steps.
size_t update_digits_bytes(int64_t M, int64_t N, int64_t K, bool same);
// lower: only j <= i (Cholesky); else every element.  y_kxn: Y is K x N
// (LU's R_U), else N x K.
cudaError_t launch_update_digits(double *C, int64_t ldc, const double *X, int64_t ldx,
                                 const double *Y, int64_t ldy, int64_t M, int64_t N, int64_t K,
                                 bool lower, bool y_kxn, const int *status, int *err,
                                 int64_t spin_limit, void *work, size_t work_bytes, int max_ctas,
                                 cudaStream_t st);
// GB_OPT_RESIDUAL 2 (default): the digit products from this order up
constexpr int64_t SPLIT_RESIDUAL_MIN_N = 2048;
size_t split_a_bytes(int64_t n);
size_t split_x_bytes(int64_t n, int64_t nrhs, int sm_count);
cudaError_t launch_split_a(const double *A, int64_t lda, int64_t n, void *work, double *anorm,
                           cudaStream_t st);
cudaError_t launch_residual_split(const void *awork, int64_t n, const double *X, int64_t ldx,
                                  const double *B, int64_t ldb, double *R, int64_t ldr,
                                  int64_t nrhs, double *norms, void *xwork, int sm_count, int *err,
                                  long long wait_ns, cudaStream_t st);
cudaError_t launch_axpy_cols(double *X, int64_t ldx, const double *D, int64_t ldd, int64_t n,
                             int64_t nrhs, cudaStream_t st);
template <typename Tf>
cudaError_t launch_backward_error(int is_lu, const double *A, int64_t lda, const Tf *F,
                                  int64_t ldf, int64_t n, double *acc, cudaStream_t st);
template <typename Tf>
cudaError_t launch_check_diag(const Tf *F, int64_t ldf, int64_t n, int *flag, cudaStream_t st);

// Batched (batched.cu): one persistent launch over a plan in device memory
// (order = LPT permutation, per-matrix order n, step, pointer, leading
// dimension, info); `ticket` is reset by the launcher.
constexpr int BATCH_MAX_N = 1024;
constexpr int BATCH_BUCKETS = 32;  // step table: orders 1..1024 in buckets of 32
size_t batched_smem_bytes();
template <typename T>
cudaError_t launch_chol_batched_plan(int count, const int *order, const int *n, const int *step,
                                     void *const *A, const int64_t *lda, void *const *L,
                                     const int64_t *ldl, int *info, int *ticket, int sm_count,
                                     int exact, cudaStream_t st);
// The same for Algorithm 2 (compact LU written to L[i] with ldl[i]).
template <typename T>
cudaError_t launch_lu_batched_plan(int count, const int *order, const int *n, const int *step,
                                   void *const *A, const int64_t *lda, void *const *LU,
                                   const int64_t *ldlu, int *info, int *ticket, int sm_count,
                                   int exact, cudaStream_t st);
// Algorithm 3 (qr.cu).  Column steps of columns [col0, col0 + bb) of the
// n x n working matrix Qm on one cluster of 8 CTAs (bb <= qr_panel_max_cols).
int64_t qr_panel_max_cols(int64_t n, size_t esz);
template <typename T>
cudaError_t launch_qr_panel(T *Qm, int64_t ldq, int64_t n, int64_t col0, int bb, int *status,
                            int *err, int64_t spin_limit, cudaStream_t st);
// C := X^T Y (X: K x M, Y: K x N, row-major); upper: C's upper triangle,
// zeros below.  Skinny results split K into `work` when it is large enough
// (gemm_tn_work_bytes).
size_t gemm_tn_work_bytes(size_t esz, int sm_count);
template <typename T>
cudaError_t launch_gemm_tn(T *C, int64_t ldc, const T *X, int64_t ldx, const T *Y, int64_t ldy,
                           int64_t M, int64_t N, int64_t K, bool upper, const int *status,
                           void *work, size_t work_bytes, int sm_count, cudaStream_t st);
template <typename T>
cudaError_t launch_fill_spd(T *base, int64_t stride, int count, int n, cudaStream_t st);

}  // namespace gb
