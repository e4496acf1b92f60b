// Exported C entry points of gbchol (declared in include/gbchol.h) and the
// host-side block loops of Algorithms 1 and 2 (arXiv:1812.02056, Sec. 2).
//
// Block loop (Cholesky; LU is the same with the U panel alongside):
//   for z = 0, s, 2s, ...:                     checkpoint z, block width sb
//     for each inner block [j0, j0+bw) of [z, z+sb):   bw <= inner step
//       diagonal block column steps            (panel.cu, chol_diag_kernel)
//       rows below the block                   (panel.cu, chol_rows_kernel)
//       rest of the s-block's columns -= this inner block's product
//     A[z+sb.., z+sb..] -= R R^T, R = L[z+sb.., z..z+sb)   (the delayed
//                                              rank-s update; SIMT or tcgen05)
// With s <= inner step each s-block is one inner block and the loop is
// Algorithm 1 as written: the columns of a block are finished from the
// columns since z, and the trailing matrix sees one update every s columns.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <memory>
#include <cmath>
#include <string>
#include <vector>

#include "gb_internal.cuh"

namespace gb {

static thread_local std::string g_last_error;
std::atomic<uint64_t> g_launches{0};

void record_cuda_error(cudaError_t e, const char *what, const char *file, int line) {
  char buf[512];
  snprintf(buf, sizeof buf, "%s:%d: %s -> %s", file, line, what, cudaGetErrorString(e));
  g_last_error = buf;
}

const char *last_error_message() { return g_last_error.c_str(); }

gb_status ws_reserve(gb_handle *h, int slot, size_t bytes, cudaStream_t stream) {
  Workspace &w = h->ws[slot];
  if (w.bytes >= bytes) return GB_OK;
  if (w.ptr) {
    GB_CUDA_TRY(cudaStreamSynchronize(stream));
    GB_CUDA_TRY(cudaFree(w.ptr));
    w.ptr = nullptr;
    w.bytes = 0;
  }
  size_t want = std::max<size_t>(bytes, 1 << 20);
  if (cudaMalloc(&w.ptr, want) != cudaSuccess) {
    cudaGetLastError();
    w.ptr = nullptr;
    return GB_ERR_NOMEM;
  }
  w.bytes = want;
  return GB_OK;
}

namespace {

// ---------------------------------------------------------------- helpers
bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

size_t elem_size_factor(gb_dtype dt) { return dt == GB_F64 ? 8 : 4; }
size_t elem_size_input(gb_dtype dt) { return dt == GB_F32 ? 4 : 8; }
bool valid_dtype(int dt) { return dt >= GB_F64 && dt <= GB_MIX_BF16X3; }
bool is_mixed(gb_dtype dt) { return dt == GB_MIX_BF16 || dt == GB_MIX_F16 || dt == GB_MIX_BF16X3; }
int split_of(gb_dtype dt) { return dt == GB_MIX_BF16X3 ? 3 : 1; }

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// A caller buffer that may live on the host: device copy for the duration of
// a call, released in stream order.
struct Staged {
  void *dev = nullptr;
  const void *host_src = nullptr;
  void *host_dst = nullptr;
  int64_t rows = 0, cols = 0, ld = 0, ldd = 0;
  size_t esz = 0;
  bool owned = false;
  cudaStream_t st = nullptr;

  // Take `p` (rows x cols, leading dimension ld, element size esz).  When
  // `p` is host memory, allocate a dense device copy (copying in when
  // copy_in) and remember to copy out at finish() when copy_out.
  gb_status take(const void *p, int64_t r, int64_t c, int64_t l, size_t e, bool copy_in,
                 bool copy_out, cudaStream_t s, cudaMemPool_t pool) {
    rows = r;
    cols = c;
    ld = l;
    esz = e;
    st = s;
    if (!p || is_device_ptr(p)) {
      dev = const_cast<void *>(p);
      ldd = l;
      return GB_OK;
    }
    ldd = c > 0 ? c : 1;
    size_t bytes = (size_t)std::max<int64_t>(r, 1) * (size_t)ldd * e;
    const cudaError_t ae =
        pool ? cudaMallocFromPoolAsync(&dev, bytes, pool, s) : cudaMallocAsync(&dev, bytes, s);
    if (ae != cudaSuccess) {
      cudaGetLastError();
      dev = nullptr;
      return GB_ERR_NOMEM;
    }
    owned = true;
    if (copy_out) host_dst = const_cast<void *>(p);
    if (copy_in && r > 0 && c > 0) {
      if (l == c)  // dense rows: one linear copy
        GB_CUDA_TRY(cudaMemcpyAsync(dev, p, (size_t)r * c * e, cudaMemcpyHostToDevice, s));
      else
        GB_CUDA_TRY(cudaMemcpy2DAsync(dev, ldd * e, p, l * e, c * e, r, cudaMemcpyHostToDevice, s));
    }
    return GB_OK;
  }
  gb_status finish() {
    if (host_dst && rows > 0 && cols > 0) {
      if (ld == cols)
        GB_CUDA_TRY(cudaMemcpyAsync(host_dst, dev, (size_t)rows * cols * esz,
                                    cudaMemcpyDeviceToHost, st));
      else
        GB_CUDA_TRY(cudaMemcpy2DAsync(host_dst, ld * esz, dev, ldd * esz, cols * esz, rows,
                                      cudaMemcpyDeviceToHost, st));
    }
    return GB_OK;
  }
  ~Staged() {
    if (owned && dev) cudaFreeAsync(dev, st);
  }
  bool on_host() const { return owned; }
};

// Status word for `info`: the caller's int when it is device memory, else
// the handle's scratch word copied out at the end.
struct InfoWord {
  int *dev = nullptr;
  int *host = nullptr;
  gb_status init(gb_handle *h, int *info, cudaStream_t st) {
    if (is_device_ptr(info)) {
      dev = info;
    } else {
      dev = h->d_status;
      host = info;
    }
    GB_CUDA_TRY(cudaMemsetAsync(dev, 0, sizeof(int), st));
    return GB_OK;
  }
  gb_status finish(cudaStream_t st) {
    if (host) {
      GB_CUDA_TRY(cudaMemcpyAsync(host, dev, sizeof(int), cudaMemcpyDeviceToHost, st));
      GB_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return GB_OK;
  }
};

int tune_bucket(int64_t n) {
  int b = 0;
  while (b < 31 && ((int64_t)2 << b) <= n) ++b;
  return b;  // floor(log2 n) for n >= 1
}

// The tuned (s, inner step) for a call with s = 0, or {0, 0} when none.
gb_handle::TunedStep tuned_step(const gb_handle *h, int kind, gb_dtype dt, int64_t n) {
  if (kind < 0 || kind > 2 || dt < 0 || dt > 4 || n < 1) return {};
  return h->tuned[kind][dt][tune_bucket(n)];
}

int64_t default_step(gb_dtype dt, int64_t n) {
  (void)n;
  switch (dt) {
    case GB_F64: return 256;
    case GB_F32: return 256;
    default: return 1024;
  }
}

// ---------------------------------------------------------------- profile
cudaEvent_t take_event(gb_handle *h) {
  if (!h->prof_pool.empty()) {
    cudaEvent_t e = h->prof_pool.back();
    h->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Records an event pair around the launches made in its scope when the
// handle's profile option is on.
struct PhaseTimer {
  gb_handle *h;
  cudaStream_t st;
  int phase;
  double flops, bytes;
  cudaEvent_t a = nullptr, b = nullptr;
  PhaseTimer(gb_handle *h_, cudaStream_t st_, int phase_, double flops_, double bytes_)
      : h(h_), st(st_), phase(phase_), flops(flops_), bytes(bytes_) {
    if (!h->profile) return;
    a = take_event(h);
    b = take_event(h);
    if (a && b) cudaEventRecord(a, st);
  }
  ~PhaseTimer() {
    if (!a || !b) return;
    cudaEventRecord(b, st);
    h->prof_pending.push_back({phase, a, b, flops, bytes});
  }
};

// Number of (i, j), 0 <= i < M, 0 <= j < N, with i + diag >= j.
double lower_count(int64_t M, int64_t N, int64_t diag) {
  double c = 0;
  for (int64_t j0 = 0; j0 < N; j0 += 4096) {  // closed form per column strip
    const int64_t j1 = std::min(N, j0 + 4096);
    for (int64_t j = j0; j < j1; ++j) {
      const int64_t first = std::max<int64_t>(0, j - diag);
      if (first < M) c += (double)(M - first);
    }
  }
  return c;
}

double update_flops(int64_t M, int64_t N, int64_t K, bool lower) {
  return 2.0 * (double)K * (lower ? lower_count(M, N, 0) : (double)M * N);
}

double update_bytes(int64_t M, int64_t N, int64_t K, bool lower, size_t e) {
  const double c = lower ? lower_count(M, N, 0) : (double)M * N;
  return (double)e * (2.0 * c + (double)(M + N) * K);
}

// ------------------------------------------------------------ block loops
// C[i][j] -= sum_k X[i][k] X[j][k] over the lower part of an M x N block
// (Cholesky's delayed update or part of it), on the tensor cores for the
// mixed dtypes, on the CUDA cores otherwise.  `pack_slot` names the packed-
// operand workspace of the stream the call is issued on.
// C -= X op(Y), no mask, through one Strassen level when the option is on
// and the block is large enough to profit; `slot` is the stream's workspace.
template <typename T>
gb_status general_update(gb_handle *h, T *C, int64_t ldc, const T *X, int64_t ldx, const T *Y,
                         int64_t ldy, int64_t M, int64_t N, int64_t K, bool nn, int *status,
                         int slot, cudaStream_t st) {
  if (h->strassen && std::min(M, N) >= 512 && K >= 32) {
    gb_status r = ws_reserve(h, slot, strassen_work_bytes(M, N, K, sizeof(T)), st);
    if (r != GB_OK) return r;
    GB_CUDA_TRY(launch_update_strassen<T>(C, ldc, X, ldx, Y, ldy, M, N, K, nn, status,
                                          h->ws[slot].ptr, h->ws[slot].bytes, st));
    return GB_OK;
  }
  GB_CUDA_TRY(launch_update_simt<T>(C, ldc, X, ldx, Y, ldy, M, N, K, nn, false, 0, status, st));
  return GB_OK;
}

template <typename T>
gb_status chol_update(gb_handle *h, gb_dtype dt, T *C, const T *X, const T *Y, int64_t ld,
                      int64_t M, int64_t N, int64_t K, int *status, int pack_slot,
                      cudaStream_t st) {
  if (M <= 0 || N <= 0 || K <= 0) return GB_OK;
  if constexpr (sizeof(T) == 8) {
    if (dt == GB_F64 && h->f64_update == 1 && tc_supported(h->device)) {
      // FP64 accuracy from exact digit products on the tensor cores
      const bool same = X == Y && N <= M;
      gb_status ws = ws_reserve(h, pack_slot, update_digits_bytes(M, N, K, same), st);
      if (ws != GB_OK) return ws;
      // the rest of an update under look-ahead leaves SMs to the column
      // steps, whose CTAs could not share an SM with the update's
      const int ctas = st == h->aux ? std::max(1, h->sm_count - h->digits_reserve) : h->sm_count;
      GB_CUDA_TRY(launch_update_digits(C, ld, X, ld, Y, ld, M, N, K, true, false, status,
                                       h->d_err, h->spin_limit, h->ws[pack_slot].ptr,
                                       h->ws[pack_slot].bytes, ctas, st));
      return GB_OK;
    }
  }
  if constexpr (sizeof(T) == 4) {
    if (is_mixed(dt) && h->tc_update) {
      TcUpdateArgs a{};
      a.C = reinterpret_cast<float *>(C);
      a.ldc = ld;
      a.X = reinterpret_cast<const float *>(X);
      a.ldx = ld;
      a.Y = reinterpret_cast<const float *>(Y);
      a.ldy = ld;
      a.M = M;
      a.N = N;
      a.K = K;
      a.nn = false;
      a.lower = true;
      a.diag = 0;
      a.f16 = (dt == GB_MIX_F16);
      a.split = split_of(dt);
      a.status = status;
      a.err = h->d_err;
      a.spin_limit = h->spin_limit;
      a.cluster = h->tc_update;
      gb_status ws = ws_reserve(h, pack_slot, tc_pack_bytes(M, N, K, false, a.split), st);
      if (ws != GB_OK) return ws;
      a.pack = h->ws[pack_slot].ptr;
      a.pack_bytes = h->ws[pack_slot].bytes;
      GB_CUDA_TRY(launch_update_tc(a, st));
      return GB_OK;
    }
  }
  if (h->strassen && M == N && X == Y && M >= 1024 && K >= 32) {
    // square lower update: two classical halves on the diagonal, the
    // off-diagonal block C21 -= R2 R1^T through Strassen
    const int64_t m1 = M / 2, m2 = M - m1;
    const int slot = pack_slot == WS_PANEL2 ? WS_STRAS2 : WS_STRAS;
    GB_CUDA_TRY(launch_update_simt<T>(C, ld, X, ld, X, ld, m1, m1, K, false, true, 0, status, st));
    gb_status r = general_update<T>(h, C + m1 * ld, ld, X + m1 * ld, ld, X, ld, m2, m1, K, false,
                                    status, slot, st);
    if (r != GB_OK) return r;
    GB_CUDA_TRY(launch_update_simt<T>(C + m1 * ld + m1, ld, X + m1 * ld, ld, X + m1 * ld, ld, m2,
                                      m2, K, false, true, 0, status, st));
    return GB_OK;
  }
  GB_CUDA_TRY(launch_update_simt<T>(C, ld, X, ld, Y, ld, M, N, K, false, true, 0, status, st));
  return GB_OK;
}

template <typename T, typename Tc>
gb_status chol_blocked_on(gb_handle *h, int64_t n, int64_t s, T *W, int64_t ld, int *status,
                          gb_dtype dt, cudaStream_t st, bool la);

// Look-ahead runs the column steps and each next-block update on the
// high-priority stream and the rest of each update on the low-priority one,
// forked from and joined back to the caller's stream.
template <typename T, typename Tc>
gb_status chol_blocked(gb_handle *h, int64_t n, int64_t s, T *W, int64_t ld, int *status,
                       gb_dtype dt, cudaStream_t st) {
  const bool la = h->lookahead && h->hi && h->aux && n > s + s;
  if (!la) return chol_blocked_on<T, Tc>(h, n, s, W, ld, status, dt, st, false);
  GB_CUDA_TRY(cudaEventRecord(h->ev_fork, st));
  GB_CUDA_TRY(cudaStreamWaitEvent(h->hi, h->ev_fork, 0));
  gb_status r = chol_blocked_on<T, Tc>(h, n, s, W, ld, status, dt, h->hi, true);
  GB_CUDA_TRY(cudaEventRecord(h->ev_join, h->hi));
  GB_CUDA_TRY(cudaStreamWaitEvent(st, h->ev_join, 0));
  return r;
}

template <typename T, typename Tc>
gb_status chol_blocked_on(gb_handle *h, int64_t n, int64_t s, T *W, int64_t ld, int *status,
                          gb_dtype dt, cudaStream_t st, bool la) {
  const int64_t b = std::max(1, std::min(64, h->inner_step));
  const size_t e = sizeof(T);
  if (la && is_mixed(dt) && h->tc_update) {
    // both pack workspaces at their largest before anything is in flight
    const int64_t m0 = n - std::min(s, n);
    const size_t pb = tc_pack_bytes(m0, m0, std::min(s, n), false, split_of(dt));
    gb_status r = ws_reserve(h, WS_PANEL, pb, st);
    if (r == GB_OK) r = ws_reserve(h, WS_PANEL2, pb, h->aux);
    if (r != GB_OK) return r;
  }
  if (h->inner_lookahead == 1 && h->aux2 && is_mixed(dt) && h->tc_update) {
    const size_t pb = tc_pack_bytes(n, n, std::min(s, n), false, split_of(dt));
    gb_status r = ws_reserve(h, WS_INNER, pb, h->aux2);
    if (r != GB_OK) return r;
  }
  if (dt == GB_F64 && h->f64_update == 1) {
    // the digit workspaces of every stream at their largest before anything
    // is in flight (a later growth would free a buffer another stream uses)
    const size_t db = update_digits_bytes(n, n, std::min(s, n), true);
    gb_status r = ws_reserve(h, WS_PANEL, db, st);
    if (r == GB_OK && la) r = ws_reserve(h, WS_PANEL2, db, h->aux);
    if (r == GB_OK && h->aux2) r = ws_reserve(h, WS_INNER, db, h->aux2);
    if (r != GB_OK) return r;
  }
  bool rest_pending = false;
  // host input arriving in column slabs (h->cin): wait for slab k on `on`
  auto slab_ready = [&](int64_t col, cudaStream_t on) -> gb_status {
    if (!h->cin.active || col >= n) return GB_OK;
    GB_CUDA_TRY(cudaStreamWaitEvent(on, h->ev_in[(size_t)(col / h->cin.s)], 0));
    return GB_OK;
  };
  for (int64_t z = 0; z < n; z += s) {
    const int64_t sb = std::min(s, n - z);
    const int64_t pe = z + sb;  // end of this s-block
    gb_status rw = slab_ready(z, st);  // the s-block's columns have arrived
    if (rw != GB_OK) return rw;
    // mixed dtypes: the products inside the s-block on the tensor cores, or
    // in FP32 on the CUDA cores (GB_OPT_INNER_CUDA_CORES)
    const gb_dtype di = (is_mixed(dt) && h->inner_cuda_cores) ? GB_F32 : dt;
    // Columns [c, hi) (rows from c down) receive the product of columns
    // [k0, k0 + K) (rows from c down).  With GB_OPT_INNER_LOOKAHEAD the next
    // inner block's columns receive it first, on the column-step stream, and
    // the rest of the range on aux2 while the next column steps run; every
    // later write to the range from `st` waits for that rest first.
    // 2 (default): FP64 only (n = 8192: 1061.8 -> 1063.5 GFLOP/s; the mixed
    // dtypes measured slower, their tensor-core rest competing with the
    // column steps for SMs)
    const bool ila = h->aux2 && (h->inner_lookahead == 1 ||
                                 (h->inner_lookahead == 2 && dt == GB_F64));
    bool inner_pending = false;
    auto give = [&](int64_t c, int64_t hi, int64_t k0, int64_t K) -> gb_status {
      const int64_t nb = ila ? std::min(b, hi - c) : hi - c;
      if (inner_pending) GB_CUDA_TRY(cudaStreamWaitEvent(st, h->ev_ir, 0));
      {
        PhaseTimer t(h, st, GB_PHASE_INNER, update_flops(n - c, nb, K, true),
                     update_bytes(n - c, nb, K, true, e));
        const T *R = W + c * ld + k0;
        gb_status r = chol_update<T>(h, di, W + c * ld + c, R, R, ld, n - c, nb, K, status,
                                     WS_PANEL, st);
        if (r != GB_OK) return r;
      }
      const int64_t c2 = c + nb;
      if (c2 >= hi) return GB_OK;
      GB_CUDA_TRY(cudaEventRecord(h->ev_ip, st));
      GB_CUDA_TRY(cudaStreamWaitEvent(h->aux2, h->ev_ip, 0));
      {
        PhaseTimer t(h, h->aux2, GB_PHASE_INNER, update_flops(n - c2, hi - c2, K, true),
                     update_bytes(n - c2, hi - c2, K, true, e));
        const T *R = W + c2 * ld + k0;
        gb_status r = chol_update<T>(h, di, W + c2 * ld + c2, R, R, ld, n - c2, hi - c2, K, status,
                                     WS_INNER, h->aux2);
        if (r != GB_OK) return r;
      }
      GB_CUDA_TRY(cudaEventRecord(h->ev_ir, h->aux2));
      inner_pending = true;
      return GB_OK;
    };
    // columns [lo, hi) of the s-block, all rows from lo down, given every
    // earlier column's contribution: inner blocks of b columns, each giving
    // its product to the range's remaining columns; with GB_OPT_INNER_RECURSIVE
    // a range wider than two inner blocks is split in halves (multiples of
    // b), the right half receiving the whole left half in one product.
    auto flat = [&](int64_t lo, int64_t hi) -> gb_status {
      for (int64_t j0 = lo; j0 < hi; j0 += b) {
        const int bw = (int)std::min(b, hi - j0);
        const int64_t r0 = j0 + bw;
        {
          // diagonal block and the rows below it
          PhaseTimer t(h, st, GB_PHASE_PANEL,
                       (double)bw * bw * bw / 3.0 + (double)(n - r0) * bw * bw,
                       (double)bw * bw * e + 2.0 * (double)(n - r0) * bw * e);
          GB_CUDA_TRY(launch_chol_panel<T>(W, ld, j0, bw, n - r0, status, h->d_arrivals, st));
        }
        if (r0 < hi) {  // the range's remaining columns receive this inner block
          gb_status r = give(r0, hi, j0, bw);
          if (r != GB_OK) return r;
        }
      }
      return GB_OK;
    };
    // 2 (default): halves except for the FP32 dtype, whose CUDA-core inner
    // updates measured faster flat (n = 8192: 10.23 against 10.40 ms)
    const bool halves = h->inner_recursive == 1 || (h->inner_recursive == 2 && dt != GB_F32);
    auto range = [&](auto &&self, int64_t lo, int64_t hi) -> gb_status {
      if (!halves || hi - lo <= 2 * b) return flat(lo, hi);
      const int64_t mid = lo + ((hi - lo) / 2 + b - 1) / b * b;
      gb_status r = self(self, lo, mid);
      if (r == GB_OK) r = give(mid, hi, lo, mid - lo);
      if (r != GB_OK) return r;
      return self(self, mid, hi);
    };
    {
      gb_status r = range(range, z, pe);
      if (r != GB_OK) return r;
      // the block column is final: later readers of it on `st` see every write
      if (inner_pending) GB_CUDA_TRY(cudaStreamWaitEvent(st, h->ev_ir, 0));
    }
    if (h->cout.active) {
      // columns [z, pe) are final (rows above z are zero): copy them out
      GB_CUDA_TRY(cudaEventRecord(h->ev_cpy, st));
      GB_CUDA_TRY(cudaStreamWaitEvent(h->cpy, h->ev_cpy, 0));
      // rows from z down (the zeros above the block column are written on
      // the host by factor_common)
      const auto &c = h->cout;
      GB_CUDA_TRY(cudaMemcpy2DAsync((char *)c.host + (z * c.ldh + z) * c.esz, c.ldh * c.esz,
                                    (const char *)c.dev + (z * c.ldd + z) * c.esz, c.ldd * c.esz,
                                    sb * c.esz, n - z, cudaMemcpyDeviceToHost, h->cpy));
    }
    if (pe >= n) break;
    // delayed rank-sb update A[pe.., pe..] -= R R^T, R = L[pe.., z..pe)
    const int64_t m = n - pe;
    const T *R = W + pe * ld + z;
    // first block with host input still arriving: the trailing update in
    // strips of one slab each (the lower part of columns [c, c + s), rows
    // from c), each after its slab; every element still receives the same
    // K-sum.  Later blocks find every slab in place.
    const bool strips = h->cin.active && z == 0;
    auto strip_update = [&](int64_t q, int slot, cudaStream_t on) -> gb_status {
      for (int64_t c = q; c < n; c += s) {
        gb_status r = slab_ready(c, on);
        if (r != GB_OK) return r;
        const int64_t w = std::min(s, n - c);
        const T *Rc = W + c * ld + z;
        r = chol_update<T>(h, dt, W + c * ld + c, Rc, Rc, ld, n - c, w, sb, status, slot, on);
        if (r != GB_OK) return r;
      }
      return GB_OK;
    };
    if (!la) {
      PhaseTimer t(h, st, GB_PHASE_UPDATE, update_flops(m, m, sb, true),
                   update_bytes(m, m, sb, true, e));
      gb_status r = strips ? strip_update(pe, WS_PANEL, st)
                           : chol_update<T>(h, dt, W + pe * ld + pe, R, R, ld, m, m, sb, status,
                                            WS_PANEL, st);
      if (r != GB_OK) return r;
      continue;
    }
    const int64_t nb = std::min(s, n - pe);  // width of the next s-block
    const int64_t q = pe + nb;  // the rest: rows and columns from q on
    // GB_OPT_EARLY_REST: the rest of this update needs only this block's
    // columns, not the next block's update: start it first, alongside that
    // update.  2 (default): FP64 only (n = 8192, s = 256: 172.2 -> 170.1 ms;
    // the FP32 and mixed dtypes measured 4-8% slower, the narrow update on
    // the critical path sharing the SMs with the rest)
    const bool early = q < n && (h->early_rest == 1 || (h->early_rest == 2 && dt == GB_F64));
    if (early) {
      GB_CUDA_TRY(cudaEventRecord(h->ev_next, st));
      GB_CUDA_TRY(cudaStreamWaitEvent(h->aux, h->ev_next, 0));
    }
    // the previous rest-update wrote the next block's columns: wait for it
    if (rest_pending) GB_CUDA_TRY(cudaStreamWaitEvent(st, h->ev_rest, 0));
    {
      PhaseTimer t(h, st, GB_PHASE_UPDATE, update_flops(m, nb, sb, true),
                   update_bytes(m, nb, sb, true, e));
      gb_status r = slab_ready(pe, st);  // the next block's columns have arrived
      if (r == GB_OK)
        r = chol_update<T>(h, dt, W + pe * ld + pe, R, R, ld, m, nb, sb, status, WS_PANEL, st);
      if (r != GB_OK) return r;
    }
    if (q < n) {
      if (!early) {
        GB_CUDA_TRY(cudaEventRecord(h->ev_next, st));
        GB_CUDA_TRY(cudaStreamWaitEvent(h->aux, h->ev_next, 0));
      }
      const T *Rq = W + q * ld + z;
      PhaseTimer t(h, h->aux, GB_PHASE_UPDATE, update_flops(n - q, n - q, sb, true),
                   update_bytes(n - q, n - q, sb, true, e));
      gb_status r = strips ? strip_update(q, WS_PANEL2, h->aux)
                           : chol_update<T>(h, dt, W + q * ld + q, Rq, Rq, ld, n - q, n - q, sb,
                                            status, WS_PANEL2, h->aux);
      if (r != GB_OK) return r;
      GB_CUDA_TRY(cudaEventRecord(h->ev_rest, h->aux));
      rest_pending = true;
    }
  }
  if (rest_pending) GB_CUDA_TRY(cudaStreamWaitEvent(st, h->ev_rest, 0));
  return GB_OK;
}

// ---------------------------------------------------- left-looking variant
// The same sums as Algorithm 1 in another grouping (tile accumulation): the
// trailing matrix is never updated; when the s-block [z, z + sb) is reached,
// its columns receive every earlier column's contribution at once,
//   W[z.., z..pe) -= L[z.., 0..z) L[z..pe, 0..z)^T   (K = z >> s),
// on the tensor cores from a resident 16-bit copy of L (each finished block
// column is rounded once into it), then the column steps run as before.
// Mixed dtypes with one 16-bit plane (BF16, FP16); s a multiple of 64.
template <typename T, typename Tc>
gb_status chol_left_on(gb_handle *h, int64_t n, int64_t s, T *W, int64_t ld, int *status,
                       gb_dtype dt, cudaStream_t st) {
  static_assert(sizeof(T) == 4, "tensor-core path: FP32 working matrix");
  const int64_t b = std::max(1, std::min(64, h->inner_step));
  const int64_t ldp = (n + 63) / 64 * 64;  // resident copy: rows of ldp 16-bit elements
  const bool f16 = dt == GB_MIX_F16;
  gb_status r = ws_reserve(h, WS_LEFT, (size_t)n * (size_t)ldp * 2 + 256, st);
  if (r != GB_OK) return r;
  uint16_t *Lp = reinterpret_cast<uint16_t *>(h->ws[WS_LEFT].ptr);
  for (int64_t z = 0; z < n; z += s) {
    const int64_t sb = std::min(s, n - z);
    const int64_t pe = z + sb;
    if (z > 0) {
      PhaseTimer t(h, st, GB_PHASE_UPDATE, update_flops(n - z, sb, z, true),
                   (double)8 * lower_count(n - z, sb, 0) + 2.0 * (double)(n - z + sb) * z);
      TcUpdateArgs a{};
      a.C = reinterpret_cast<float *>(W + z * ld + z);
      a.ldc = ld;
      a.M = n - z;
      a.N = sb;
      a.K = z;
      a.nn = false;
      a.lower = true;
      a.diag = 0;
      a.f16 = f16;
      a.split = 1;
      a.status = status;
      a.err = h->d_err;
      a.spin_limit = h->spin_limit;
      a.cluster = h->tc_update;
      a.xpack = Lp + z * ldp;  // rows z.., columns 0..z of the resident L
      a.ypack = Lp + z * ldp;  // its first sb rows
      a.ldxp = ldp;
      a.ldyp = ldp;
      GB_CUDA_TRY(launch_update_tc(a, st));
    }
    for (int64_t j0 = z; j0 < pe; j0 += b) {
      const int bw = (int)std::min(b, pe - j0);
      const int64_t r0 = j0 + bw;
      {
        PhaseTimer t(h, st, GB_PHASE_PANEL,
                     (double)bw * bw * bw / 3.0 + (double)(n - r0) * bw * bw,
                     (double)bw * bw * 4 + 2.0 * (double)(n - r0) * bw * 4);
        GB_CUDA_TRY(launch_chol_panel<T>(W, ld, j0, bw, n - r0, status, h->d_arrivals, st));
      }
      if (r0 < pe) {
        PhaseTimer t(h, st, GB_PHASE_INNER, update_flops(n - r0, pe - r0, bw, true),
                     update_bytes(n - r0, pe - r0, bw, true, 4));
        const T *R = W + r0 * ld + j0;
        const gb_dtype di = (is_mixed(dt) && h->inner_cuda_cores) ? GB_F32 : dt;
        r = chol_update<T>(h, di, W + r0 * ld + r0, R, R, ld, n - r0, pe - r0, bw, status,
                           WS_PANEL, st);
        if (r != GB_OK) return r;
      }
    }
    if (pe < n) {  // round the finished block column into the resident copy
      PhaseTimer t(h, st, GB_PHASE_COPY, 0.0, (double)(n - z) * sb * 6);
      GB_CUDA_TRY(launch_pack16(reinterpret_cast<const float *>(W + z * ld + z), ld, n - z, sb,
                                Lp + z * ldp + z, ldp, f16, st));
    }
  }
  return GB_OK;
}

// C -= X Y (LU's R_L R_U, full block), tensor cores for the mixed dtypes,
// CUDA cores (optionally one Strassen level) otherwise.
template <typename T>
gb_status lu_update(gb_handle *h, gb_dtype dt, T *C, const T *X, const T *Y, int64_t ld,
                    int64_t M, int64_t N, int64_t K, int *status, int pack_slot,
                    cudaStream_t st) {
  if (M <= 0 || N <= 0 || K <= 0) return GB_OK;
  if constexpr (sizeof(T) == 8) {
    if (dt == GB_F64 && h->f64_update == 1 && tc_supported(h->device)) {
      // FP64 accuracy from exact digit products on the tensor cores: the
      // whole M x N block, R_U (K x N) cut into digits by columns
      gb_status ws = ws_reserve(h, pack_slot, update_digits_bytes(M, N, K, false), st);
      if (ws != GB_OK) return ws;
      // the rest of an update under look-ahead leaves SMs to the column
      // steps, whose CTAs could not share an SM with the update's
      const int ctas = st == h->aux ? std::max(1, h->sm_count - h->digits_reserve) : h->sm_count;
      GB_CUDA_TRY(launch_update_digits(C, ld, X, ld, Y, ld, M, N, K, false, true, status,
                                       h->d_err, h->spin_limit, h->ws[pack_slot].ptr,
                                       h->ws[pack_slot].bytes, ctas, st));
      return GB_OK;
    }
  }
  if constexpr (sizeof(T) == 4) {
    if (is_mixed(dt) && h->tc_update) {
      TcUpdateArgs a{};
      a.C = reinterpret_cast<float *>(C);
      a.ldc = ld;
      a.X = reinterpret_cast<const float *>(X);
      a.ldx = ld;
      a.Y = reinterpret_cast<const float *>(Y);
      a.ldy = ld;
      a.M = M;
      a.N = N;
      a.K = K;
      a.nn = true;
      a.lower = false;
      a.diag = 0;
      a.f16 = (dt == GB_MIX_F16);
      a.split = split_of(dt);
      a.status = status;
      a.err = h->d_err;
      a.spin_limit = h->spin_limit;
      a.cluster = h->tc_update;
      gb_status ws = ws_reserve(h, pack_slot, tc_pack_bytes(M, N, K, true, a.split), st);
      if (ws != GB_OK) return ws;
      a.pack = h->ws[pack_slot].ptr;
      a.pack_bytes = h->ws[pack_slot].bytes;
      GB_CUDA_TRY(launch_update_tc(a, st));
      return GB_OK;
    }
  }
  return general_update<T>(h, C, ld, X, ld, Y, ld, M, N, K, true, status,
                           pack_slot == WS_PANEL2 ? WS_STRAS2 : WS_STRAS, st);
}

// The products inside an s-block of Algorithm 2 (C -= R_L R_U, R_U K x N):
// FP64 multiply-adds on the CUDA cores, or the digit products of
// GB_OPT_F64_UPDATE on `st`'s workspace (WS_PANEL, reserved at its largest
// by lu_blocked_on).
template <typename T>
gb_status lu_inner_update(gb_handle *h, gb_dtype dt, T *C, const T *X, const T *Y, int64_t ld,
                          int64_t M, int64_t N, int64_t K, int *status, cudaStream_t st) {
  if (M <= 0 || N <= 0 || K <= 0) return GB_OK;
  if constexpr (sizeof(T) == 8) {
    if (dt == GB_F64 && h->f64_update == 1 && tc_supported(h->device)) {
      gb_status ws = ws_reserve(h, WS_PANEL, update_digits_bytes(M, N, K, false), st);
      if (ws != GB_OK) return ws;
      GB_CUDA_TRY(launch_update_digits(C, ld, X, ld, Y, ld, M, N, K, false, true, status,
                                       h->d_err, h->spin_limit, h->ws[WS_PANEL].ptr,
                                       h->ws[WS_PANEL].bytes, h->sm_count, st));
      return GB_OK;
    }
  }
  GB_CUDA_TRY(launch_update_simt<T>(C, ld, X, ld, Y, ld, M, N, K, true, false, 0, status, st));
  return GB_OK;
}

template <typename T, typename Tc>
gb_status lu_blocked_on(gb_handle *h, int64_t n, int64_t s, T *W, int64_t ld, int *status,
                        gb_dtype dt, cudaStream_t st, bool la);

template <typename T, typename Tc>
gb_status lu_blocked(gb_handle *h, int64_t n, int64_t s, T *W, int64_t ld, int *status,
                     gb_dtype dt, cudaStream_t st) {
  const bool la = h->lookahead && h->hi && h->aux && n > s + s;
  if (!la) return lu_blocked_on<T, Tc>(h, n, s, W, ld, status, dt, st, false);
  GB_CUDA_TRY(cudaEventRecord(h->ev_fork, st));
  GB_CUDA_TRY(cudaStreamWaitEvent(h->hi, h->ev_fork, 0));
  gb_status r = lu_blocked_on<T, Tc>(h, n, s, W, ld, status, dt, h->hi, true);
  GB_CUDA_TRY(cudaEventRecord(h->ev_join, h->hi));
  GB_CUDA_TRY(cudaStreamWaitEvent(st, h->ev_join, 0));
  return r;
}

template <typename T, typename Tc>
gb_status lu_blocked_on(gb_handle *h, int64_t n, int64_t s, T *W, int64_t ld, int *status,
                        gb_dtype dt, cudaStream_t st, bool la) {
  const int64_t b = std::max(1, std::min(64, h->inner_step));
  const size_t e = sizeof(T);
  if (la && is_mixed(dt) && h->tc_update) {
    const int64_t m0 = n - std::min(s, n);
    const size_t pb = tc_pack_bytes(m0, m0, std::min(s, n), true, split_of(dt));
    gb_status r = ws_reserve(h, WS_PANEL, pb, st);
    if (r == GB_OK) r = ws_reserve(h, WS_PANEL2, pb, h->aux);
    if (r != GB_OK) return r;
  }
  if (dt == GB_F64 && h->f64_update == 1) {
    // the digit workspaces of both streams at their largest before anything
    // is in flight (a later growth would free a buffer another stream uses)
    const size_t db = update_digits_bytes(n, n, std::min(s, n), false);
    gb_status r = ws_reserve(h, WS_PANEL, db, st);
    if (r == GB_OK && la) r = ws_reserve(h, WS_PANEL2, db, h->aux);
    if (r != GB_OK) return r;
  }
  bool rest_pending = false;
  for (int64_t z = 0; z < n; z += s) {
    const int64_t sb = std::min(s, n - z);
    const int64_t pe = z + sb;
    for (int64_t j0 = z; j0 < pe; j0 += b) {
      const int bw = (int)std::min(b, pe - j0);
      {
        PhaseTimer t(h, st, GB_PHASE_DIAG, 2.0 * (double)bw * bw * bw / 3.0, 2.0 * bw * bw * e);
        GB_CUDA_TRY((launch_lu_diag<T, Tc>(W, ld, j0, bw, status, st)));
      }
      const int64_t r0 = j0 + bw;
      if (r0 < n) {
        {
          PhaseTimer t(h, st, GB_PHASE_PANEL, (double)(n - r0) * bw * bw,
                       2.0 * (double)(n - r0) * bw * e);
          GB_CUDA_TRY(launch_lu_rows<T>(W, ld, r0, n - r0, j0, bw, status, st));  // L below
        }
        PhaseTimer t(h, st, GB_PHASE_PANEL, (double)(n - r0) * bw * bw,
                     2.0 * (double)(n - r0) * bw * e);
        GB_CUDA_TRY(launch_lu_cols<T>(W, ld, r0, n - r0, j0, bw, status, st));  // U right
      }
      if (r0 < pe) {
        {
          // the s-block's remaining columns (all rows below) ...
          PhaseTimer t(h, st, GB_PHASE_INNER, update_flops(n - r0, pe - r0, bw, false),
                       update_bytes(n - r0, pe - r0, bw, false, e));
          gb_status r = lu_inner_update<T>(h, dt, W + r0 * ld + r0, W + r0 * ld + j0,
                                           W + j0 * ld + r0, ld, n - r0, pe - r0, bw, status, st);
          if (r != GB_OK) return r;
        }
        // ... and the s-block's remaining rows right of the block
        if (pe < n) {
          PhaseTimer t(h, st, GB_PHASE_INNER, update_flops(pe - r0, n - pe, bw, false),
                       update_bytes(pe - r0, n - pe, bw, false, e));
          gb_status r = lu_inner_update<T>(h, dt, W + r0 * ld + pe, W + r0 * ld + j0,
                                           W + j0 * ld + pe, ld, pe - r0, n - pe, bw, status, st);
          if (r != GB_OK) return r;
        }
      }
    }
    if (pe >= n) break;
    // delayed rank-sb update A[pe.., pe..] -= R_L R_U
    const int64_t m = n - pe;
    const T *RL = W + pe * ld + z;  // rows pe.., columns z..pe
    const T *RU = W + z * ld + pe;  // rows z..pe, columns pe..
    if (!la) {
      PhaseTimer t(h, st, GB_PHASE_UPDATE, update_flops(m, m, sb, false),
                   update_bytes(m, m, sb, false, e));
      gb_status r = lu_update<T>(h, dt, W + pe * ld + pe, RL, RU, ld, m, m, sb, status, WS_PANEL, st);
      if (r != GB_OK) return r;
      continue;
    }
    const int64_t nb = std::min(s, n - pe);
    const int64_t q = pe + nb;
    if (rest_pending) GB_CUDA_TRY(cudaStreamWaitEvent(st, h->ev_rest, 0));
    {
      // the next block's L columns (all rows) and U rows (all columns)
      PhaseTimer t(h, st, GB_PHASE_UPDATE,
                   update_flops(m, nb, sb, false) + update_flops(nb, n - q, sb, false),
                   update_bytes(m, nb, sb, false, e) + update_bytes(nb, n - q, sb, false, e));
      gb_status r = lu_update<T>(h, dt, W + pe * ld + pe, RL, RU, ld, m, nb, sb, status, WS_PANEL, st);
      if (r == GB_OK && q < n)
        r = lu_update<T>(h, dt, W + pe * ld + q, RL, RU + nb, ld, nb, n - q, sb, status, WS_PANEL,
                         st);
      if (r != GB_OK) return r;
    }
    if (q < n) {
      GB_CUDA_TRY(cudaEventRecord(h->ev_next, st));
      GB_CUDA_TRY(cudaStreamWaitEvent(h->aux, h->ev_next, 0));
      PhaseTimer t(h, h->aux, GB_PHASE_UPDATE, update_flops(n - q, n - q, sb, false),
                   update_bytes(n - q, n - q, sb, false, e));
      gb_status r = lu_update<T>(h, dt, W + q * ld + q, RL + nb * ld, RU + nb, ld, n - q, n - q, sb,
                                 status, WS_PANEL2, h->aux);
      if (r != GB_OK) return r;
      GB_CUDA_TRY(cudaEventRecord(h->ev_rest, h->aux));
      rest_pending = true;
    }
  }
  if (rest_pending) GB_CUDA_TRY(cudaStreamWaitEvent(st, h->ev_rest, 0));
  return GB_OK;
}

// Common driver of gb_chol_factor / gb_lu_factor.
// ------------------------------------------------------------- Algorithm 3
// Fast QR with step s: Q (n x n, ldq) holds the working matrix M and ends
// as Q; every s columns the trailing columns lose their components along
// the block just finished (C := B_Q^T B_M, M -= B_Q C).  Inside a block the
// column steps run in inner blocks of b columns (the paper's remark that s
// may vary, Sec. 2): the panel kernel orthogonalises b columns one after
// the other, and the rest of the block's columns receive the same two-GEMM
// projection for those b columns.  Finally R := Q^T A (upper triangle).
template <typename T>
gb_status qr_blocked(gb_handle *h, int64_t n, int64_t s, const T *A, int64_t lda, T *Q,
                     int64_t ldq, T *R, int64_t ldr, int *status, cudaStream_t st) {
  const int64_t bmax = qr_panel_max_cols(n, sizeof(T));
  if (bmax < 1) return GB_ERR_UNSUPPORTED;
  const int64_t b =
      std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(s, (int64_t)h->qr_inner), bmax));
  const size_t esz = sizeof(T);
  const int64_t sw = std::min(s, n);
  gb_status r = ws_reserve(h, WS_QR, (size_t)sw * (size_t)n * esz + 256, st);
  if (r != GB_OK) return r;
  const size_t wbytes = gemm_tn_work_bytes(esz, h->sm_count);
  if ((r = ws_reserve(h, WS_PANEL2, wbytes, st)) != GB_OK) return r;
  T *Cw = reinterpret_cast<T *>(h->ws[WS_QR].ptr);
  void *work = h->ws[WS_PANEL2].ptr;
  for (int64_t z = 0; z < n; z += s) {
    const int64_t sb = std::min(s, n - z);
    for (int64_t z2 = z; z2 < z + sb; z2 += b) {
      const int64_t bb = std::min(b, z + sb - z2);
      {
        PhaseTimer tp(h, st, GB_PHASE_PANEL, 4.0 * (double)n * (double)bb * (double)bb, 0.0);
        GB_CUDA_TRY(launch_qr_panel<T>(Q, ldq, n, z2, (int)bb, status, h->d_err, h->spin_limit,
                                       st));
      }
      const int64_t rest = z + sb - (z2 + bb);
      if (rest > 0) {
        PhaseTimer ti(h, st, GB_PHASE_INNER, 4.0 * (double)n * (double)bb * (double)rest,
                      3.0 * (double)n * (double)rest * (double)esz);
        GB_CUDA_TRY(launch_gemm_tn<T>(Cw, rest, Q + z2, ldq, Q + z2 + bb, ldq, bb, rest, n, false,
                                      status, work, h->ws[WS_PANEL2].bytes, h->sm_count, st));
        GB_CUDA_TRY(launch_update_simt<T>(Q + z2 + bb, ldq, Q + z2, ldq, Cw, rest, n, rest, bb,
                                          true, false, 0, status, st));
      }
    }
    const int64_t m = n - z - sb;
    if (m > 0) {
      PhaseTimer tu(h, st, GB_PHASE_UPDATE, 4.0 * (double)n * (double)sb * (double)m,
                    3.0 * (double)n * (double)m * (double)esz);
      GB_CUDA_TRY(launch_gemm_tn<T>(Cw, m, Q + z, ldq, Q + z + sb, ldq, sb, m, n, false, status,
                                    work, h->ws[WS_PANEL2].bytes, h->sm_count, st));
      GB_CUDA_TRY(launch_update_simt<T>(Q + z + sb, ldq, Q + z, ldq, Cw, m, n, m, sb, true, false,
                                        0, status, st));
    }
  }
  PhaseTimer tr(h, st, GB_PHASE_UPDATE, (double)n * (double)n * (double)(n + 1),
                2.0 * (double)n * (double)n * (double)esz);
  GB_CUDA_TRY(launch_gemm_tn<T>(R, ldr, Q, ldq, A, lda, n, n, n, true, status, nullptr, 0,
                                h->sm_count, st));
  return GB_OK;
}

gb_status qr_common(gb_handle *h, int64_t n, int64_t s, gb_dtype dt, const void *A, int64_t lda,
                    void *Q, int64_t ldq, void *R, int64_t ldr, int *info, void *stream) {
  if (!h) return -1;
  if (n < 0 || n > (int64_t)1 << 30) return -2;
  if (s < 0) return -3;
  if (!valid_dtype(dt)) return -4;
  if (dt != GB_F64 && dt != GB_F32) return GB_ERR_UNSUPPORTED;
  if (n > 0 && !A) return -5;
  if (lda < std::max<int64_t>(1, n)) return -6;
  if (n > 0 && !Q) return -7;
  if (ldq < std::max<int64_t>(1, n)) return -8;
  if (n > 0 && !R) return -9;
  if (ldr < std::max<int64_t>(1, n)) return -10;
  if (!info) return -11;
  const size_t esz = elem_size_input(dt);
  auto span = [&](const void *p, int64_t ld) {
    const char *b = (const char *)p;
    return std::make_pair(b, b + ((size_t)std::max<int64_t>(n - 1, 0) * ld + n) * esz);
  };
  if (n > 0) {  // Q and R are written while A is still read
    auto a = span(A, lda), q = span(Q, ldq), rr = span(R, ldr);
    if (q.first < a.second && a.first < q.second) return -7;
    if (rr.first < a.second && a.first < rr.second) return -9;
    if (rr.first < q.second && q.first < rr.second) return -9;
  }
  DeviceGuard g(h->device);
  std::lock_guard<std::mutex> lk(h->mu);
  cudaStream_t st = (cudaStream_t)stream;
  const int saved_inner = h->qr_inner;
  struct RestoreInner {
    gb_handle *h;
    int v;
    ~RestoreInner() { h->qr_inner = v; }
  } restore_inner{h, saved_inner};
  if (s == 0) {
    const auto t = tuned_step(h, 2, dt, n);
    if (t.s > 0) {
      s = t.s;
      h->qr_inner = t.b;
    } else {
      s = 64;
    }
  }
  InfoWord iw;
  gb_status r = iw.init(h, info, st);
  if (r != GB_OK) return r;
  if (n == 0) return iw.finish(st);
  Staged sa, sq, sr;
  if ((r = sa.take(A, n, n, lda, esz, true, false, st, h->stage_pool)) != GB_OK) return r;
  if ((r = sq.take(Q, n, n, ldq, esz, false, true, st, h->stage_pool)) != GB_OK) return r;
  if ((r = sr.take(R, n, n, ldr, esz, false, true, st, h->stage_pool)) != GB_OK) return r;
  if (dt == GB_F64) {
    GB_CUDA_TRY((launch_copy_matrix<double, double>((const double *)sa.dev, sa.ldd,
                                                    (double *)sq.dev, sq.ldd, n, false, st)));
    r = qr_blocked<double>(h, n, s, (const double *)sa.dev, sa.ldd, (double *)sq.dev, sq.ldd,
                           (double *)sr.dev, sr.ldd, iw.dev, st);
  } else {
    GB_CUDA_TRY((launch_copy_matrix<float, float>((const float *)sa.dev, sa.ldd, (float *)sq.dev,
                                                  sq.ldd, n, false, st)));
    r = qr_blocked<float>(h, n, s, (const float *)sa.dev, sa.ldd, (float *)sq.dev, sq.ldd,
                          (float *)sr.dev, sr.ldd, iw.dev, st);
  }
  if (r != GB_OK) return r;
  if ((r = sq.finish()) != GB_OK) return r;
  if ((r = sr.finish()) != GB_OK) return r;
  if ((r = iw.finish(st)) != GB_OK) return r;
  if (sa.on_host() || sq.on_host() || sr.on_host()) GB_CUDA_TRY(cudaStreamSynchronize(st));
  return GB_OK;
}

// Host input for the right-looking Cholesky: on the copy stream, for each
// column slab [q, q + s): its rows from q down go to the staging buffer, are
// cast into the working matrix (zero above the slab's diagonal) and the rows
// above q are zeroed; ev_in[k] marks slab k ready.  Only the lower triangle
// crosses the link.  The factorization waits for each slab where it first
// reads or updates it.
gb_status slab_copy_in(gb_handle *h, gb_dtype dt, const void *A, int64_t lda, void *Ad,
                       int64_t ldad, void *W, int64_t ldw, int64_t n, int64_t s, cudaStream_t st) {
  const int64_t ns = (n + s - 1) / s;
  while ((int64_t)h->ev_in.size() < ns) {
    cudaEvent_t e = nullptr;
    GB_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    h->ev_in.push_back(e);
  }
  const size_t ein = elem_size_input(dt), ef = elem_size_factor(dt);
  GB_CUDA_TRY(cudaEventRecord(h->ev_cpy, st));  // after the staging allocations
  GB_CUDA_TRY(cudaStreamWaitEvent(h->cpy, h->ev_cpy, 0));
  for (int64_t k = 0; k < ns; ++k) {
    const int64_t q = k * s, w = std::min(s, n - q);
    const char *src = (const char *)A + ((size_t)q * lda + q) * ein;
    char *dst = (char *)Ad + ((size_t)q * ldad + q) * ein;
    GB_CUDA_TRY(cudaMemcpy2DAsync(dst, ldad * ein, src, lda * ein, w * ein, n - q,
                                  cudaMemcpyHostToDevice, h->cpy));
    cudaError_t e;
    if (dt == GB_F64)
      e = launch_copy_slab<double, double>((const double *)dst, ldad, (double *)W + q * ldw + q, ldw,
                                           n - q, w, true, h->cpy);
    else if (dt == GB_F32)
      e = launch_copy_slab<float, float>((const float *)dst, ldad, (float *)W + q * ldw + q, ldw,
                                         n - q, w, true, h->cpy);
    else
      e = launch_copy_slab<double, float>((const double *)dst, ldad, (float *)W + q * ldw + q, ldw,
                                          n - q, w, true, h->cpy);
    GB_CUDA_TRY(e);
    if (q > 0)
      GB_CUDA_TRY(cudaMemset2DAsync((char *)W + q * ef, ldw * ef, 0, w * ef, q, h->cpy));
    GB_CUDA_TRY(cudaEventRecord(h->ev_in[(size_t)k], h->cpy));
  }
  h->cin.active = true;
  h->cin.s = s;
  return GB_OK;
}

gb_status factor_common(bool is_lu, gb_handle *h, int64_t n, int64_t s, gb_dtype dt,
                        const void *A, int64_t lda, void *L, int64_t ldl, int *info,
                        void *stream) {
  if (!h) return -1;
  if (n < 0) return -2;
  if (s < 0) return -3;
  if (!valid_dtype(dt)) return -4;
  if (n > 0 && !A) return -5;
  if (lda < std::max<int64_t>(1, n)) return -6;
  if (n > 0 && !L) return -7;
  if (ldl < std::max<int64_t>(1, n)) return -8;
  if (!info) return -9;
  if (n > (int64_t)1 << 30) return -2;
  DeviceGuard g(h->device);
  std::lock_guard<std::mutex> lk(h->mu);
  cudaStream_t st = (cudaStream_t)stream;
  // s = 0: the step gb_tune_step chose for this order, with its inner step
  // for this call only; else the default rule
  const int saved_inner = h->inner_step;
  struct RestoreInner {
    gb_handle *h;
    int v;
    ~RestoreInner() { h->inner_step = v; }
  } restore_inner{h, saved_inner};
  if (s == 0) {
    const auto t = tuned_step(h, is_lu ? 1 : 0, dt, n);
    if (t.s > 0) {
      s = t.s;
      h->inner_step = t.b;
    } else {
      s = default_step(dt, n);
    }
  }
  const size_t ein = elem_size_input(dt), ef = elem_size_factor(dt);
  const bool alias = (A == (const void *)L);
  if (alias && ein != ef) return -7;  // in place needs one element type

  InfoWord iw;
  gb_status r = iw.init(h, info, st);
  if (r != GB_OK) return r;
  if (n == 0) return iw.finish(st);

  // host input, Cholesky, right-looking loop, not in place: A goes in by
  // column slabs while the factorization starts (slab_copy_in)
  const bool left_mixed = !is_lu && is_mixed(dt) && h->left_looking && h->tc_update &&
                          split_of(dt) == 1 && s % 64 == 0 && s < n && n % 8 == 0;
  const bool stream_in = !is_lu && !left_mixed && !alias && !is_device_ptr(A) && h->cpy;
  Staged sa, sl;
  if (alias) {
    if ((r = sl.take(L, n, n, ldl, ef, true, true, st, h->stage_pool)) != GB_OK) return r;
    sa.dev = sl.dev;
    sa.ldd = sl.ldd;
  } else {
    if ((r = sa.take(A, n, n, lda, ein, !stream_in, false, st, h->stage_pool)) != GB_OK) return r;
    if ((r = sl.take(L, n, n, ldl, ef, false, true, st, h->stage_pool)) != GB_OK) return r;
  }
  const int64_t ld = sl.ldd;
  const bool lower_only = !is_lu;
  // host output, Cholesky, right-looking loop: stream the finished block
  // columns out during the factorization instead of copying L at the end
  struct CopyGuard {  // on any return: the staging buffers are freed on `st` after the copies
    gb_handle *h;
    cudaStream_t st;
    ~CopyGuard() {
      const bool copying = h->cin.active || h->cout.active;
      h->cin.active = false;
      h->cout.active = false;
      if (!copying) return;
      cudaEventRecord(h->ev_cpy, h->cpy);
      cudaStreamWaitEvent(st, h->ev_cpy, 0);
    }
  } copy_guard{h, st};
  if (!is_lu && !left_mixed && sl.host_dst && h->cpy) {
    h->cout = {true, sl.host_dst, ldl, sl.dev, ld, n, ef};
    GB_CUDA_TRY(cudaEventRecord(h->ev_cpy, st));  // the copy stream starts after the set-up
    GB_CUDA_TRY(cudaStreamWaitEvent(h->cpy, h->ev_cpy, 0));
  }
  std::unique_ptr<PhaseTimer> tcopy(new PhaseTimer(h, st, GB_PHASE_COPY, 0.0,
                                                   (double)n * n * (double)(ein + ef)));
  if (stream_in) {
    if ((r = slab_copy_in(h, dt, A, lda, sa.dev, sa.ldd, sl.dev, ld, n, s, st)) != GB_OK) return r;
  }
  switch (dt) {
    case GB_F64: {
      double *W = (double *)sl.dev;
      if (!stream_in)
        GB_CUDA_TRY((launch_copy_matrix<double, double>((const double *)sa.dev, sa.ldd, W, ld, n,
                                                        lower_only, st)));
      tcopy.reset();
      r = is_lu ? lu_blocked<double, double>(h, n, s, W, ld, iw.dev, dt, st)
                : chol_blocked<double, double>(h, n, s, W, ld, iw.dev, dt, st);
      break;
    }
    case GB_F32: {
      float *W = (float *)sl.dev;
      if (!stream_in)
        GB_CUDA_TRY((launch_copy_matrix<float, float>((const float *)sa.dev, sa.ldd, W, ld, n,
                                                      lower_only, st)));
      tcopy.reset();
      r = is_lu ? lu_blocked<float, float>(h, n, s, W, ld, iw.dev, dt, st)
                : chol_blocked<float, float>(h, n, s, W, ld, iw.dev, dt, st);
      break;
    }
    default: {  // mixed: FP64 in, FP32 working matrix, FP64 diagonal blocks
      float *W = (float *)sl.dev;
      if (!stream_in)
        GB_CUDA_TRY((launch_copy_matrix<double, float>((const double *)sa.dev, sa.ldd, W, ld, n,
                                                       lower_only, st)));
      tcopy.reset();
      const bool left = left_mixed;
      r = is_lu  ? lu_blocked<float, double>(h, n, s, W, ld, iw.dev, dt, st)
          : left ? chol_left_on<float, double>(h, n, s, W, ld, iw.dev, dt, st)
                 : chol_blocked<float, double>(h, n, s, W, ld, iw.dev, dt, st);
      break;
    }
  }
  if (r != GB_OK) return r;
  if (h->cout.active) {
    // while the device works: the zeros above each row's block column, in
    // the host buffer (the copy stream sends only rows from each block
    // column's first row down)
    const auto &c = h->cout;
    for (int64_t i = 0; i < n; ++i) {
      const int64_t j0 = (i / s + 1) * s;
      if (j0 < n) memset((char *)c.host + (i * c.ldh + j0) * c.esz, 0, (size_t)(n - j0) * c.esz);
    }
  }
  if (h->cout.active) {  // every block column went out on the copy stream
    h->cout.active = false;
    sl.host_dst = nullptr;
    GB_CUDA_TRY(cudaEventRecord(h->ev_cpy, h->cpy));
    GB_CUDA_TRY(cudaStreamWaitEvent(st, h->ev_cpy, 0));
  }
  if ((r = sl.finish()) != GB_OK) return r;
  if ((r = iw.finish(st)) != GB_OK) return r;
  if (sl.on_host() || sa.on_host()) GB_CUDA_TRY(cudaStreamSynchronize(st));
  return GB_OK;
}

// ------------------------------------------------------------------ solves
// L Y = B then L^T X = Y (Cholesky) or U X = Y (LU), through inverted
// diagonal blocks.  The inverses depend on the factor only: computed once per
// solve call and reused by every refinement step.
template <typename Tf>
struct SolvePlan {
  Tf *dinv_lo = nullptr;  // inverses of the diagonal blocks of L
  Tf *dinv_up = nullptr;  // of L^T (Cholesky) or of the unit U (LU)
  Tf *m_lo = nullptr;     // coupling blocks of the two sweeps
  Tf *m_up = nullptr;
};

template <typename Tf>
gb_status solve_prepare(gb_handle *h, bool is_lu, const Tf *F, int64_t ldf, int64_t n,
                        SolvePlan<Tf> &p, cudaStream_t st) {
  const size_t one = trsm_inv_bytes(n, sizeof(Tf));
  gb_status r = ws_reserve(h, WS_DINV, 4 * one, st);
  if (r != GB_OK) return r;
  char *base = (char *)h->ws[WS_DINV].ptr;
  p.dinv_lo = (Tf *)base;
  p.dinv_up = (Tf *)(base + one);
  p.m_lo = (Tf *)(base + 2 * one);
  p.m_up = (Tf *)(base + 3 * one);
  const int up = is_lu ? TRSM_UNIT_UPPER : TRSM_LOWER_T;
  GB_CUDA_TRY(launch_diag_inv<Tf>(F, ldf, n, TRSM_LOWER, p.dinv_lo, st));
  GB_CUDA_TRY(launch_diag_inv<Tf>(F, ldf, n, up, p.dinv_up, st));
  GB_CUDA_TRY(launch_coupling<Tf>(F, ldf, p.dinv_lo, n, TRSM_LOWER, p.m_lo, st));
  GB_CUDA_TRY(launch_coupling<Tf>(F, ldf, p.dinv_up, n, up, p.m_up, st));
  return GB_OK;
}

template <typename Tf>
gb_status tri_solve(gb_handle *h, bool is_lu, const Tf *F, int64_t ldf, const SolvePlan<Tf> &p,
                    double *X, int64_t ldx, int64_t n, int64_t nrhs, cudaStream_t st) {
  unsigned e1 = ++h->sync_epoch;
  if (e1 == 0) e1 = ++h->sync_epoch;
  GB_CUDA_TRY((launch_trsm_inv<Tf>(F, ldf, p.dinv_lo, p.m_lo, X, ldx, n, nrhs, TRSM_LOWER,
                                   h->d_sync, e1, h->d_err, h->spin_limit, st,
                                   h->test_withhold - 1)));
  unsigned e2 = ++h->sync_epoch;
  if (e2 == 0) e2 = ++h->sync_epoch;
  GB_CUDA_TRY((launch_trsm_inv<Tf>(F, ldf, p.dinv_up, p.m_up, X, ldx, n, nrhs,
                                   is_lu ? TRSM_UNIT_UPPER : TRSM_LOWER_T, h->d_sync, e2, h->d_err,
                                   h->spin_limit, st)));
  return GB_OK;
}

gb_status read_device_error(gb_handle *h, cudaStream_t st) {
  int err = 0;
  GB_CUDA_TRY(cudaMemcpyAsync(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  GB_CUDA_TRY(cudaStreamSynchronize(st));
  if (err) {
    GB_CUDA_TRY(cudaMemsetAsync(h->d_err, 0, sizeof(int), st));
    GB_CUDA_TRY(cudaStreamSynchronize(st));
    return (err & DEV_ERR_TIMEOUT) ? GB_ERR_TIMEOUT : GB_ERR_CUDA;
  }
  return GB_OK;
}

// The residual r = b - A x of refinement (GB_OPT_RESIDUAL): digit products
// on the tensor cores (residual_tc.cu) when chosen and its workspace can be
// had, else FP64 on the CUDA cores.  Both compute ||A||_inf into
// h->d_scalars[0] here, and per call the norms of r, x and b into
// h->d_scalars[1..3 nrhs].
bool split_residual(const gb_handle *h, int64_t n) {
  if (h->residual == 0 || n <= 0) return false;
  if (h->residual == 2 && n < SPLIT_RESIDUAL_MIN_N) return false;
  return tc_supported(h->device);
}

struct ResidualPlan {
  double *R = nullptr;       // n x nrhs (row-major, ld nrhs)
  void *work = nullptr;      // partial sums (FP64) or the digits of x (split)
  size_t work_bytes = 0;
  const void *awork = nullptr;  // the digits of A and row scales (split)
};

gb_status residual_prepare(gb_handle *h, const double *A, int64_t lda, int64_t n, int64_t nrhs,
                           ResidualPlan &rp, cudaStream_t st) {
  if ((size_t)(1 + 3 * nrhs) > 4096) return GB_ERR_UNSUPPORTED;
  if (split_residual(h, n) && ws_reserve(h, WS_SPLIT, split_a_bytes(n), st) == GB_OK)
    rp.awork = h->ws[WS_SPLIT].ptr;
  const size_t rbytes = ((size_t)n * nrhs * 8 + 255) / 256 * 256;
  rp.work_bytes = rp.awork ? split_x_bytes(n, nrhs, h->sm_count)
                           : residual_work_bytes(n, nrhs, h->sm_count);
  gb_status r = ws_reserve(h, WS_SOLVE, rbytes + rp.work_bytes, st);
  if (r != GB_OK) return r;
  rp.R = (double *)h->ws[WS_SOLVE].ptr;
  rp.work = rp.work_bytes ? (char *)h->ws[WS_SOLVE].ptr + rbytes : nullptr;
  double *norms = h->d_scalars;
  if (rp.awork) GB_CUDA_TRY(launch_split_a(A, lda, n, const_cast<void *>(rp.awork), norms, st));
  else GB_CUDA_TRY(launch_inf_norm_rows(A, lda, n, norms, st));
  return GB_OK;
}

gb_status residual_run(gb_handle *h, const ResidualPlan &rp, const double *A, int64_t lda,
                       const double *X, int64_t ldx, const double *B, int64_t ldb, int64_t n,
                       int64_t nrhs, cudaStream_t st) {
  double *norms = h->d_scalars + 1;
  if (rp.awork) {
    // a launch takes milliseconds; one second bounds every single wait
    const long long wait_ns = std::min<long long>((long long)h->spin_limit * 100LL, 1000000000LL);
    GB_CUDA_TRY(launch_residual_split(rp.awork, n, X, ldx, B, ldb, rp.R, nrhs, nrhs, norms,
                                      rp.work, h->sm_count, h->d_err, wait_ns, st));
  } else {
    GB_CUDA_TRY(launch_residual(A, lda, X, ldx, B, ldb, rp.R, nrhs, n, nrhs, norms,
                                (double *)rp.work, rp.work_bytes, h->sm_count, st));
  }
  return GB_OK;
}

template <typename Tf>
gb_status solve_common(bool is_lu, gb_handle *h, int64_t n, int64_t nrhs, const Tf *F,
                       int64_t ldf, const double *A, int64_t lda, const double *B, int64_t ldb,
                       double *X, int64_t ldx, const gb_refine_opts *opts, gb_solve_stats *stats,
                       cudaStream_t st) {
  const double tol = (opts && opts->tol > 0) ? opts->tol : 1e-14;
  const int max_iter = (opts && opts->max_iter >= 0) ? opts->max_iter : 30;
  if (stats) {
    stats->iterations = 0;
    stats->converged = 1;
    stats->eta = 0.0;
  }
  // a zero or non-finite pivot makes the substitutions meaningless
  GB_CUDA_TRY(launch_check_diag<Tf>(F, ldf, n, h->d_status, st));
  int bad = 0;
  GB_CUDA_TRY(cudaMemcpyAsync(&bad, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  GB_CUDA_TRY(cudaStreamSynchronize(st));
  if (bad) return GB_ERR_BREAKDOWN;

  if (X != B)
    GB_CUDA_TRY(cudaMemcpy2DAsync(X, ldx * 8, B, ldb * 8, nrhs * 8, n, cudaMemcpyDeviceToDevice, st));
  SolvePlan<Tf> plan;
  gb_status r = solve_prepare<Tf>(h, is_lu, F, ldf, n, plan, st);
  if (r != GB_OK) return r;
  r = tri_solve<Tf>(h, is_lu, F, ldf, plan, X, ldx, n, nrhs, st);
  if (r != GB_OK) return r;
  if (!A) return read_device_error(h, st);

  // iterative refinement in FP64
  ResidualPlan rp;
  if ((r = residual_prepare(h, A, lda, n, nrhs, rp, st)) != GB_OK) return r;
  double *R = rp.R;
  double *norms = h->d_scalars;  // [0]: ||A||_inf; [1..]: 3 * nrhs norms
  std::vector<double> hn(1 + 3 * nrhs);
  int it = 0;
  double eta = 0.0;
  for (;;) {
    if ((r = residual_run(h, rp, A, lda, X, ldx, B, ldb, n, nrhs, st)) != GB_OK) return r;
    GB_CUDA_TRY(cudaMemcpyAsync(hn.data(), norms, sizeof(double) * hn.size(),
                                cudaMemcpyDeviceToHost, st));
    int errw = 0;  // an expired device wait ends the refinement at once
    GB_CUDA_TRY(cudaMemcpyAsync(&errw, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    GB_CUDA_TRY(cudaStreamSynchronize(st));
    if (errw) {
      eta = INFINITY;
      break;
    }
    const double anorm = hn[0];
    eta = 0.0;
    for (int64_t c = 0; c < nrhs; ++c) {
      const double rn = hn[1 + c], xn = hn[1 + nrhs + c], bn = hn[1 + 2 * nrhs + c];
      const double den = anorm * xn + bn;
      double e = den > 0 ? rn / den : (rn > 0 ? INFINITY : 0.0);
      if (!std::isfinite(e) || !std::isfinite(den)) e = INFINITY;  // NaN/Inf: not converged
      if (e > eta) eta = e;
    }
    if (!std::isfinite(eta)) break;  // the iterate is lost; report non-convergence
    if (eta <= tol || it >= max_iter) break;
    if ((r = tri_solve<Tf>(h, is_lu, F, ldf, plan, R, nrhs, n, nrhs, st)) != GB_OK) return r;
    GB_CUDA_TRY(launch_axpy_cols(X, ldx, R, nrhs, n, nrhs, st));
    ++it;
  }
  if (stats) {
    stats->iterations = it;
    stats->eta = eta;
    stats->converged = eta <= tol ? 1 : 0;
  }
  if ((r = read_device_error(h, st)) != GB_OK) return r;
  return eta <= tol ? GB_OK : GB_ERR_NOT_CONVERGED;
}

gb_status solve_entry(bool is_lu, gb_handle *h, int64_t n, int64_t nrhs, gb_dtype factor_dt,
                      const void *F, int64_t ldf, const double *A, int64_t lda, const double *B,
                      int64_t ldb, double *X, int64_t ldx, const gb_refine_opts *opts,
                      gb_solve_stats *stats, void *stream) {
  if (!h) return -1;
  if (n < 0) return -2;
  if (nrhs < 0) return -3;
  if (!valid_dtype(factor_dt)) return -4;
  if (n > 0 && !F) return -5;
  if (ldf < std::max<int64_t>(1, n)) return -6;
  if (A && lda < std::max<int64_t>(1, n)) return -8;
  if (n > 0 && nrhs > 0 && !B) return -9;
  if (ldb < std::max<int64_t>(1, nrhs)) return -10;
  if (n > 0 && nrhs > 0 && !X) return -11;
  if (ldx < std::max<int64_t>(1, nrhs)) return -12;
  if (A && X == B) return -11;
  if (nrhs > 1365) return -3;  // norms scratch holds 3 * nrhs + 1 doubles
  DeviceGuard g(h->device);
  std::lock_guard<std::mutex> lk(h->mu);
  cudaStream_t st = (cudaStream_t)stream;
  if (stats) {
    stats->iterations = 0;
    stats->converged = 1;
    stats->eta = 0.0;
  }
  if (n == 0 || nrhs == 0) return GB_OK;
  const size_t ef = elem_size_factor(factor_dt);
  Staged sf, sa, sb, sx;
  gb_status r;
  if ((r = sf.take(F, n, n, ldf, ef, true, false, st, h->stage_pool)) != GB_OK) return r;
  if (A && (r = sa.take(A, n, n, lda, 8, true, false, st, h->stage_pool)) != GB_OK) return r;
  if (X == B) {
    if ((r = sx.take(X, n, nrhs, ldx, 8, true, true, st, h->stage_pool)) != GB_OK) return r;
    sb.dev = sx.dev;
    sb.ldd = sx.ldd;
  } else {
    if ((r = sb.take(B, n, nrhs, ldb, 8, true, false, st, h->stage_pool)) != GB_OK) return r;
    if ((r = sx.take(X, n, nrhs, ldx, 8, false, true, st, h->stage_pool)) != GB_OK) return r;
  }
  if (factor_dt == GB_F64)
    r = solve_common<double>(is_lu, h, n, nrhs, (const double *)sf.dev, sf.ldd,
                             (const double *)sa.dev, sa.ldd, (const double *)sb.dev, sb.ldd,
                             (double *)sx.dev, sx.ldd, opts, stats, st);
  else
    r = solve_common<float>(is_lu, h, n, nrhs, (const float *)sf.dev, sf.ldd,
                            (const double *)sa.dev, sa.ldd, (const double *)sb.dev, sb.ldd,
                            (double *)sx.dev, sx.ldd, opts, stats, st);
  if (r != GB_OK && r != GB_ERR_NOT_CONVERGED) return r;
  gb_status r2 = sx.finish();
  if (r2 != GB_OK) return r2;
  if (sx.on_host() || sf.on_host() || sa.on_host() || sb.on_host())
    GB_CUDA_TRY(cudaStreamSynchronize(st));
  return r;
}

}  // namespace
}  // namespace gb

using namespace gb;

// =================================================================== C ABI
extern "C" {

const char *gb_status_string(gb_status st) {
  switch (st) {
    case GB_OK: return "success";
    case GB_ERR_NOMEM: return "allocation failed";
    case GB_ERR_CUDA: return "CUDA runtime error";
    case GB_ERR_TIMEOUT: return "bounded device wait expired";
    case GB_ERR_NOT_CONVERGED: return "iterative refinement did not reach the tolerance";
    case GB_ERR_REJECTED: return "request rejected: footprint exceeds the budget";
    case GB_ERR_UNSUPPORTED: return "unsupported combination of options";
    case GB_ERR_BREAKDOWN: return "factor has a zero or non-finite pivot";
    case GB_ERR_STATE: return "object used in the wrong state";
    default: return st < 0 && st > -100 ? "invalid argument" : "unknown status";
  }
}

int gb_version(void) { return 100; }

const char *gb_last_error(void) { return gb::last_error_message(); }

gb_status gb_create(gb_handle **out, int device) {
  if (!out) return -1;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return GB_ERR_CUDA;
  }
  DeviceGuard g(device);
  gb_handle *h = new (std::nothrow) gb_handle();
  if (!h) return GB_ERR_NOMEM;
  h->device = device;
  cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, device);
  bool ok = cudaMalloc(&h->d_status, sizeof(int)) == cudaSuccess &&
            cudaMalloc(&h->d_err, sizeof(int)) == cudaSuccess &&
            cudaMalloc(&h->d_sync, sizeof(int) * SYNC_WORDS) == cudaSuccess &&
            cudaMalloc(&h->d_scalars, sizeof(double) * 4096) == cudaSuccess &&
            cudaMalloc(&h->d_arrivals, sizeof(unsigned long long)) == cudaSuccess;
  if (ok)
    ok = cudaMemset(h->d_status, 0, sizeof(int)) == cudaSuccess &&
         cudaMemset(h->d_err, 0, sizeof(int)) == cudaSuccess &&
         cudaMemset(h->d_sync, 0, sizeof(int) * SYNC_WORDS) == cudaSuccess &&
         cudaMemset(h->d_arrivals, 0, sizeof(unsigned long long)) == cudaSuccess &&
         cudaDeviceSynchronize() == cudaSuccess;
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  if (ok)
    ok = cudaStreamCreateWithPriority(&h->hi, cudaStreamNonBlocking, prio_hi) == cudaSuccess &&
         cudaStreamCreateWithPriority(&h->aux, cudaStreamNonBlocking, prio_lo) == cudaSuccess &&
         cudaEventCreateWithFlags(&h->ev_next, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&h->ev_rest, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) == cudaSuccess &&
         cudaStreamCreateWithFlags(&h->cpy, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&h->ev_cpy, cudaEventDisableTiming) == cudaSuccess &&
         cudaStreamCreateWithPriority(&h->aux2, cudaStreamNonBlocking, prio_hi) == cudaSuccess &&
         cudaEventCreateWithFlags(&h->ev_ip, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&h->ev_ir, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    gb_destroy(h);
    return GB_ERR_NOMEM;
  }
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = device;
  if (cudaMemPoolCreate(&h->stage_pool, &props) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;  // never trim at synchronisation points
    cudaMemPoolSetAttribute(h->stage_pool, cudaMemPoolAttrReleaseThreshold, &keep);
  } else {
    cudaGetLastError();
    h->stage_pool = nullptr;  // staging falls back to the device's default pool
  }
  *out = h;
  return GB_OK;
}

gb_status gb_destroy(gb_handle *h) {
  if (!h) return GB_OK;
  DeviceGuard g(h->device);
  cudaDeviceSynchronize();
  for (auto &r : h->prof_pending) {
    if (r.owns_start) cudaEventDestroy(r.start);
    cudaEventDestroy(r.stop);
  }
  for (auto e : h->prof_pool) cudaEventDestroy(e);
  for (auto &w : h->ws)
    if (w.ptr) cudaFree(w.ptr);
  if (h->d_status) cudaFree(h->d_status);
  if (h->d_err) cudaFree(h->d_err);
  if (h->d_sync) cudaFree(h->d_sync);
  if (h->d_scalars) cudaFree(h->d_scalars);
  if (h->d_arrivals) cudaFree(h->d_arrivals);
  if (h->ev_next) cudaEventDestroy(h->ev_next);
  if (h->ev_rest) cudaEventDestroy(h->ev_rest);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->ev_cpy) cudaEventDestroy(h->ev_cpy);
  if (h->ev_ip) cudaEventDestroy(h->ev_ip);
  if (h->ev_ir) cudaEventDestroy(h->ev_ir);
  if (h->aux2) cudaStreamDestroy(h->aux2);
  for (cudaEvent_t e : h->ev_in) cudaEventDestroy(e);
  if (h->cpy) cudaStreamDestroy(h->cpy);
  if (h->hi) cudaStreamDestroy(h->hi);
  if (h->aux) cudaStreamDestroy(h->aux);
  if (h->stage_pool) cudaMemPoolDestroy(h->stage_pool);
  delete h;
  return GB_OK;
}

gb_status gb_set_option(gb_handle *h, gb_option opt, int64_t v) {
  if (!h) return -1;
  switch (opt) {
    case GB_OPT_INNER_STEP:
      if (v < 1 || v > 64) return -3;
      h->inner_step = (int)v;
      return GB_OK;
    case GB_OPT_USE_GRAPHS: h->use_graphs = v ? 1 : 0; return GB_OK;
    case GB_OPT_TC_UPDATE:
      if (v < 0 || v > 2) return -3;
      h->tc_update = (int)v;
      return GB_OK;
    case GB_OPT_SPIN_LIMIT:
      if (v < 1) return -3;
      h->spin_limit = v;
      return GB_OK;
    case GB_OPT_PROFILE: h->profile = v ? 1 : 0; return GB_OK;
    case GB_OPT_BATCHED_EXACT: h->batched_exact = v ? 1 : 0; return GB_OK;
    case GB_OPT_LOOKAHEAD: h->lookahead = v ? 1 : 0; return GB_OK;
    case GB_OPT_STRASSEN: h->strassen = v ? 1 : 0; return GB_OK;
    case GB_OPT_QR_INNER_STEP:
      if (v < 1 || v > 256) return -3;
      h->qr_inner = (int)v;
      return GB_OK;
    case GB_OPT_LEFT_LOOKING: h->left_looking = v ? 1 : 0; return GB_OK;
    case GB_OPT_TEST_WITHHOLD:
      if (v < 0 || v > (int64_t)1 << 30) return -3;
      h->test_withhold = (int)v;
      return GB_OK;
    case GB_OPT_INNER_CUDA_CORES: h->inner_cuda_cores = v ? 1 : 0; return GB_OK;
    case GB_OPT_INNER_RECURSIVE:
      if (v < 0 || v > 2) return -3;
      h->inner_recursive = (int)v;
      return GB_OK;
    case GB_OPT_INNER_LOOKAHEAD:
      if (v < 0 || v > 2) return -3;
      h->inner_lookahead = (int)v;
      return GB_OK;
    case GB_OPT_EARLY_REST:
      if (v < 0 || v > 2) return -3;
      h->early_rest = (int)v;
      return GB_OK;
    case GB_OPT_RESIDUAL:
      if (v < 0 || v > 2) return -3;
      h->residual = (int)v;
      return GB_OK;
    case GB_OPT_F64_UPDATE:
      if (v < 0 || v > 1) return -3;
      h->f64_update = (int)v;
      return GB_OK;
    default: return -2;
  }
}

gb_status gb_get_option(gb_handle *h, gb_option opt, int64_t *v) {
  if (!h) return -1;
  if (!v) return -3;
  switch (opt) {
    case GB_OPT_INNER_STEP: *v = h->inner_step; return GB_OK;
    case GB_OPT_USE_GRAPHS: *v = h->use_graphs; return GB_OK;
    case GB_OPT_TC_UPDATE: *v = h->tc_update; return GB_OK;
    case GB_OPT_SPIN_LIMIT: *v = h->spin_limit; return GB_OK;
    case GB_OPT_PROFILE: *v = h->profile; return GB_OK;
    case GB_OPT_BATCHED_EXACT: *v = h->batched_exact; return GB_OK;
    case GB_OPT_LOOKAHEAD: *v = h->lookahead; return GB_OK;
    case GB_OPT_STRASSEN: *v = h->strassen; return GB_OK;
    case GB_OPT_QR_INNER_STEP: *v = h->qr_inner; return GB_OK;
    case GB_OPT_LEFT_LOOKING: *v = h->left_looking; return GB_OK;
    case GB_OPT_TEST_WITHHOLD: *v = h->test_withhold; return GB_OK;
    case GB_OPT_INNER_CUDA_CORES: *v = h->inner_cuda_cores; return GB_OK;
    case GB_OPT_INNER_RECURSIVE: *v = h->inner_recursive; return GB_OK;
    case GB_OPT_INNER_LOOKAHEAD: *v = h->inner_lookahead; return GB_OK;
    case GB_OPT_EARLY_REST: *v = h->early_rest; return GB_OK;
    case GB_OPT_RESIDUAL: *v = h->residual; return GB_OK;
    case GB_OPT_F64_UPDATE: *v = h->f64_update; return GB_OK;
    default: return -2;
  }
}

gb_status gb_chol_factor(gb_handle *h, int64_t n, int64_t s, gb_dtype dt, const void *A,
                         int64_t lda, void *L, int64_t ldl, int *info, void *stream) {
  return factor_common(false, h, n, s, dt, A, lda, L, ldl, info, stream);
}

gb_status gb_lu_factor(gb_handle *h, int64_t n, int64_t s, gb_dtype dt, const void *A,
                       int64_t lda, void *LU, int64_t ldlu, int *info, void *stream) {
  return factor_common(true, h, n, s, dt, A, lda, LU, ldlu, info, stream);
}

gb_status gb_qr_factor(gb_handle *h, int64_t n, int64_t s, gb_dtype dt, const void *A,
                       int64_t lda, void *Q, int64_t ldq, void *R, int64_t ldr, int *info,
                       void *stream) {
  return qr_common(h, n, s, dt, A, lda, Q, ldq, R, ldr, info, stream);
}

gb_status gb_chol_solve(gb_handle *h, int64_t n, int64_t nrhs, gb_dtype factor_dt, const void *L,
                        int64_t ldl, const double *A, int64_t lda, const double *B, int64_t ldb,
                        double *X, int64_t ldx, const gb_refine_opts *opts,
                        gb_solve_stats *stats, void *stream) {
  return solve_entry(false, h, n, nrhs, factor_dt, L, ldl, A, lda, B, ldb, X, ldx, opts, stats,
                     stream);
}

gb_status gb_lu_solve(gb_handle *h, int64_t n, int64_t nrhs, gb_dtype factor_dt, const void *LU,
                      int64_t ldlu, const double *A, int64_t lda, const double *B, int64_t ldb,
                      double *X, int64_t ldx, const gb_refine_opts *opts, gb_solve_stats *stats,
                      void *stream) {
  return solve_entry(true, h, n, nrhs, factor_dt, LU, ldlu, A, lda, B, ldb, X, ldx, opts, stats,
                     stream);
}

gb_status gb_backward_error(gb_handle *h, int is_lu, int64_t n, gb_dtype factor_dt,
                            const double *A, int64_t lda, const void *F, int64_t ldf,
                            double *out, void *stream) {
  if (!h) return -1;
  if (n < 0) return -3;
  if (!valid_dtype(factor_dt)) return -4;
  if (n > 0 && !A) return -5;
  if (lda < std::max<int64_t>(1, n)) return -6;
  if (n > 0 && !F) return -7;
  if (ldf < std::max<int64_t>(1, n)) return -8;
  if (!out) return -9;
  if (n > 0 && (!is_device_ptr(A) || !is_device_ptr(F))) return -5;
  DeviceGuard g(h->device);
  std::lock_guard<std::mutex> lk(h->mu);
  cudaStream_t st = (cudaStream_t)stream;
  *out = 0.0;
  if (n == 0) return GB_OK;
  if (factor_dt == GB_F64)
    GB_CUDA_TRY(launch_backward_error<double>(is_lu, A, lda, (const double *)F, ldf, n,
                                              h->d_scalars, st));
  else
    GB_CUDA_TRY(launch_backward_error<float>(is_lu, A, lda, (const float *)F, ldf, n,
                                             h->d_scalars, st));
  double acc[2];
  GB_CUDA_TRY(cudaMemcpyAsync(acc, h->d_scalars, sizeof acc, cudaMemcpyDeviceToHost, st));
  GB_CUDA_TRY(cudaStreamSynchronize(st));
  *out = acc[1] > 0 ? std::sqrt(acc[0] / acc[1]) : 0.0;
  return GB_OK;
}

gb_status gb_residual(gb_handle *h, int64_t n, int64_t nrhs, const double *A, int64_t lda,
                      const double *X, int64_t ldx, const double *B, int64_t ldb, double *R,
                      int64_t ldr, double *eta, void *stream) {
  if (!h) return -1;
  if (n < 0) return -2;
  if (nrhs < 0 || nrhs > 1365) return -3;
  if (n > 0 && (!A || !is_device_ptr(A))) return -4;
  if (lda < std::max<int64_t>(1, n)) return -5;
  const bool work = n > 0 && nrhs > 0;
  if (work && (!X || !is_device_ptr(X))) return -6;
  if (ldx < std::max<int64_t>(1, nrhs)) return -7;
  if (work && (!B || !is_device_ptr(B))) return -8;
  if (ldb < std::max<int64_t>(1, nrhs)) return -9;
  if (work && (!R || !is_device_ptr(R))) return -10;
  if (ldr < std::max<int64_t>(1, nrhs)) return -11;
  DeviceGuard g(h->device);
  std::lock_guard<std::mutex> lk(h->mu);
  cudaStream_t st = (cudaStream_t)stream;
  if (eta) *eta = 0.0;
  if (!work) return GB_OK;
  ResidualPlan rp;
  gb_status r = residual_prepare(h, A, lda, n, nrhs, rp, st);
  if (r != GB_OK) return r;
  if ((r = residual_run(h, rp, A, lda, X, ldx, B, ldb, n, nrhs, st)) != GB_OK) return r;
  GB_CUDA_TRY(cudaMemcpy2DAsync(R, ldr * 8, rp.R, nrhs * 8, nrhs * 8, n, cudaMemcpyDeviceToDevice,
                                st));
  std::vector<double> hn(1 + 3 * nrhs);
  GB_CUDA_TRY(cudaMemcpyAsync(hn.data(), h->d_scalars, sizeof(double) * hn.size(),
                              cudaMemcpyDeviceToHost, st));
  if ((r = read_device_error(h, st)) != GB_OK) return r;
  if (eta) {
    double e = 0.0;
    for (int64_t c = 0; c < nrhs; ++c) {
      const double den = hn[0] * hn[1 + nrhs + c] + hn[1 + 2 * nrhs + c];
      double ec = den > 0 ? hn[1 + c] / den : (hn[1 + c] > 0 ? INFINITY : 0.0);
      if (!std::isfinite(ec) || !std::isfinite(den)) ec = INFINITY;
      e = std::max(e, ec);
    }
    *eta = e;
  }
  return GB_OK;
}

}  // extern "C"

namespace gb {
namespace {

// Step for a matrix of order n when the caller passes s = 0: the tuned
// bucket entry if gb_batched_tune ran, else a rule measured on GB300
// (small orders: Crout-like wide steps are latency-bound; 32 balances the
// column steps against the delayed update).
int batched_default_step(const gb_handle *h, int dtype_index, int n) {
  const int b = std::min(BATCH_BUCKETS - 1, std::max(0, (n - 1) / 32));
  const int t = h->batched_step[dtype_index][b];
  if (t > 0) return t;
  return n <= 32 ? n : 32;
}

// Build the plan (LPT order, steps) on the host and upload it into the
// handle's batched workspace; remembered in h->plan.
gb_status batched_upload(gb_handle *h, int64_t count, const int64_t *n, void *const *A,
                         const int64_t *lda, void *const *L, const int64_t *ldl, gb_dtype dt,
                         const int *steps, cudaStream_t st, int lu = 0) {
  const int di = dt == GB_F64 ? 0 : 1;
  std::vector<int> order((size_t)count), nn((size_t)count), ss((size_t)count);
  for (int64_t i = 0; i < count; ++i) {
    order[i] = (int)i;
    nn[i] = (int)n[i];
    // the tuned table is Cholesky's; LU takes the default rule
    ss[i] = steps ? steps[i] : lu ? std::min((int)n[i], 32) : batched_default_step(h, di, (int)n[i]);
  }
  // longest processing time first: orders by n^3, descending
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return nn[a] > nn[b]; });
  const size_t c = (size_t)count;
  const size_t off_n = c * 4, off_s = 2 * c * 4, off_a = ((3 * c * 4 + 15) / 16) * 16;
  const size_t off_la = off_a + c * 8, off_l = off_la + c * 8, off_ll = off_l + c * 8;
  const size_t off_t = off_ll + c * 8, total = off_t + 16;
  std::vector<unsigned char> blob(total, 0);
  memcpy(blob.data(), order.data(), c * 4);
  memcpy(blob.data() + off_n, nn.data(), c * 4);
  memcpy(blob.data() + off_s, ss.data(), c * 4);
  memcpy(blob.data() + off_a, A, c * 8);
  memcpy(blob.data() + off_la, lda, c * 8);
  memcpy(blob.data() + off_l, L, c * 8);
  memcpy(blob.data() + off_ll, ldl, c * 8);
  gb_status r = ws_reserve(h, WS_MISC, total, st);
  if (r != GB_OK) return r;
  unsigned char *d = (unsigned char *)h->ws[WS_MISC].ptr;
  GB_CUDA_TRY(cudaMemcpyAsync(d, blob.data(), total, cudaMemcpyHostToDevice, st));
  GB_CUDA_TRY(cudaStreamSynchronize(st));  // the host blob goes out of scope
  auto &p = h->plan;
  p.count = (int)count;
  p.dt = dt;
  p.order = (const int *)d;
  p.n = (const int *)(d + off_n);
  p.step = (const int *)(d + off_s);
  p.A = (void *const *)(d + off_a);
  p.lda = (const int64_t *)(d + off_la);
  p.L = (void *const *)(d + off_l);
  p.ldl = (const int64_t *)(d + off_ll);
  p.ticket = (int *)(d + off_t);
  p.lu = lu;
  return GB_OK;
}

// Launch the persistent kernel over the uploaded plan (capturable).
gb_status batched_launch(gb_handle *h, int *info_dev, cudaStream_t st) {
  const auto &p = h->plan;
  if (p.count <= 0) return GB_OK;
  if (p.lu) {
    if (p.dt == GB_F64)
      GB_CUDA_TRY(launch_lu_batched_plan<double>(p.count, p.order, p.n, p.step, p.A, p.lda, p.L,
                                                 p.ldl, info_dev, p.ticket, h->sm_count,
                                                 h->batched_exact, st));
    else
      GB_CUDA_TRY(launch_lu_batched_plan<float>(p.count, p.order, p.n, p.step, p.A, p.lda, p.L,
                                                p.ldl, info_dev, p.ticket, h->sm_count,
                                                h->batched_exact, st));
    return GB_OK;
  }
  if (p.dt == GB_F64)
    GB_CUDA_TRY(launch_chol_batched_plan<double>(p.count, p.order, p.n, p.step, p.A, p.lda, p.L,
                                                 p.ldl, info_dev, p.ticket, h->sm_count,
                                                 h->batched_exact, st));
  else
    GB_CUDA_TRY(launch_chol_batched_plan<float>(p.count, p.order, p.n, p.step, p.A, p.lda, p.L,
                                                p.ldl, info_dev, p.ticket, h->sm_count,
                                                h->batched_exact, st));
  return GB_OK;
}

gb_status batched_check(gb_handle *h, int64_t count, const int64_t *n, void *const *A,
                        const int64_t *lda, void *const *L, const int64_t *ldl, gb_dtype dt,
                        int64_t s) {
  if (!h) return -1;
  if (count < 0 || count > (1 << 26)) return -2;
  if (count > 0 && !n) return -3;
  if (count > 0 && !A) return -4;
  if (count > 0 && !lda) return -5;
  if (count > 0 && !L) return -6;
  if (count > 0 && !ldl) return -7;
  if (dt != GB_F64 && dt != GB_F32) return -8;
  if (s < 0) return -9;
  for (int64_t i = 0; i < count; ++i) {
    if (n[i] < 0 || n[i] > BATCH_MAX_N) return -3;
    if (lda[i] < std::max<int64_t>(1, n[i])) return -5;
    if (ldl[i] < std::max<int64_t>(1, n[i])) return -7;
    if (n[i] > 0 && (!A[i] || !is_device_ptr(A[i]))) return -4;
    if (n[i] > 0 && (!L[i] || !is_device_ptr(L[i]))) return -6;
  }
  return GB_OK;
}

}  // namespace
}  // namespace gb

namespace gb {
namespace {

gb_status batched_plan_common(gb_handle *h, int64_t count, const int64_t *n, void *const *A,
                              const int64_t *lda, void *const *L, const int64_t *ldl, gb_dtype dt,
                              int64_t s, void *stream, int lu) {
  gb_status r = batched_check(h, count, n, A, lda, L, ldl, dt, s);
  if (r != GB_OK) return r;
  DeviceGuard g(h->device);
  std::lock_guard<std::mutex> lk(h->mu);
  std::vector<int> steps;
  if (s > 0) steps.assign((size_t)count, (int)std::min<int64_t>(s, 1 << 20));
  if (count == 0) {
    h->plan = gb_handle::BatchPlanDev{};
    return GB_OK;
  }
  return batched_upload(h, count, n, A, lda, L, ldl, dt, s > 0 ? steps.data() : nullptr,
                        (cudaStream_t)stream, lu);
}

gb_status factor_batched_common(gb_handle *h, int64_t count, const int64_t *n, void *const *A,
                                const int64_t *lda, void *const *L, const int64_t *ldl,
                                gb_dtype dt, int64_t s, int *info, void *stream, int lu) {
  gb_status r = batched_check(h, count, n, A, lda, L, ldl, dt, s);
  if (r != GB_OK) return r;
  if (count > 0 && !info) return -10;
  if (count == 0) return GB_OK;
  DeviceGuard g(h->device);
  std::lock_guard<std::mutex> lk(h->mu);
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int> steps;
  if (s > 0) steps.assign((size_t)count, (int)std::min<int64_t>(s, 1 << 20));
  if ((r = batched_upload(h, count, n, A, lda, L, ldl, dt, s > 0 ? steps.data() : nullptr, st,
                          lu)) != GB_OK)
    return r;
  int *info_dev = info;
  int *info_scratch = nullptr;
  const bool host_info = !is_device_ptr(info);
  if (host_info) {
    if (cudaMallocAsync((void **)&info_scratch, sizeof(int) * count, st) != cudaSuccess) {
      cudaGetLastError();
      return GB_ERR_NOMEM;
    }
    info_dev = info_scratch;
  }
  r = batched_launch(h, info_dev, st);
  if (r == GB_OK && host_info) {
    if (cudaMemcpyAsync(info, info_scratch, sizeof(int) * count, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      r = GB_ERR_CUDA;
  }
  if (info_scratch) cudaFreeAsync(info_scratch, st);
  return r;
}

}  // namespace
}  // namespace gb

extern "C" gb_status gb_batched_plan(gb_handle *h, int64_t count, const int64_t *n,
                                     void *const *A, const int64_t *lda, void *const *L,
                                     const int64_t *ldl, gb_dtype dt, int64_t s, void *stream) {
  return batched_plan_common(h, count, n, A, lda, L, ldl, dt, s, stream, 0);
}

extern "C" gb_status gb_lu_batched_plan(gb_handle *h, int64_t count, const int64_t *n,
                                        void *const *A, const int64_t *lda, void *const *LU,
                                        const int64_t *ldlu, gb_dtype dt, int64_t s,
                                        void *stream) {
  return batched_plan_common(h, count, n, A, lda, LU, ldlu, dt, s, stream, 1);
}

extern "C" gb_status gb_batched_run(gb_handle *h, int *info, void *stream) {
  if (!h) return -1;
  if (h->plan.count > 0 && !info) return -2;
  if (h->plan.count > 0 && !is_device_ptr(info)) return -2;
  DeviceGuard g(h->device);
  std::lock_guard<std::mutex> lk(h->mu);
  return batched_launch(h, info, (cudaStream_t)stream);
}

extern "C" gb_status gb_chol_factor_batched(gb_handle *h, int64_t count, const int64_t *n,
                                            void *const *A, const int64_t *lda, void *const *L,
                                            const int64_t *ldl, gb_dtype dt, int64_t s, int *info,
                                            void *stream) {
  return factor_batched_common(h, count, n, A, lda, L, ldl, dt, s, info, stream, 0);
}

extern "C" gb_status gb_lu_factor_batched(gb_handle *h, int64_t count, const int64_t *n,
                                          void *const *A, const int64_t *lda, void *const *LU,
                                          const int64_t *ldlu, gb_dtype dt, int64_t s, int *info,
                                          void *stream) {
  return factor_batched_common(h, count, n, A, lda, LU, ldlu, dt, s, info, stream, 1);
}

extern "C" gb_status gb_batched_tune(gb_handle *h, gb_dtype dt, int64_t n_max, int *steps_out,
                                     void *stream) {
  if (!h) return -1;
  if (dt != GB_F64 && dt != GB_F32) return -2;
  if (n_max < 1 || n_max > BATCH_MAX_N) return -3;
  DeviceGuard g(h->device);
  cudaStream_t st = (cudaStream_t)stream;
  const int di = dt == GB_F64 ? 0 : 1;
  const size_t esz = dt == GB_F64 ? 8 : 4;
  const int per = 2 * std::max(1, h->sm_count);  // two waves of matrices per bucket
  const int nb = (int)((n_max + 31) / 32);
  const int cand[] = {8, 16, 32, 48, 64, 96, 128};
  void *buf = nullptr;
  const int64_t stride = (int64_t)n_max * n_max;
  if (cudaMalloc(&buf, (size_t)per * stride * esz) != cudaSuccess) {
    cudaGetLastError();
    return GB_ERR_NOMEM;
  }
  int *info = nullptr;
  if (cudaMalloc((void **)&info, sizeof(int) * per) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(buf);
    return GB_ERR_NOMEM;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  gb_status r = GB_OK;
  std::vector<int64_t> nv(per), lv(per);
  std::vector<void *> pv(per);
  std::vector<int> sv(per);
  for (int b = 0; b < nb && r == GB_OK; ++b) {
    const int n = std::min<int>((int)n_max, 32 * b + 24);  // representative order of the bucket
    float best = 1e30f;
    int best_s = 32;
    for (int c : cand) {
      if (c > n && c != cand[0]) break;
      for (int i = 0; i < per; ++i) {
        nv[i] = n;
        lv[i] = n;
        pv[i] = (char *)buf + (size_t)i * stride * esz;
        sv[i] = std::min(c, n);
      }
      for (int rep = 0; rep < 2 && r == GB_OK; ++rep) {  // rep 0 warms up
        cudaError_t e = dt == GB_F64 ? launch_fill_spd<double>((double *)buf, stride, per, n, st)
                                     : launch_fill_spd<float>((float *)buf, stride, per, n, st);
        if (e != cudaSuccess) {
          record_cuda_error(e, "fill_spd", __FILE__, __LINE__);
          r = GB_ERR_CUDA;
          break;
        }
        {
          std::lock_guard<std::mutex> lk(h->mu);
          r = batched_upload(h, per, nv.data(), pv.data(), lv.data(), pv.data(), lv.data(), dt,
                             sv.data(), st);
          if (r == GB_OK) {
            cudaEventRecord(e0, st);
            r = batched_launch(h, info, st);
            cudaEventRecord(e1, st);
          }
        }
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep == 1 && ms < best) {
          best = ms;
          best_s = sv[0];
        }
      }
    }
    h->batched_step[di][b] = best_s;
    if (steps_out) steps_out[b] = best_s;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(st);
  cudaFree(info);
  cudaFree(buf);
  return r;
}

extern "C" gb_status gb_tune_step(gb_handle *h, int kind, gb_dtype dt, int64_t n, int64_t *s_out,
                                  int64_t *b_out, void *stream) {
  if (!h) return -1;
  if (kind < 0 || kind > 2) return -2;
  if (!valid_dtype(dt)) return -3;
  if (kind == 2 && dt != GB_F64 && dt != GB_F32) return GB_ERR_UNSUPPORTED;
  if (n < 2 || n > 65536) return -4;
  DeviceGuard g(h->device);
  cudaStream_t st = (cudaStream_t)stream;
  const size_t ein = elem_size_input(dt), ef = kind == 2 ? ein : elem_size_factor(dt);
  const size_t nn = (size_t)n * (size_t)n;
  void *A = nullptr, *F = nullptr, *R = nullptr;
  int *info = nullptr;
  gb_status r = GB_OK;
  if (cudaMalloc(&A, nn * ein) != cudaSuccess || cudaMalloc(&F, nn * ef) != cudaSuccess ||
      (kind == 2 && cudaMalloc(&R, nn * ef) != cudaSuccess) ||
      cudaMalloc((void **)&info, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    r = GB_ERR_NOMEM;
  }
  // the test matrix n I + ones: symmetric positive definite, every leading
  // minor positive, full rank
  if (r == GB_OK) {
    const cudaError_t e = ein == 8 ? launch_fill_spd<double>((double *)A, (int64_t)nn, 1, (int)n, st)
                                   : launch_fill_spd<float>((float *)A, (int64_t)nn, 1, (int)n, st);
    if (e != cudaSuccess) {
      record_cuda_error(e, "fill_spd", __FILE__, __LINE__);
      r = GB_ERR_CUDA;
    }
  }
  const int64_t steps[] = {32, 64, 128, 256, 512, 1024};
  const int inner_chol[] = {16, 32, 64}, inner_qr[] = {8, 16, 32};
  const int *inner = kind == 2 ? inner_qr : inner_chol;
  int &knob = kind == 2 ? h->qr_inner : h->inner_step;
  int saved;
  {
    std::lock_guard<std::mutex> lk(h->mu);
    saved = knob;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int64_t best_s = 0;
  int best_b = 0;
  for (int64_t s : steps) {
    if (r != GB_OK) break;
    if (s >= n && s != steps[0]) break;
    for (int bi = 0; bi < 3 && r == GB_OK; ++bi) {
      const int b = inner[bi];
      if (b > s) continue;
      {
        std::lock_guard<std::mutex> lk(h->mu);
        knob = b;
      }
      float ms = 0;
      for (int rep = 0; rep < 2 && r == GB_OK; ++rep) {  // rep 0 warms up
        cudaEventRecord(e0, st);
        if (kind == 0)
          r = gb_chol_factor(h, n, s, dt, A, n, F, n, info, stream);
        else if (kind == 1)
          r = gb_lu_factor(h, n, s, dt, A, n, F, n, info, stream);
        else
          r = gb_qr_factor(h, n, s, dt, A, n, F, n, R, n, info, stream);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
          cudaGetLastError();
          r = GB_ERR_CUDA;
        }
        cudaEventElapsedTime(&ms, e0, e1);
      }
      int host_info = 0;
      if (r == GB_OK && cudaMemcpy(&host_info, info, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        r = GB_ERR_CUDA;
      // steps ascend: a larger step must be 3% faster to replace a smaller
      // one (the smaller step is at least as accurate, and for the mixed
      // dtypes a less accurate factor can cost a refinement step)
      const float need = (best_s == 0 || best_s == s) ? best : 0.97f * best;
      if (r == GB_OK && host_info == 0 && ms < need) {
        best = ms;
        best_s = s;
        best_b = b;
      }
    }
  }
  {
    std::lock_guard<std::mutex> lk(h->mu);
    knob = saved;
    if (r == GB_OK && best_s > 0) h->tuned[kind][dt][tune_bucket(n)] = {best_s, best_b};
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(A);
  cudaFree(F);
  if (R) cudaFree(R);
  if (info) cudaFree(info);
  if (r == GB_OK && best_s == 0) r = GB_ERR_BREAKDOWN;
  if (r == GB_OK) {
    if (s_out) *s_out = best_s;
    if (b_out) *b_out = best_b;
  }
  return r;
}

extern "C" uint64_t gb_kernel_launches(void) { return gb::g_launches.load(); }

extern "C" gb_status gb_profile_read(gb_handle *h, gb_profile *out) {
  if (!h) return -1;
  if (!out) return -2;
  DeviceGuard g(h->device);
  std::lock_guard<std::mutex> lk(h->mu);
  gb_status r = GB_OK;
  for (auto &rec : h->prof_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(rec.stop) != cudaSuccess ||
        cudaEventElapsedTime(&ms, rec.start, rec.stop) != cudaSuccess) {
      cudaGetLastError();
      r = GB_ERR_CUDA;
    }
    if (rec.phase >= 0 && rec.phase < GB_NUM_PHASES) {
      out->launches[rec.phase] += 1;
      out->ms[rec.phase] += ms;
      out->flops[rec.phase] += rec.flops;
      out->bytes[rec.phase] += rec.bytes;
    }
    if (rec.owns_start) h->prof_pool.push_back(rec.start);
    h->prof_pool.push_back(rec.stop);
  }
  h->prof_pending.clear();
  return r;
}

extern "C" gb_status gb_rank_update(gb_handle *h, gb_dtype dt, int lower, int y_is_kxn, int64_t M,
                                    int64_t N, int64_t K, void *C, int64_t ldc, const void *X,
                                    int64_t ldx, const void *Y, int64_t ldy, void *stream) {
  if (!h) return -1;
  if (!valid_dtype(dt)) return -2;
  if (M < 0) return -5;
  if (N < 0) return -6;
  if (K < 0) return -7;
  if (M > 0 && N > 0 && !C) return -8;
  if (ldc < std::max<int64_t>(1, N)) return -9;
  if (M > 0 && K > 0 && !X) return -10;
  if (ldx < std::max<int64_t>(1, K)) return -11;
  if (N > 0 && K > 0 && !Y) return -12;
  if (ldy < std::max<int64_t>(1, y_is_kxn ? N : K)) return -13;
  if (M == 0 || N == 0 || K == 0) return GB_OK;
  DeviceGuard g(h->device);
  std::lock_guard<std::mutex> lk(h->mu);
  cudaStream_t st = (cudaStream_t)stream;
  const bool nn = y_is_kxn != 0;
  int *status = h->d_status;
  GB_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), st));
  if (dt == GB_F64 && h->f64_update == 1 && tc_supported(h->device)) {
    const bool same = !nn && X == Y && ldx == ldy && N <= M;
    gb_status r = ws_reserve(h, WS_PANEL, update_digits_bytes(M, N, K, same), st);
    if (r != GB_OK) return r;
    GB_CUDA_TRY(launch_update_digits((double *)C, ldc, (const double *)X, ldx, (const double *)Y,
                                     ldy, M, N, K, lower != 0, nn, status, h->d_err,
                                     h->spin_limit, h->ws[WS_PANEL].ptr, h->ws[WS_PANEL].bytes,
                                     h->sm_count, st));
  } else if (dt == GB_F64 && !lower) {
    gb_status r = general_update<double>(h, (double *)C, ldc, (const double *)X, ldx,
                                         (const double *)Y, ldy, M, N, K, nn, status, WS_STRAS, st);
    if (r != GB_OK) return r;
  } else if (dt == GB_F32 && !lower) {
    gb_status r = general_update<float>(h, (float *)C, ldc, (const float *)X, ldx,
                                        (const float *)Y, ldy, M, N, K, nn, status, WS_STRAS, st);
    if (r != GB_OK) return r;
  } else if (dt == GB_F64) {
    GB_CUDA_TRY(launch_update_simt<double>((double *)C, ldc, (const double *)X, ldx,
                                           (const double *)Y, ldy, M, N, K, nn, lower != 0, 0,
                                           status, st));
  } else if (dt == GB_F32) {
    GB_CUDA_TRY(launch_update_simt<float>((float *)C, ldc, (const float *)X, ldx,
                                          (const float *)Y, ldy, M, N, K, nn, lower != 0, 0,
                                          status, st));
  } else {
    TcUpdateArgs a{};
    a.C = (float *)C;
    a.ldc = ldc;
    a.X = (const float *)X;
    a.ldx = ldx;
    a.Y = (const float *)Y;
    a.ldy = ldy;
    a.M = M;
    a.N = N;
    a.K = K;
    a.nn = nn;
    a.lower = lower != 0;
    a.diag = 0;
    a.f16 = dt == GB_MIX_F16;
    a.split = split_of(dt);
    a.status = status;
    a.err = h->d_err;
    a.spin_limit = h->spin_limit;
    a.cluster = h->tc_update;
    gb_status r = ws_reserve(h, WS_PANEL, tc_pack_bytes(M, N, K, nn, split_of(dt)), st);
    if (r != GB_OK) return r;
    a.pack = h->ws[WS_PANEL].ptr;
    a.pack_bytes = h->ws[WS_PANEL].bytes;
    // under the profile option: packing timed as GB_PHASE_COPY, the
    // tensor-core kernel as GB_PHASE_UPDATE
    cudaEvent_t e0 = nullptr, e2 = nullptr;
    if (h->profile) {
      e0 = take_event(h);
      a.packed = take_event(h);
      e2 = take_event(h);
      if (!e0 || !a.packed || !e2) {
        for (cudaEvent_t ev : {e0, a.packed, e2})
          if (ev) h->prof_pool.push_back(ev);
        e0 = e2 = a.packed = nullptr;
      } else {
        cudaEventRecord(e0, st);
      }
    }
    cudaError_t e = launch_update_tc(a, st);
    if (e0 && e != cudaSuccess) {
      for (cudaEvent_t ev : {e0, a.packed, e2}) h->prof_pool.push_back(ev);
    } else if (e0) {
      cudaEventRecord(e2, st);
      // FP32 rows read once, 16-bit planes written; C read and written once
      const double planes = (double)split_of(dt);
      const double rows = (double)(M + (a.X == a.Y && !nn && M == N ? 0 : N));
      const double cells = lower ? lower_count(M, N, 0) : (double)M * N;
      h->prof_pending.push_back({GB_PHASE_COPY, e0, a.packed, 0.0, (4.0 + 2.0 * planes) * rows * K});
      h->prof_pending.push_back({GB_PHASE_UPDATE, a.packed, e2, update_flops(M, N, K, lower != 0),
                                 8.0 * cells + 2.0 * planes * (double)(M + N) * K, false});
    }
    if (e == cudaErrorNotSupported) return GB_ERR_UNSUPPORTED;
    GB_CUDA_TRY(e);
  }
  return GB_OK;
}
