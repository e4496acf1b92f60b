// Exact digits of FP64 values for products on the tensor cores (the
// refinement residual in residual_tc.cu, the FP64-accurate delayed update in
// update_digits.cu).  A row (or column) of values is scaled by 2^e, e the
// binary exponent of its largest magnitude, and each value's fixed-point
// word floor(|v| 2^(55 - e)) is cut into RP digits of RW bits, each stored
// exactly as a BF16 integer with the value's sign.  Digit p weighs
// 2^(-RW (p + 1)).  Only integer operations and one packed BF16
// subtraction per two digits: nothing runs on the FP64 pipe.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gb {
namespace dg {

constexpr int RW = 5;    // bits per digit
constexpr int RP = 11;   // digits: 55 fractional bits

static __device__ __forceinline__ double finite_abs_r(double v) {
  const double a = fabs(v);
  return a <= 1.7976931348623157e308 ? a : __longlong_as_double(0x7ff0000000000000LL);
}
static __device__ __forceinline__ void atomic_max_nonneg_r(double *addr, double v) {
  atomicMax(reinterpret_cast<long long *>(addr), __double_as_longlong(v));
}
// binary exponent e with m <= 2^e for the largest magnitude m of a row or
// column (m = 0 or non-finite: 0)
static __device__ __forceinline__ int scale_exp(double m) {
  if (!(m > 0.0) || !(m <= 1.7976931348623157e308)) return 0;
  int e;
  frexp(m, &e);  // m = f 2^e, f in [0.5, 1)
  return e;
}

// The 55-bit fixed-point word floor(|v| 2^(55 - e)) of v (|v| < 2^e) and
// its sign as a BF16 sign bit; a non-finite v sets `bad`.
static __device__ __forceinline__ unsigned long long fixed_of(double v, int e, uint32_t &sgn, bool &bad) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  sgn = (uint32_t)(bits >> 48) & 0x8000u;
  const int ex = (int)((bits >> 52) & 0x7ff);
  bad = ex == 0x7ff;
  if (ex == 0) return 0ull;  // zero and subnormals (far below the 2^-55 truncation)
  const unsigned long long m = ((bits & 0xfffffffffffffull) | (1ull << 52)) << 2;
  // |v| 2^(55 - e) = m 2^(ex - 1022 - e) with m = significand x 4; the
  // exponent is <= 0 whenever |v| < 2^e
  const int r = 1022 + e - ex;
  return r <= 0 ? m : (r < 64 ? m >> r : 0ull);
}

// Digits p of two values as one word of two BF16 bit patterns (low half:
// the first): digit p = bits [55 - RW (p+1), 60 - RW (p+1)) of the fixed-
// point word.  128 + d (d < 128) has the BF16 pattern 0x4300 | d, so one
// packed BF16 subtraction of 128 gives both digits exactly; the signs are
// then or-ed in (a zero digit may carry a sign: -0 adds nothing).
template <int P>
static __device__ __forceinline__ uint32_t digit_pair(unsigned long long wa, unsigned long long wb,
                                               uint32_t signs) {
  constexpr int k = RW * (RP - 1 - P);
  const uint32_t da = (uint32_t)(wa >> k) & ((1u << RW) - 1u);
  const uint32_t db = (uint32_t)(wb >> k) & ((1u << RW) - 1u);
  uint32_t word = da | (db << 16) | 0x43004300u;
  __nv_bfloat162 x = *reinterpret_cast<__nv_bfloat162 *>(&word);
  x = __hsub2(x, __nv_bfloat162(__float2bfloat16_rn(128.0f), __float2bfloat16_rn(128.0f)));
  return *reinterpret_cast<uint32_t *>(&x) | signs;
}

template <int P>
static __device__ __forceinline__ void digit_pairs(unsigned long long wa, unsigned long long wb,
                                            uint32_t signs, uint32_t nan_mask,
                                            uint32_t (&out)[RP]) {
  out[P] = digit_pair<P>(wa, wb, signs);
  if (P == 0) out[0] |= nan_mask;  // a non-finite value: a NaN digit
  if constexpr (P + 1 < RP) digit_pairs<P + 1>(wa, wb, signs, nan_mask, out);
}

// Digit planes of two values (v, w): out[p] = the two BF16 digits p.
static __device__ __forceinline__ void digits2(double v, double w, int e, uint32_t (&out)[RP]) {
  uint32_t sa, sb;
  bool ba, bb;
  const unsigned long long wa = fixed_of(v, e, sa, ba);
  const unsigned long long wb = fixed_of(w, e, sb, bb);
  const uint32_t nan_mask = (ba ? 0x7fc0u : 0u) | (bb ? 0x7fc00000u : 0u);
  digit_pairs<0>(wa, wb, sa | (sb << 16), nan_mask, out);
}

static __device__ __forceinline__ double pow2_neg(int k) {  // 2^-k, 0 <= k < 1000
  return __longlong_as_double((long long)(1023 - k) << 52);
}

}  // namespace dg
}  // namespace gb
