// Double-FP32 arithmetic: an FP64 number a held as the FP32 pair (hi, lo) =
// (fl32(a), fl32(a - hi)).  A multiply-add forms the product of two pairs from
// FP32 operations with its rounding error (the exact error of hi * hi by one
// FMA, the cross terms hi * lo by FMAs) and adds it to a running pair (s, c)
// by two-sum (Knuth): s takes the rounded sum, c the exact rounding errors and
// the cross terms.  The _rn intrinsics keep the compiler from contracting or
// reordering these steps.
#pragma once
#include <cuda_runtime.h>

namespace rw {

__device__ __forceinline__ void df_mac(float& s, float& c, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  const float e = __fmaf_rn(ah, bh, -p);
  const float t = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, e));
  const float s1 = __fadd_rn(s, p);
  const float bb = __fsub_rn(s1, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(s1, bb)), __fsub_rn(p, bb));
  s = s1;
  c = __fadd_rn(c, __fadd_rn(err, t));
}

// (H, L) += (s + c): two-sum of the running pair with a chunk's sum; the
// chunk accumulators restart at zero.
__device__ __forceinline__ void df_flush(float& H, float& L, float& s, float& c) {
  const float h1 = __fadd_rn(H, s);
  const float bb = __fsub_rn(h1, H);
  const float err = __fadd_rn(__fsub_rn(H, __fsub_rn(h1, bb)), __fsub_rn(s, bb));
  H = h1;
  L = __fadd_rn(L, __fadd_rn(err, c));
  s = 0.f;
  c = 0.f;
}

// FP64 value -> (hi, lo) pair.
__device__ __forceinline__ void df_split(double v, float& h, float& l) {
  h = __double2float_rn(v);
  l = __double2float_rn(v - double(h));
}

// The same split from the bit pattern, with integer operations only (this
// part's FP64 units run at 1/64 of its FP32 rate, so a conversion and a
// subtraction in FP64 per staged entry would cost as much as the products):
// hi = v with its significand truncated to 24 bits, lo = the remaining 29
// bits truncated to 24, so |v - hi - lo| <= 2^-47 |v|.  Values whose
// pieces would leave FP32's normal range take the FP64 route.
__device__ __forceinline__ void df_split_bits(double v, float& h, float& l) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
  if ((b << 1) == 0ull) {  // +-0 (padding): no FP64 work
    h = l = 0.f;
    return;
  }
  const int e = int((b >> 52) & 0x7FF);
  if (e < 950 || e > 1150) {
    df_split(v, h, l);
    return;
  }
  const unsigned sign = static_cast<unsigned>(b >> 63) << 31;
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  h = __uint_as_float(sign | (static_cast<unsigned>(e - 896) << 23) | static_cast<unsigned>(m >> 29));
  const unsigned long long r = m & 0x1FFFFFFFull;
  if (r == 0) {
    l = 0.f;
    return;
  }
  const int p = 63 - __clzll(static_cast<long long>(r));  // leading bit of the rest, 0..28
  const unsigned frac = p >= 23 ? static_cast<unsigned>((r >> (p - 23)) & 0x7FFFFF)
                                : static_cast<unsigned>((r << (23 - p)) & 0x7FFFFF);
  l = __uint_as_float(sign | (static_cast<unsigned>(e - 948 + p) << 23) | frac);
}

// FP32 -> FP64 by its bit pattern (exact), the FP64 conversion only for
// zero, subnormals, infinities and NaN.
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xFF;
  if (ex == 0 || ex == 255) return (u << 1) == 0u ? __longlong_as_double(static_cast<long long>(u >> 31) << 63) : double(f);
  const unsigned long long b = (static_cast<unsigned long long>(u >> 31) << 63) |
                               (static_cast<unsigned long long>(ex + 896) << 52) |
                               (static_cast<unsigned long long>(u & 0x7FFFFF) << 29);
  return __longlong_as_double(static_cast<long long>(b));
}

}  // namespace rw
