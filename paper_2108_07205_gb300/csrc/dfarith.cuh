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

}  // namespace rw
