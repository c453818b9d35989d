// Double-float arithmetic for the products with the inverse factor S.
//
// A value is carried as the unevaluated sum hi + lo of two floats (Dekker
// 1971). The products with S run on the FP32 pipe with error-free
// transformations: a product of two such values takes the exact product of
// the high parts through one FMA (p = hi*hi rounded, e = fma(hi, hi, -p)
// exactly), adds the two cross terms, and drops lo*lo (relative size 2^-48);
// sums take Knuth's branch-free TwoSum. A dot product accumulated this way
// carries about twice the FP32 precision (relative error of order 2^-44 per
// term against the sum of magnitudes) at a fraction of the cost of FP64 FMAs,
// whose rate on this part is 2 per clock per SM. Every operation is an
// explicitly rounded intrinsic, so the compiler neither contracts nor
// reorders them. Values must stay inside the FP32 range (|x| < 3e38).
#pragma once
#include <cuda_runtime.h>

namespace pdk {

__device__ __forceinline__ float2 df_split(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}

__device__ __forceinline__ double df_join(float2 a) { return (double)a.x + (double)a.y; }

// (h, l) += s * x
__device__ __forceinline__ void df_mac(float& h, float& l, float2 s, float2 x) {
  const float p = __fmul_rn(s.x, x.x);
  const float e = __fmaf_rn(s.x, x.x, -p);                          // s.x * x.x - p, exact
  const float t = __fmaf_rn(s.x, x.y, __fmaf_rn(s.y, x.x, e));       // cross terms + e
  const float sum = __fadd_rn(h, p);                                  // TwoSum(h, p)
  const float bb = __fsub_rn(sum, h);
  const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(sum, bb)), __fsub_rn(p, bb));
  h = sum;
  l = __fadd_rn(l, __fadd_rn(err, t));
}

// a + b, renormalised so that |lo| <= ulp(hi) / 2
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  const float s = __fadd_rn(a.x, b.x);
  const float bb = __fsub_rn(s, a.x);
  const float err = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));
  const float l = __fadd_rn(err, __fadd_rn(a.y, b.y));
  const float h = __fadd_rn(s, l);                                    // Fast2Sum(s, l): |s| >= |l| or s = 0
  return make_float2(h, __fsub_rn(l, __fsub_rn(h, s)));
}

// a + x for a plain float x (TwoSum of the high part, then renormalised)
__device__ __forceinline__ float2 df_add_f(float2 a, float x) {
  const float s = __fadd_rn(a.x, x);
  const float bb = __fsub_rn(s, a.x);
  const float err = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(x, bb));
  const float l = __fadd_rn(a.y, err);
  const float h = __fadd_rn(s, l);
  return make_float2(h, __fsub_rn(l, __fsub_rn(h, s)));
}

__device__ __forceinline__ float2 df_shfl_xor(float2 a, int o) {
  return make_float2(__shfl_xor_sync(0xffffffffu, a.x, o), __shfl_xor_sync(0xffffffffu, a.y, o));
}

// warp-wide sum, identical in every lane (TwoSum is exact, hence symmetric)
__device__ __forceinline__ float2 df_warp_sum(float2 a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a = df_add(a, df_shfl_xor(a, o));
  return a;
}

}  // namespace pdk
