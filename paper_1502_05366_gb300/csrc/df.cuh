// Double-float arithmetic on the FP32 pipe: every value is the unevaluated
// sum hi + lo of two floats (about 48 significant bits).  Sums use TwoSum
// (Knuth), products TwoProduct by fma (Dekker 1971), dot products the
// compensated scheme Dot2 (Ogita, Rump & Oishi 2005).  The rounding primitives
// use the _rn intrinsics so that no product is fused into a neighbouring sum.
// Shared by the pivoted-QR kernels of the FP32 path.
#pragma once
#include <cstdint>

namespace rsvd {

__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}
// |a| >= |b| or a == 0
__device__ __forceinline__ void df_fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ double df_to_d(float h, float l) { return (double)h + (double)l; }
// (a_h + a_l) + (b_h + b_l) as a normalised pair.
__device__ __forceinline__ void df_add(float ah, float al, float bh, float bl, float& h, float& l) {
  float s, e;
  df_two_sum(ah, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(al, bl));
  df_fast_two_sum(s, e, h, l);
}
// (a_h + a_l)(b_h + b_l) as a normalised pair (the a_l b_l term dropped).
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float& h, float& l) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  df_fast_two_sum(p, e, h, l);
}
// sqrt of a positive pair: y = sqrtf(a_h), one Newton step y + (a - y^2) / (2y)
// with the residual a - y^2 formed exactly (TwoProduct).
__device__ __forceinline__ void df_sqrt(float ah, float al, float& h, float& l) {
  const float y = sqrtf(ah);
  const float yy = __fmul_rn(y, y);
  const float ye = __fmaf_rn(y, y, -yy);
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(ah, yy), ye), al);
  const float c = __fdiv_rn(r, __fmul_rn(2.f, y));
  df_fast_two_sum(y, c, h, l);
}
// 1 / (b_h + b_l): y = 1 / b_h, one Newton step y + y (1 - b y) with 1 - b y
// formed from the exact product b_h y.
__device__ __forceinline__ void df_recip(float bh, float bl, float& h, float& l) {
  const float y = __frcp_rn(bh);
  const float p = __fmul_rn(bh, y);
  const float pe = __fmaf_rn(bh, y, -p);
  const float r = __fsub_rn(__fsub_rn(__fsub_rn(1.f, p), pe), __fmul_rn(bl, y));
  df_fast_two_sum(y, __fmul_rn(y, r), h, l);
}
// Warp sum of double-float partial sums (s, e): TwoSum on the leading parts,
// errors accumulated; every lane ends with the total.
__device__ __forceinline__ void df_warp_sum(float& s, float& e) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float os = __shfl_xor_sync(0xffffffffu, s, o);
    const float oe = __shfl_xor_sync(0xffffffffu, e, o);
    float t;
    df_two_sum(s, os, s, t);
    e = __fadd_rn(e, __fadd_rn(oe, t));
  }
}
__device__ __forceinline__ void d_to_df(double x, float& h, float& l) {
  h = __double2float_rn(x);
  l = __double2float_rn(x - (double)h);
}

// Residual norms as double-float pairs with a total order (hi, then lo); a
// pivoted column has hi = -1.  All comparisons and norm updates of the
// double-float kernel run on the FP32 pipe.
struct DF {
  float h, l;
};
__device__ __forceinline__ bool df_gt(DF x, DF y) { return x.h > y.h || (x.h == y.h && x.l > y.l); }
__device__ __forceinline__ bool df_eq(DF x, DF y) { return x.h == y.h && x.l == y.l; }
struct Top2F {
  DF b1;
  int64_t i1;
  DF b2;
};
__device__ __forceinline__ Top2F merge_top2f(Top2F x, Top2F y) {
  const bool xfirst = df_gt(x.b1, y.b1) || (df_eq(x.b1, y.b1) && x.i1 < y.i1);
  const Top2F& f = xfirst ? x : y;
  const Top2F& o = xfirst ? y : x;
  Top2F r;
  r.b1 = f.b1;
  r.i1 = f.i1;
  r.b2 = df_gt(f.b2, o.b1) ? f.b2 : o.b1;
  return r;
}
// Double-float square x^2 of a pair.
__device__ __forceinline__ void df_sqr(float xh, float xl, float& ph, float& pe) {
  ph = __fmul_rn(xh, xh);
  pe = __fmaf_rn(xh, xh, -ph);
  pe = __fmaf_rn(2.0f * xh, xl, pe);
}
// Dot2 accumulation of x^2 into (s, e).
__device__ __forceinline__ void df_acc_sqr(float xh, float xl, float& s, float& e) {
  float ph, pe, t;
  df_sqr(xh, xl, ph, pe);
  df_two_sum(s, ph, s, t);
  e = __fadd_rn(e, __fadd_rn(t, pe));
}


}  // namespace rsvd
