// Double-word ("double-float") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits.  On GB300 a dependent FP64 FMA takes ~400 cycles
// and an FP64 sqrt or divide ~650, while an FP32 FMA takes ~4.5: the
// latency-bound inner loops of the factorisations (Jacobi rotations,
// Householder reflectors) run several times faster in double-word arithmetic,
// whose ~2^-48 relative precision is far inside the 1e-10 the results are
// held to.  FP64 stays at the boundary: inputs are split on load, outputs
// recombined on store.
//
// Building blocks (each written from its published description):
//   two_sum       Knuth, TAOCP vol. 2, 4.2.2: s + e = a + b exactly.
//   fast_two_sum  Dekker (1971): the same when |a| >= |b|.
//   two_prod      exact product with one FMA: p + e = a b.
//   dw_add        Joldes, Muller & Popescu (2017), "Tight and rigorous error
//                 bounds for basic building blocks of double-word
//                 arithmetic", the accurate DW + DW sum (relative error
//                 <= 3 u^2).
//   dw_mul        same paper, DW x DW with FMA (relative error <= 5 u^2).
//   dw_mul_f      DW x float with FMA.
//   dw_dot_step   one step of the compensated dot product of Ogita, Rump &
//                 Oishi (2005) ("Dot2"): the high parts are accumulated with
//                 two_sum, every rounding error in a plain float sum.
// The compiler must not contract or reassociate these sequences: they use
// explicit fmaf where a fused operation is meant and no fast-math flags.
#pragma once

#include <cuda_runtime.h>

namespace vp {

struct dw {
  float hi, lo;
};

__device__ __forceinline__ dw two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}

__device__ __forceinline__ dw fast_two_sum(float a, float b) {
  const float s = a + b;
  const float e = b - (s - a);
  return {s, e};
}

__device__ __forceinline__ dw two_prod(float a, float b) {
  const float p = a * b;
  const float e = fmaf(a, b, -p);
  return {p, e};
}

__device__ __forceinline__ dw dw_add(dw x, dw y) {
  const dw s = two_sum(x.hi, y.hi);
  const dw t = two_sum(x.lo, y.lo);
  const float c = s.lo + t.hi;
  const dw v = fast_two_sum(s.hi, c);
  const float w = t.lo + v.lo;
  return fast_two_sum(v.hi, w);
}

__device__ __forceinline__ dw dw_neg(dw x) { return {-x.hi, -x.lo}; }

__device__ __forceinline__ dw dw_mul(dw x, dw y) {
  const dw c = two_prod(x.hi, y.hi);
  const float tl0 = x.lo * y.lo;
  const float tl1 = fmaf(x.hi, y.lo, tl0);
  const float cl2 = fmaf(x.lo, y.hi, tl1);
  const float cl3 = c.lo + cl2;
  return fast_two_sum(c.hi, cl3);
}

__device__ __forceinline__ dw dw_mul_f(dw x, float y) {
  const dw c = two_prod(x.hi, y);
  const float cl3 = fmaf(x.lo, y, c.lo);
  return fast_two_sum(c.hi, cl3);
}

// FP64 <-> DW.  The split is exact to the 48 bits a DW holds.
__device__ __forceinline__ dw dw_from(double x) {
  const float hi = __double2float_rn(x);
  const float lo = __double2float_rn(x - (double)hi);
  return {hi, lo};
}
__device__ __forceinline__ double dw_to(dw x) { return (double)x.hi + (double)x.lo; }

// Compensated dot-product accumulator (Dot2): s + c approximates the sum.
struct dw_acc {
  float s = 0.f, c = 0.f;
};
__device__ __forceinline__ void dw_dot_step(dw_acc& a, dw x, dw y) {
  const dw p = two_prod(x.hi, y.hi);
  const float cross = fmaf(x.hi, y.lo, x.lo * y.hi);
  const dw t = two_sum(a.s, p.hi);
  a.s = t.hi;
  a.c += t.lo + (p.lo + cross);
}
__device__ __forceinline__ dw dw_acc_value(const dw_acc& a) { return fast_two_sum(a.s, a.c); }

// Warp sum of DW values: two_sum on the high parts, the errors and low parts
// in a float, renormalised at the end.
__device__ __forceinline__ dw dw_warp_sum(dw v) {
  float s = v.hi, c = v.lo;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
    const float c2 = __shfl_xor_sync(0xffffffffu, c, o);
    const dw t = two_sum(s, s2);
    s = t.hi;
    c = c + c2 + t.lo;
  }
  return fast_two_sum(s, c);
}

// 1 / sqrt(x) for x > 0 to DW accuracy: FP32 seed and one Newton step
// y <- y + y (1 - x y^2) / 2 evaluated in DW (the correction is small, so
// its own rounding is of order u^2).
__device__ __forceinline__ dw dw_rsqrt(dw x) {
  const float y0 = rsqrtf(x.hi);
  const dw y2 = two_prod(y0, y0);
  const dw xy2 = dw_mul(x, y2);
  const dw r = dw_add({1.0f, 0.0f}, dw_neg(xy2));  // 1 - x y0^2, of order u
  const float corr = 0.5f * y0 * r.hi;
  return fast_two_sum(y0, corr);
}

// sqrt(x) for x >= 0: FP32 root y0, then y0 + (x - y0^2) / (2 y0) with the
// residual x - y0^2 formed in DW (Newton's step for y^2 = x).
__device__ __forceinline__ dw dw_sqrt(dw x) {
  if (!(x.hi > 0.f)) return {0.f, 0.f};
  const float y0 = sqrtf(x.hi);
  const dw r = dw_add(x, dw_neg(two_prod(y0, y0)));
  return fast_two_sum(y0, r.hi / (2.0f * y0));
}

// a / b: FP32 quotient q0, then one step of long division on the DW
// remainder a - q0 b.
__device__ __forceinline__ dw dw_div(dw a, dw b) {
  const float q0 = a.hi / b.hi;
  const dw r = dw_add(a, dw_neg(dw_mul_f(b, q0)));
  return fast_two_sum(q0, r.hi / b.hi);
}

// x * 2^e for a DW value (exact unless the low part leaves the FP32 range).
__device__ __forceinline__ dw dw_ldexp(dw x, int e) { return {ldexpf(x.hi, e), ldexpf(x.lo, e)}; }

}  // namespace vp
