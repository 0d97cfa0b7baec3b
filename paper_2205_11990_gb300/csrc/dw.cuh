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

// x * 2^e for a DW value (exact unless the low part leaves the FP32 range).
__device__ __forceinline__ dw dw_ldexp(dw x, int e) { return {ldexpf(x.hi, e), ldexpf(x.lo, e)}; }

// Lane-strided loops over rows i = i0 + lane, i0 + lane + 32, ... < m, in
// batches of four rows per lane: the four loads are issued before any
// arithmetic and the four stores after it, so that the dependent chains of
// four rows overlap (the compiler cannot reorder the loads of one row past
// the store of another through shared-memory pointers).  The accumulation
// order of each lane is unchanged (rows ascending), so results are identical
// to the plain loop.
__device__ __forceinline__ void dw_dot_rows(dw_acc& acc, const dw* __restrict__ a, const dw* __restrict__ b, int i0,
                                            int m, int lane) {
  int i = i0 + lane;
  for (; i + 96 < m; i += 128) {
    const dw a0 = a[i], a1 = a[i + 32], a2 = a[i + 64], a3 = a[i + 96];
    const dw b0 = b[i], b1 = b[i + 32], b2 = b[i + 64], b3 = b[i + 96];
    dw_dot_step(acc, a0, b0);
    dw_dot_step(acc, a1, b1);
    dw_dot_step(acc, a2, b2);
    dw_dot_step(acc, a3, b3);
  }
  for (; i < m; i += 32) dw_dot_step(acc, a[i], b[i]);
}

// c[i] <- c[i] - w v[i] over the same rows.
__device__ __forceinline__ void dw_axpy_rows(dw* c, const dw* v, dw w, int i0, int m, int lane) {
  int i = i0 + lane;
  for (; i + 96 < m; i += 128) {
    const dw c0 = c[i], c1 = c[i + 32], c2 = c[i + 64], c3 = c[i + 96];
    const dw v0 = v[i], v1 = v[i + 32], v2 = v[i + 64], v3 = v[i + 96];
    const dw r0 = dw_add(c0, dw_neg(dw_mul(w, v0)));
    const dw r1 = dw_add(c1, dw_neg(dw_mul(w, v1)));
    const dw r2 = dw_add(c2, dw_neg(dw_mul(w, v2)));
    const dw r3 = dw_add(c3, dw_neg(dw_mul(w, v3)));
    c[i] = r0;
    c[i + 32] = r1;
    c[i + 64] = r2;
    c[i + 96] = r3;
  }
  for (; i < m; i += 32) c[i] = dw_add(c[i], dw_neg(dw_mul(w, v[i])));
}

// Sum of squares of x[i] 2^-e over the rows (the same steps as a
// dw_dot_step of each scaled value with itself).
__device__ __forceinline__ void dw_sumsq_rows(dw_acc& acc, const dw* __restrict__ x, int e, int i0, int m, int lane) {
  int i = i0 + lane;
  for (; i + 96 < m; i += 128) {
    const dw x0 = dw_ldexp(x[i], -e), x1 = dw_ldexp(x[i + 32], -e), x2 = dw_ldexp(x[i + 64], -e),
             x3 = dw_ldexp(x[i + 96], -e);
    dw_dot_step(acc, x0, x0);
    dw_dot_step(acc, x1, x1);
    dw_dot_step(acc, x2, x2);
    dw_dot_step(acc, x3, x3);
  }
  for (; i < m; i += 32) {
    const dw x0 = dw_ldexp(x[i], -e);
    dw_dot_step(acc, x0, x0);
  }
}

// x[i] <- (x[i] 2^-e) s over the rows.
__device__ __forceinline__ void dw_scale_rows(dw* x, int e, dw s, int i0, int m, int lane) {
  int i = i0 + lane;
  for (; i + 96 < m; i += 128) {
    const dw x0 = x[i], x1 = x[i + 32], x2 = x[i + 64], x3 = x[i + 96];
    x[i] = dw_mul(dw_ldexp(x0, -e), s);
    x[i + 32] = dw_mul(dw_ldexp(x1, -e), s);
    x[i + 64] = dw_mul(dw_ldexp(x2, -e), s);
    x[i + 96] = dw_mul(dw_ldexp(x3, -e), s);
  }
  for (; i < m; i += 32) x[i] = dw_mul(dw_ldexp(x[i], -e), s);
}

// max |x[i].hi| over the rows (one lane's part).
__device__ __forceinline__ float dw_absmax_rows(const dw* x, int i0, int m, int lane) {
  float mx = 0.f;
  int i = i0 + lane;
  for (; i + 96 < m; i += 128)
    mx = fmaxf(fmaxf(fmaxf(mx, fabsf(x[i].hi)), fmaxf(fabsf(x[i + 32].hi), fabsf(x[i + 64].hi))), fabsf(x[i + 96].hi));
  for (; i < m; i += 32) mx = fmaxf(mx, fabsf(x[i].hi));
  return mx;
}

// Plane rotation of two rows over q < m: (u, v) <- (c u - s v, s u + c v),
// four columns per lane per batch (loads first, stores last).
__device__ __forceinline__ void dw_rot_rows(dw* ri, dw* rj, dw cs, dw sn, int m, int lane) {
  int q = lane;
  for (; q + 96 < m; q += 128) {
    const dw u0 = ri[q], u1 = ri[q + 32], u2 = ri[q + 64], u3 = ri[q + 96];
    const dw v0 = rj[q], v1 = rj[q + 32], v2 = rj[q + 64], v3 = rj[q + 96];
    ri[q] = dw_add(dw_mul(cs, u0), dw_neg(dw_mul(sn, v0)));
    rj[q] = dw_add(dw_mul(sn, u0), dw_mul(cs, v0));
    ri[q + 32] = dw_add(dw_mul(cs, u1), dw_neg(dw_mul(sn, v1)));
    rj[q + 32] = dw_add(dw_mul(sn, u1), dw_mul(cs, v1));
    ri[q + 64] = dw_add(dw_mul(cs, u2), dw_neg(dw_mul(sn, v2)));
    rj[q + 64] = dw_add(dw_mul(sn, u2), dw_mul(cs, v2));
    ri[q + 96] = dw_add(dw_mul(cs, u3), dw_neg(dw_mul(sn, v3)));
    rj[q + 96] = dw_add(dw_mul(sn, u3), dw_mul(cs, v3));
  }
  for (; q < m; q += 32) {
    const dw u = ri[q], v = rj[q];
    ri[q] = dw_add(dw_mul(cs, u), dw_neg(dw_mul(sn, v)));
    rj[q] = dw_add(dw_mul(sn, u), dw_mul(cs, v));
  }
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


}  // namespace vp
