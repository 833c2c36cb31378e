// Double-float ("dd") values: a real held as the unevaluated sum hi + lo of two FP32 numbers
// with |lo| <= ulp(hi)/2, about 48 significant bits, evaluated with FP32 instructions only.
// GB300 runs FP64 arithmetic at a small fraction of its FP32 rate, so the batched columns'
// FP64-accuracy finishing phase can run in dd instead (no counterpart in the paper).
//
// The error-free transformations are the classical ones: TwoSum (Knuth, TAOCP vol. 2,
// 4.2.2), FastTwoSum (Dekker 1971, for |a| >= |b|) and TwoProduct with a fused multiply-add
// (the rounding error of a*b is fma(a, b, -a*b) exactly). On these, addition follows the
// "sloppy" double-double sum (one TwoSum of the high parts, the low parts added, one
// renormalisation), multiplication the FMA product with the cross terms folded in, and
// division and square root one Newton correction of an FP32 first guess (Karp and
// Markstein 1997 for the square root). Relative error per operation ~2^-46 (the sum's
// error is bounded by 2^-46 (|a| + |b|), enough for states whose residual is taken to
// 1e-10). The operations have the interface of lbm_vec.cuh, so the per-node physics of
// lbm_physics.cuh compiles for dd unchanged.
#pragma once

#include "lbm_physics.cuh"
#include "lbm_vec.cuh"

#include <cuda_runtime.h>

namespace lbm {

struct dd {
  float hi, lo;
};

__device__ __forceinline__ dd dd_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return dd{s, e};
}
__device__ __forceinline__ dd dd_fast_two_sum(float a, float b) {  // |a| >= |b| or a = 0
  const float s = __fadd_rn(a, b);
  return dd{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dd dd_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return dd{p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ dd operator+(dd a, dd b) {
  const dd s = dd_two_sum(a.hi, b.hi);
  return dd_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dd operator-(dd a) { return dd{-a.hi, -a.lo}; }
__device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }
__device__ __forceinline__ dd operator*(dd a, dd b) {
  const dd p = dd_two_prod(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.lo, p.lo);
  e = __fmaf_rn(a.lo, b.hi, e);
  return dd_fast_two_sum(p.hi, e);
}
__device__ __forceinline__ dd fmadd(dd a, dd b, dd c) { return a * b + c; }

// a / b: q1 = a/b in FP32, then one correction from the dd remainder a - b q1
__device__ __forceinline__ dd fast_div(dd a, dd b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const dd r = a - b * dd{q1, 0.f};
  const float q2 = __fdiv_rn(r.hi, b.hi);
  return dd_fast_two_sum(q1, q2);
}

// sqrt of max(x, 0) with `bad` set when x < 0 or NaN, as for the other value types
__device__ __forceinline__ dd sqrt_checked(dd x, bool& bad) {
  if (!(x.hi >= 0.f) || (x.hi == 0.f && x.lo < 0.f)) {
    bad = true;
    return dd{0.f, 0.f};
  }
  if (x.hi == 0.f) return dd{0.f, 0.f};
  const float s = __fsqrt_rn(x.hi);
  const dd r = x - dd_two_prod(s, s);  // x - s^2, exact up to x's own lo
  return dd_fast_two_sum(s, __fdiv_rn(r.hi, __fadd_rn(s, s)));
}

__device__ __forceinline__ bool nonpositive(dd x) { return !(x.hi > 0.f) && !(x.hi == 0.f && x.lo > 0.f); }
__device__ __forceinline__ double hsum(dd x) { return double(x.hi) + double(x.lo); }

// nearest dd of a double: hi = the FP32 rounding, lo = the FP32 rounding of the rest
__host__ __device__ inline dd dd_of(double c) {
  const float h = float(c);
  return dd{h, float(c - double(h))};
}

template <>
struct VecTraits<dd> {
  using scalar = float;
  static constexpr int width = 1;
  __device__ static dd cst(double c) { return dd_of(c); }
};

template <>
__host__ __device__ inline dd from_double<dd>(double x) {
  return dd_of(x);
}

// per-thread mass partial of dd values: three dd chains (the values' own precision)
template <>
struct Acc<dd> {
  dd s[3] = {dd{0.f, 0.f}, dd{0.f, 0.f}, dd{0.f, 0.f}};
  __device__ void add9(const dd (&v)[9]) {
#pragma unroll
    for (int i = 0; i < 9; ++i) s[i % 3] = s[i % 3] + v[i];
  }
  __device__ double value() const { return (hsum(s[0]) + hsum(s[1])) + hsum(s[2]); }
};

}  // namespace lbm
