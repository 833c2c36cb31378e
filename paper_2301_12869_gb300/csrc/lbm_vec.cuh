// Value types of the fused step's per-node arithmetic: float, double, and f2, a
// pair of FP32 values (two neighbouring nodes) held in one 64-bit register and
// processed by sm_100-family packed FP32 instructions (add/sub/mul/fma .rn.f32x2).
// The per-node physics in lbm_kernels.cu is written once over these types.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace lbm {

struct f2 {
  unsigned long long v;
};

__device__ __forceinline__ f2 make_f2(float a, float b) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float lo(f2 x) {
  float a;
  [[maybe_unused]] float b;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x.v));
  return a;
}
__device__ __forceinline__ float hi(f2 x) {
  [[maybe_unused]] float a;
  float b;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x.v));
  return b;
}
__device__ __forceinline__ f2 operator+(f2 a, f2 b) {
  f2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f2 operator-(f2 a, f2 b) {
  f2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f2 operator*(f2 a, f2 b) {
  f2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}

// a * b + c with one rounding
__device__ __forceinline__ float fmadd(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ f2 fmadd(f2 a, f2 b, f2 c) {
  f2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return r;
}

// constants and conversions
template <typename V>
struct VecTraits;
template <>
struct VecTraits<float> {
  using scalar = float;
  static constexpr int width = 1;
  __device__ static float cst(double c) { return float(c); }
};
template <>
struct VecTraits<double> {
  using scalar = double;
  static constexpr int width = 1;
  __device__ static double cst(double c) { return c; }
};
template <>
struct VecTraits<f2> {
  using scalar = float;
  static constexpr int width = 2;
  __device__ static f2 cst(double c) { return make_f2(float(c), float(c)); }
};
template <typename V>
__device__ __forceinline__ V cst(double c) {
  return VecTraits<V>::cst(c);
}

// Division and square root: IEEE in FP64 (the FP64 path is checked to 1e-14); in FP32
// the fast intrinsics __fdividef (<= 2 ulp) and rsqrtf (<= 2 ulp), and for node pairs the
// approximate reciprocal and square root instructions (rcp.approx / sqrt.approx, a few
// ulp), add at most a few ulp, far inside the FP32 path's 1e-6 bound against the FP64
// oracle.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double fast_div(double a, double b) { return a / b; }
__device__ __forceinline__ float fast_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ f2 fast_div(f2 a, f2 b) { return a * make_f2(rcp_approx(lo(b)), rcp_approx(hi(b))); }

// sqrt of max(x, 0); sets `bad` when x < 0 or NaN (psi undefined)
__device__ __forceinline__ double sqrt_checked(double x, bool& bad) {
  if (!(x >= 0.0)) {
    bad = true;
    x = 0.0;
  }
  return sqrt(x);
}
__device__ __forceinline__ float sqrt_checked(float x, bool& bad) {
  if (!(x >= 0.f)) {
    bad = true;
    x = 0.f;
  }
  return x > 0.f ? x * rsqrtf(x) : 0.f;
}
__device__ __forceinline__ f2 sqrt_checked(f2 x, bool& bad) {
  const float s = lo(x), t = hi(x);
  if (!(s >= 0.f) || !(t >= 0.f)) bad = true;
  return make_f2(sqrt_approx(fmaxf(s, 0.f)), sqrt_approx(fmaxf(t, 0.f)));
}

// true if any component is <= 0 or NaN
__device__ __forceinline__ bool nonpositive(double x) { return !(x > 0.0); }
__device__ __forceinline__ bool nonpositive(float x) { return !(x > 0.f); }
__device__ __forceinline__ bool nonpositive(f2 x) { return !(lo(x) > 0.f) || !(hi(x) > 0.f); }

// a value of type V from a double (one component)
template <typename V>
__host__ __device__ V from_double(double x);
template <>
__host__ __device__ inline float from_double<float>(double x) {
  return float(x);
}
template <>
__host__ __device__ inline double from_double<double>(double x) {
  return x;
}

// sum of the components in FP64
__device__ __forceinline__ double hsum(double x) { return x; }
__device__ __forceinline__ double hsum(float x) { return double(x); }
__device__ __forceinline__ double hsum(f2 x) { return double(lo(x)) + double(hi(x)); }

}  // namespace lbm
