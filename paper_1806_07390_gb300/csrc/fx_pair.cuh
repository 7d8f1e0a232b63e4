// Two FP32 values processed together: the two groups a lane owns in the stage kernel of the FP32
// forms.  Additions, subtractions, multiplications and fused multiply-adds use the packed FP32
// instructions of sm_100 and later (add/sub/mul/fma .f32x2: one instruction for both values,
// each rounded exactly as the scalar instruction would round it, denormals flushed as in the
// FP32 translation units).  Comparisons, selects, minima, reciprocals and square roots act on the
// two values one by one.
#pragma once
#include <cuda_runtime.h>

namespace fx {

struct F2 {
  float x, y;
  __device__ __forceinline__ F2() {}
  __device__ __forceinline__ F2(float a, float b) : x(a), y(b) {}
  __device__ __forceinline__ explicit F2(float a) : x(a), y(a) {}
};

__device__ __forceinline__ unsigned long long f2_pack(F2 a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ F2 f2_unpack(unsigned long long r) {
  F2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
__device__ __forceinline__ F2 operator+(F2 a, F2 b) {
  unsigned long long r;
  asm("add.rn.ftz.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)));
  return f2_unpack(r);
}
__device__ __forceinline__ F2 operator-(F2 a, F2 b) {
  unsigned long long r;
  asm("sub.rn.ftz.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)));
  return f2_unpack(r);
}
__device__ __forceinline__ F2 operator*(F2 a, F2 b) {
  unsigned long long r;
  asm("mul.rn.ftz.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)));
  return f2_unpack(r);
}
__device__ __forceinline__ F2 operator-(F2 a) { return F2(-a.x, -a.y); }
__device__ __forceinline__ F2 operator+(F2 a, float b) { return a + F2(b); }
__device__ __forceinline__ F2 operator+(float a, F2 b) { return F2(a) + b; }
__device__ __forceinline__ F2 operator-(F2 a, float b) { return a - F2(b); }
__device__ __forceinline__ F2 operator-(float a, F2 b) { return F2(a) - b; }
__device__ __forceinline__ F2 operator*(F2 a, float b) { return a * F2(b); }
__device__ __forceinline__ F2 operator*(float a, F2 b) { return F2(a) * b; }

// Fused multiply-add a b + c, one rounding, for the scalar types and the pair.
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double vfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ F2 vfma(F2 a, F2 b, F2 c) {
  unsigned long long r;
  asm("fma.rn.ftz.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)), "l"(f2_pack(c)));
  return f2_unpack(r);
}
__device__ __forceinline__ F2 vfma(F2 a, float b, F2 c) { return vfma(a, F2(b), c); }
__device__ __forceinline__ F2 vfma(float a, F2 b, F2 c) { return vfma(F2(a), b, c); }

// Componentwise operations, with the scalar overloads used by code written for either type.
__device__ __forceinline__ F2 frcp(F2 a) { return F2(__fdividef(1.0f, a.x), __fdividef(1.0f, a.y)); }
__device__ __forceinline__ float vsqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ double vsqrt(double a) { return ::sqrt(a); }
__device__ __forceinline__ F2 vsqrt(F2 a) { return F2(sqrtf(a.x), sqrtf(a.y)); }
__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ F2 vmin(F2 a, F2 b) { return F2(fminf(a.x, b.x), fminf(a.y, b.y)); }
__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ F2 vmax(F2 a, F2 b) { return F2(fmaxf(a.x, b.x), fmaxf(a.y, b.y)); }
__device__ __forceinline__ float vabs(float a) { return fabsf(a); }
__device__ __forceinline__ F2 vabs(F2 a) { return F2(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ double vmin(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ double vmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ double vabs(double a) { return fabs(a); }
// x > t ? a : b, componentwise in x, a and b
__device__ __forceinline__ float vsel_gt(float x, float t, float a, float b) { return x > t ? a : b; }
__device__ __forceinline__ double vsel_gt(double x, double t, double a, double b) { return x > t ? a : b; }
__device__ __forceinline__ F2 vsel_gt(F2 x, float t, F2 a, F2 b) {
  return F2(x.x > t ? a.x : b.x, x.y > t ? a.y : b.y);
}

// Slope of the MC limiter from the one-sided slopes sL, sR and the centred slope sC: the least of
// 2|sL|, 2|sR| and |sC|, with the common sign of sL and sR, and zero where their signs differ or
// one is zero.  Where sL and sR share a sign, sC has it too (the centred difference is the sum
// of the two one-sided ones, each scaled by a positive reciprocal distance), so the sign factor
// (-1, 0 or 1, exact) replaces the product test and the selects.  FP32 and the pair.
__device__ __forceinline__ float mc_slope(float sL, float sR, float sC) {
  const float m = fminf(2.0f * fminf(fabsf(sL), fabsf(sR)), fabsf(sC));
  return m * (copysignf(0.5f, sL) + copysignf(0.5f, sR));
}
__device__ __forceinline__ F2 mc_slope(F2 sL, F2 sR, F2 sC) {
  const F2 m2 = F2(fminf(fabsf(sL.x), fabsf(sR.x)), fminf(fabsf(sL.y), fabsf(sR.y))) * 2.0f;
  const F2 m(fminf(m2.x, fabsf(sC.x)), fminf(m2.y, fabsf(sC.y)));
  return m * (F2(copysignf(0.5f, sL.x), copysignf(0.5f, sL.y)) +
              F2(copysignf(0.5f, sR.x), copysignf(0.5f, sR.y)));
}

// A value of type V from the values of the lane's two groups (the pair, or the first value), and
// component j of a value.
__device__ __forceinline__ float vpair(float a, float, float) { return a; }
__device__ __forceinline__ double vpair(double a, double, double) { return a; }
__device__ __forceinline__ F2 vpair(float a, float b, F2) { return F2(a, b); }
__device__ __forceinline__ float vget(float x, int) { return x; }
__device__ __forceinline__ double vget(double x, int) { return x; }
__device__ __forceinline__ float vget(F2 x, int j) { return j ? x.y : x.x; }

// Shared-memory access of the values of a lane's groups at p (the lane's first group): one
// value, or (F2) the two values at p[0], p[1] with one 8-byte access (p 8-byte aligned).  The
// store writes only the groups that exist (h0, h1).
__device__ __forceinline__ float ld_lane(const float* p, float) { return *p; }
__device__ __forceinline__ double ld_lane(const double* p, double) { return *p; }
__device__ __forceinline__ F2 ld_lane(const float* p, F2) {
  const float2 v = *reinterpret_cast<const float2*>(p);
  return F2(v.x, v.y);
}
__device__ __forceinline__ void st_lane(float* p, float v, bool h0, bool) { if (h0) *p = v; }
__device__ __forceinline__ void st_lane(double* p, double v, bool h0, bool) { if (h0) *p = v; }
__device__ __forceinline__ void st_lane(float* p, F2 v, bool h0, bool h1) {
  if (h1) *reinterpret_cast<float2*>(p) = make_float2(v.x, v.y);
  else if (h0) *p = v.x;
}

}  // namespace fx
