// Forward-mode dual numbers with N tangent directions, for the local Jacobians of the adjoint.
//
// The adjoint of a stage (fx_adjoint.cuh) is assembled by hand in reverse order; the few pure
// functions whose derivatives are long to write out (the coordinate-moment reconstruction with
// its limiter branches, HLLC, the M1 pressure row, the MC-limited linear reconstruction) are
// differentiated by running the forward device function itself on Dn values seeded with unit
// tangents of its inputs.  Branches test the value part, so each Jacobian is the exact
// derivative of the branch the forward took.
#pragma once
#include <cuda_runtime.h>

namespace fx {

template <class R, int N> struct Dn {
  R v;
  R d[N];
  __device__ __forceinline__ Dn() {}
  __device__ __forceinline__ Dn(R x) : v(x) {
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = R(0);
  }
  // value x with unit tangent in direction i
  __device__ __forceinline__ static Dn seed(R x, int i) {
    Dn r(x);
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = k == i ? R(1) : R(0);
    return r;
  }
  __device__ __forceinline__ Dn& operator+=(const Dn& b) { *this = *this + b; return *this; }
  __device__ __forceinline__ Dn& operator-=(const Dn& b) { *this = *this - b; return *this; }
  __device__ __forceinline__ Dn& operator*=(const Dn& b) { *this = *this * b; return *this; }

  friend __device__ __forceinline__ Dn operator+(const Dn& a, const Dn& b) {
    Dn r;
    r.v = a.v + b.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
    return r;
  }
  friend __device__ __forceinline__ Dn operator-(const Dn& a, const Dn& b) {
    Dn r;
    r.v = a.v - b.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
    return r;
  }
  friend __device__ __forceinline__ Dn operator-(const Dn& a) {
    Dn r;
    r.v = -a.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
    return r;
  }
  friend __device__ __forceinline__ Dn operator*(const Dn& a, const Dn& b) {
    Dn r;
    r.v = a.v * b.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
    return r;
  }
  friend __device__ __forceinline__ Dn operator/(const Dn& a, const Dn& b) {
    const R ib = R(1) / b.v;
    Dn r;
    r.v = a.v * ib;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
    return r;
  }
  // mixed with plain values (constants)
  friend __device__ __forceinline__ Dn operator+(const Dn& a, R b) { Dn r = a; r.v += b; return r; }
  friend __device__ __forceinline__ Dn operator+(R a, const Dn& b) { Dn r = b; r.v += a; return r; }
  friend __device__ __forceinline__ Dn operator-(const Dn& a, R b) { Dn r = a; r.v -= b; return r; }
  friend __device__ __forceinline__ Dn operator-(R a, const Dn& b) {
    Dn r;
    r.v = a - b.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = -b.d[i];
    return r;
  }
  friend __device__ __forceinline__ Dn operator*(const Dn& a, R b) {
    Dn r;
    r.v = a.v * b;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b;
    return r;
  }
  friend __device__ __forceinline__ Dn operator*(R a, const Dn& b) { return b * a; }
  friend __device__ __forceinline__ Dn operator/(const Dn& a, R b) { return a * (R(1) / b); }
  friend __device__ __forceinline__ Dn operator/(R a, const Dn& b) {
    const R ib = R(1) / b.v;
    Dn r;
    r.v = a * ib;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = -r.v * b.d[i] * ib;
    return r;
  }
  // comparisons act on the value part
  friend __device__ __forceinline__ bool operator<(const Dn& a, const Dn& b) { return a.v < b.v; }
  friend __device__ __forceinline__ bool operator>(const Dn& a, const Dn& b) { return a.v > b.v; }
  friend __device__ __forceinline__ bool operator<=(const Dn& a, const Dn& b) { return a.v <= b.v; }
  friend __device__ __forceinline__ bool operator>=(const Dn& a, const Dn& b) { return a.v >= b.v; }
  friend __device__ __forceinline__ bool operator==(const Dn& a, const Dn& b) { return a.v == b.v; }
  friend __device__ __forceinline__ bool operator<(const Dn& a, R b) { return a.v < b; }
  friend __device__ __forceinline__ bool operator>(const Dn& a, R b) { return a.v > b; }
  friend __device__ __forceinline__ bool operator<=(const Dn& a, R b) { return a.v <= b; }
  friend __device__ __forceinline__ bool operator>=(const Dn& a, R b) { return a.v >= b; }
  // elementary functions: hidden friends (found by argument-dependent lookup only, so they do
  // not hide the plain-number overloads)
  friend __device__ __forceinline__ Dn sqrt(const Dn& a) {
    Dn r;
    r.v = sqrt(a.v);
    const R h = r.v > R(0) ? R(0.5) / r.v : R(0);
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * h;
    return r;
  }
  friend __device__ __forceinline__ Dn fabs(const Dn& a) { return a.v < R(0) ? -a : a; }
  friend __device__ __forceinline__ Dn fmin(const Dn& a, const Dn& b) { return b.v < a.v ? b : a; }
  friend __device__ __forceinline__ Dn fmax(const Dn& a, const Dn& b) { return b.v > a.v ? b : a; }
  friend __device__ __forceinline__ Dn frcp(const Dn& a) { return R(1) / a; }
};

}  // namespace fx
