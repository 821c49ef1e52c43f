// Complex arithmetic on double2 / float2 (re, im) for the FTH-MS kernels.
#pragma once
#include <cuda_runtime.h>

namespace fthms {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// c + a * b
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
// c - a * b
__device__ __forceinline__ double2 cfms(double2 a, double2 b, double2 c) {
  return make_double2(fma(-a.x, b.x, fma(a.y, b.y, c.x)), fma(-a.x, b.y, fma(-a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 crecip(double2 a) {
  double d = 1.0 / fma(a.x, a.x, a.y * a.y);
  return make_double2(a.x * d, -a.y * d);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// FP32 complex helpers (mixed-precision factorisation and solves)
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cfms(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(-a.x, b.x, fmaf(a.y, b.y, c.x)), fmaf(-a.x, b.y, fmaf(-a.y, b.x, c.y)));
}
__device__ __forceinline__ float2 crecip(float2 a) {
  float d = 1.0f / fmaf(a.x, a.x, a.y * a.y);
  return make_float2(a.x * d, -a.y * d);
}
__device__ __forceinline__ double2 make_neg(double2 a) { return make_double2(-a.x, -a.y); }
__device__ __forceinline__ float2 make_neg(float2 a) { return make_float2(-a.x, -a.y); }

template <class C> struct CTraits;
template <> struct CTraits<double2> { using R = double; };
template <> struct CTraits<float2> { using R = float; };

}  // namespace fthms
