// FP64 Bessel functions of order 0 for the Helmholtz kernel (i/4) H0^(1)(z) = (i/4)(J0 + i Y0)
// of Section 2.1, in two regimes:
//   0 <= z < 20  : J0 and the regular part Yhat0 = Y0 - (2/pi)(ln(z/2) + gamma) J0, both entire
//                  (J0 = sum_k (-z^2/4)^k/(k!)^2, Yhat0 = (2/pi) sum_{k>=1} (-1)^{k+1} H_k (z^2/4)^k/(k!)^2,
//                  Abramowitz-Stegun 9.1.12-9.1.13), by 13-term Taylor expansions about the centres
//                  0.25 + 0.5 k of 40 intervals of width 1/2 (coefficients: bessel_taylor.cuh).
//   z >= 20      : Hankel's asymptotic expansion with 10 + 10 terms,
//                  H0^(1)(z) ~ sqrt(2/(pi z)) e^{i(z - pi/4)} sum_k (-i)^k a_k/z^k,
//                  a_k = 1^2 3^2 ... (2k-1)^2/(k! 8^k)  (A-S 9.2.7-9.2.10, DLMF 10.17.5).
// Accuracy (checked against arbitrary-precision values): <= 1.2e-16 absolute for J0, Yhat0 below 20,
// <= 4e-16 relative to the amplitude sqrt(2/(pi z)) above.
#pragma once
#include <cuda_runtime.h>

#include "bessel_taylor.cuh"

namespace fthms {

constexpr double kEulerGamma = 0.57721566490153286060651209008240243;
constexpr double kPiD = 3.14159265358979323846;
constexpr double kInvPi = 0.31830988618379067153776752674502872;
constexpr double kTwoOverPi = 0.63661977236758134307553505349005745;
constexpr double kSqrtHalf = 0.70710678118654752440084436210484904;
constexpr double kBesselLarge = 20.0;
constexpr double kSqrtTwoOverPi = 0.79788456080286535587989211986876373;

// Terms (k = 0..kmax of P, k = 0..kmax of Q/w) of Hankel's expansion needed at z >= 20: the first
// omitted terms a_{2kmax+2}/z^{2kmax+2} and a_{2kmax+3}/z^{2kmax+3} stay below 2^-54 from these
// bounds on (below 24.2 the 9-term sum is the one checked against arbitrary-precision values).
__device__ __forceinline__ int hankel_terms(float z) {
  return z >= 467.f ? 2 : z >= 135.f ? 3 : z >= 67.7f ? 4 : z >= 44.2f ? 5 : z >= 33.5f ? 6 : z >= 27.7f ? 7
       : z >= 24.2f ? 8 : 9;
}

// sin x and cos x for |x| <= 1 from their Taylor series (x^21/21! and x^22/22! < 2e-20 bound the
// truncation), by Horner's rule in u = x^2 with the coefficients (-1)^k/(2k+1)! and (-1)^k/(2k)!.
// Used for the per-pair phase step e^{i h R}, whose argument is small.
__device__ __forceinline__ void sincos_taylor(double x, double& s, double& c) {
  constexpr double f3 = 6.0, f5 = f3 * 20.0, f7 = f5 * 42.0, f9 = f7 * 72.0, f11 = f9 * 110.0,
                   f13 = f11 * 156.0, f15 = f13 * 210.0, f17 = f15 * 272.0, f19 = f17 * 342.0;
  constexpr double f2 = 2.0, f4 = f2 * 12.0, f6 = f4 * 30.0, f8 = f6 * 56.0, f10 = f8 * 90.0,
                   f12 = f10 * 132.0, f14 = f12 * 182.0, f16 = f14 * 240.0, f18 = f16 * 306.0,
                   f20 = f18 * 380.0;
  const double u = x * x;
  double ps = -1.0 / f19;
  ps = fma(ps, u, 1.0 / f17);
  ps = fma(ps, u, -1.0 / f15);
  ps = fma(ps, u, 1.0 / f13);
  ps = fma(ps, u, -1.0 / f11);
  ps = fma(ps, u, 1.0 / f9);
  ps = fma(ps, u, -1.0 / f7);
  ps = fma(ps, u, 1.0 / f5);
  ps = fma(ps, u, -1.0 / f3);
  s = fma(x * u, ps, x);
  double pc = 1.0 / f20;
  pc = fma(pc, u, -1.0 / f18);
  pc = fma(pc, u, 1.0 / f16);
  pc = fma(pc, u, -1.0 / f14);
  pc = fma(pc, u, 1.0 / f12);
  pc = fma(pc, u, -1.0 / f10);
  pc = fma(pc, u, 1.0 / f8);
  pc = fma(pc, u, -1.0 / f6);
  pc = fma(pc, u, 1.0 / f4);
  pc = fma(pc, u, -1.0 / f2);
  c = fma(u, pc, 1.0);
}

// Hankel coefficients a_k (filled by init_constants(); this header is included by one translation
// unit only).
__constant__ double c_hank_a[20];
__constant__ float2 c_hank_df[20];   // the same coefficients as double-float (hi, lo)
// kTaylorJ0 and kTaylorYh as double-float pairs (mixed form), split on the host at start-up.
__device__ float2 c_taylor_df[2][kTaylorIntervals][kTaylorDegree + 1];

// 0 <= z < 20: piecewise Taylor expansions of J0 and Yhat0 about c_k = 0.25 + 0.5 k (both functions
// are entire), 13 terms each, coefficients from gen_bessel_taylor.py (mpmath).  Every lane runs the
// same instruction stream (two 12-step Horner chains), whatever its interval.
__device__ __forceinline__ void bessel0_taylor(double z, double& J0, double& Yh) {
  const int k = min((int)(2.0 * z), kTaylorIntervals - 1);
  const double d = z - fma(0.5, (double)k, 0.25);
  const double* cj = kTaylorJ0[k];
  const double* cy = kTaylorYh[k];
  double j = __ldg(&cj[kTaylorDegree]), y = __ldg(&cy[kTaylorDegree]);
#pragma unroll
  for (int n = kTaylorDegree - 1; n >= 0; --n) {
    j = fma(j, d, __ldg(&cj[n]));
    y = fma(y, d, __ldg(&cy[n]));
  }
  J0 = j;
  Yh = y;
}

// Hankel asymptotics given w = 1/z, amp = sqrt(2/(pi z)) and (s, c) = (sin z, cos z).
__device__ __forceinline__ void hankel_asym_phase(double w, double amp, double s, double c, double& J0,
                                                  double& Y0) {
  const double w2 = -w * w;
  double P = c_hank_a[18], Qa = c_hank_a[19];
#pragma unroll
  for (int k = 8; k >= 0; --k) {
    P = fma(P, w2, c_hank_a[2 * k]);
    Qa = fma(Qa, w2, c_hank_a[2 * k + 1]);
  }
  Qa *= w;
  const double cx = (c + s) * kSqrtHalf;   // cos(z - pi/4)
  const double sx = (s - c) * kSqrtHalf;   // sin(z - pi/4)
  J0 = amp * fma(P, cx, Qa * sx);
  Y0 = amp * fma(P, sx, -Qa * cx);
}

// Hankel asymptotics on z >= 20: J0 and Y0.
__device__ __forceinline__ void bessel0_asym(double z, double& J0, double& Y0) {
  const double w = 1.0 / z;
  double s, c;
  sincos(z, &s, &c);
  hankel_asym_phase(w, sqrt(kTwoOverPi * w), s, c, J0, Y0);
}

// Kernel pieces used by the Nystrom rules:
//  J0(z) and either Yhat0(z) (z < 20, has_yhat = true) or Y0(z) (z >= 20, has_yhat = false).
struct Bessel0 {
  double j0;
  double y;      // Yhat0 if has_yhat else Y0
  bool has_yhat;
};

__device__ __forceinline__ Bessel0 bessel0(double z) {
  Bessel0 b;
  if (z < kBesselLarge) {
    bessel0_taylor(z, b.j0, b.y);
    b.has_yhat = true;
  } else {
    bessel0_asym(z, b.j0, b.y);
    b.has_yhat = false;
  }
  return b;
}

// Full kernel Phi = (i/4) H0^(1)(z) = (-Y0/4, J0/4) for z > 0.
__device__ __forceinline__ double2 phi_kernel(double z) {
  Bessel0 b = bessel0(z);
  double y0 = b.has_yhat ? fma(kTwoOverPi * (log(0.5 * z) + kEulerGamma), b.j0, b.y) : b.y;
  return make_double2(-0.25 * y0, 0.25 * b.j0);
}

// Log-split pieces at a pair with parameter distance dts = |t - s| > 0 and z = kappa R:
//   K1 = -J0/(2 pi),  K2 = K - K1 ln|t - s|
//      = (i/4) J0 - (J0/(2 pi)) [ln(z/(2|t-s|)) + gamma] - Yhat0/4   (z < 20)
//      = (i/4) J0 - Y0/4 + (J0/(2 pi)) ln|t-s|                       (z >= 20)
__device__ __forceinline__ void log_split(double z, double dts, double& K1, double2& K2) {
  Bessel0 b = bessel0(z);
  K1 = -0.5 * kInvPi * b.j0;
  double re;
  if (b.has_yhat) {
    re = fma(K1, log(z / (2.0 * dts)) + kEulerGamma, -0.25 * b.y);
  } else {
    re = fma(-K1, log(dts), -0.25 * b.y);
  }
  K2 = make_double2(re, 0.25 * b.j0);
}

}  // namespace fthms
