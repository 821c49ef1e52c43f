// Double-float ("df64") arithmetic on the FP32 pipe: a value is hi + lo with two floats, |lo| <=
// ulp(hi)/2, about 48 significant bits.  Built from the published error-free transformations:
// Knuth's two-sum (TAOCP vol. 2, 4.2.2) and the FMA form of Dekker's two-product (Dekker 1971).
// Products are accumulated lazily: the exact rounding error of each hi*hi product and the hi*lo
// cross terms go into the low word, which is renormalised once at the end of a sum.
#pragma once
#include <cuda_runtime.h>

namespace fthms {

struct df {
  float hi, lo;
};

// Complex double-float, laid out as float4 (re.hi, re.lo, im.hi, im.lo).
__device__ __forceinline__ float4 df_split2(double2 v) {
  const float rh = __double2float_rn(v.x);
  const float ih = __double2float_rn(v.y);
  return make_float4(rh, __double2float_rn(v.x - (double)rh), ih, __double2float_rn(v.y - (double)ih));
}

__device__ __forceinline__ double2 df_join2(float4 v) {
  return make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
}

// The _rn intrinsics keep every operation of the error-free transformations separately rounded (the
// compiler never contracts them into FMAs).
// s + e exactly (Knuth two-sum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
}

// s + e exactly for |a| >= |b|.
__device__ __forceinline__ void quick_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// Running compensated sum: hi carries the rounded sum, lo the accumulated errors and low parts.
struct dfacc {
  float hi = 0.f, lo = 0.f;
  // += (ah + al) * (bh + bl), dropping al * bl
  __device__ __forceinline__ void mac(float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    float s, t;
    two_sum(hi, p, s, t);
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(t, e));
  }
  __device__ __forceinline__ void add(float h, float l) {
    float s, t;
    two_sum(hi, h, s, t);
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(t, l));
  }
  __device__ __forceinline__ df value() const {
    df r;
    quick_two_sum(hi, lo, r.hi, r.lo);
    return r;
  }
};

// Double-float scalar arithmetic (a value is hi + lo): products from the FMA two-product with the
// cross terms, sums from two Knuth two-sums (the accurate form, safe under cancellation).
__device__ __forceinline__ df df_from(double v) {
  const float h = __double2float_rn(v);
  return df{h, __double2float_rn(v - (double)h)};
}
__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  df r;
  quick_two_sum(p, e, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ df df_add(df a, df b) {
  float s, e, t, f;
  two_sum(a.hi, b.hi, s, e);
  two_sum(a.lo, b.lo, t, f);
  e = __fadd_rn(e, t);
  quick_two_sum(s, e, s, e);
  e = __fadd_rn(e, f);
  df r;
  quick_two_sum(s, e, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

// a * b + c * d with one two-sum on the rounded products (their exact errors and the hi * lo cross
// terms added to the low word): error about 2^-46 (|ab| + |cd|).  Enough where accuracy is judged
// against the norm of a whole vector, as in the butterflies of an FFT.
__device__ __forceinline__ df df_dot2(df a, df b, df c, df d) {
  const float p = __fmul_rn(a.hi, b.hi), q = __fmul_rn(c.hi, d.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  float f = fmaf(c.hi, d.hi, -q);
  f = fmaf(c.hi, d.lo, f);
  f = fmaf(c.lo, d.hi, f);
  float s, t;
  two_sum(p, q, s, t);
  t = __fadd_rn(t, __fadd_rn(e, f));
  df r;
  quick_two_sum(s, t, r.hi, r.lo);
  return r;
}
// a + b with one two-sum on the high words; error about 2^-46 (|a| + |b|), as df_dot2.
__device__ __forceinline__ df df_add_fast(df a, df b) {
  float s, t;
  two_sum(a.hi, b.hi, s, t);
  t = __fadd_rn(t, __fadd_rn(a.lo, b.lo));
  df r;
  quick_two_sum(s, t, r.hi, r.lo);
  return r;
}

// a / b: the FP32 quotient corrected once with the double-float remainder (error about 2^-46).
__device__ __forceinline__ df df_div(df a, df b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const df r = df_sub(a, df_mul(b, df{q1, 0.f}));
  df q;
  quick_two_sum(q1, __fdiv_rn(r.hi, b.hi), q.hi, q.lo);
  return q;
}

// Complex double-float (float4 layout) for the mixed-form FFT butterflies.
__device__ __forceinline__ float4 dfc_mul(float4 a, float4 b) {
  const df re = df_dot2(df{a.x, a.y}, df{b.x, b.y}, df{-a.z, -a.w}, df{b.z, b.w});
  const df im = df_dot2(df{a.x, a.y}, df{b.z, b.w}, df{a.z, a.w}, df{b.x, b.y});
  return make_float4(re.hi, re.lo, im.hi, im.lo);
}
__device__ __forceinline__ float4 dfc_add(float4 a, float4 b) {
  const df re = df_add_fast(df{a.x, a.y}, df{b.x, b.y}), im = df_add_fast(df{a.z, a.w}, df{b.z, b.w});
  return make_float4(re.hi, re.lo, im.hi, im.lo);
}
__device__ __forceinline__ float4 dfc_sub(float4 a, float4 b) {
  const df re = df_add_fast(df{a.x, a.y}, df{-b.x, -b.y}), im = df_add_fast(df{a.z, a.w}, df{-b.z, -b.w});
  return make_float4(re.hi, re.lo, im.hi, im.lo);
}

// A double constant as a double-float pair, folded at compile time when used in a constant expression.
__host__ __device__ constexpr df df_const(double v) { return df{(float)v, (float)(v - (double)(float)v)}; }

// sin x and cos x for |x| <= 1 in double-float: the Taylor series (truncation below 2e-20, as for the
// FP64 version) by Horner's rule in u = x^2 with the coefficients (-1)^k/(2k+1)! and (-1)^k/(2k)!.
__device__ __forceinline__ void df_sincos_taylor(df x, df& s, df& c) {
  constexpr double f3 = 6.0, f5 = f3 * 20.0, f7 = f5 * 42.0, f9 = f7 * 72.0, f11 = f9 * 110.0,
                   f13 = f11 * 156.0, f15 = f13 * 210.0, f17 = f15 * 272.0, f19 = f17 * 342.0;
  constexpr double f2 = 2.0, f4 = f2 * 12.0, f6 = f4 * 30.0, f8 = f6 * 56.0, f10 = f8 * 90.0,
                   f12 = f10 * 132.0, f14 = f12 * 182.0, f16 = f14 * 240.0, f18 = f16 * 306.0,
                   f20 = f18 * 380.0;
  constexpr df ks[9] = {df_const(-1.0 / f19), df_const(1.0 / f17), df_const(-1.0 / f15), df_const(1.0 / f13),
                        df_const(-1.0 / f11), df_const(1.0 / f9),  df_const(-1.0 / f7),  df_const(1.0 / f5),
                        df_const(-1.0 / f3)};
  constexpr df kc[10] = {df_const(1.0 / f20),  df_const(-1.0 / f18), df_const(1.0 / f16), df_const(-1.0 / f14),
                         df_const(1.0 / f12),  df_const(-1.0 / f10), df_const(1.0 / f8),  df_const(-1.0 / f6),
                         df_const(1.0 / f4),   df_const(-1.0 / f2)};
  const df u = df_mul(x, x);
  df ps = ks[0];
#pragma unroll
  for (int k = 1; k < 9; ++k) ps = df_add(df_mul(ps, u), ks[k]);
  s = df_add(x, df_mul(df_mul(x, u), ps));
  df pc = kc[0];
#pragma unroll
  for (int k = 1; k < 10; ++k) pc = df_add(df_mul(pc, u), kc[k]);
  c = df_add(df{1.f, 0.f}, df_mul(u, pc));
}

// sin(pi D / den) for |D| < den < 2^24, den divisible by 4, in double-float: the fraction reduced in
// integers to a = Da / den in [0, 1/4] (sin(pi (1 - t)) = sin(pi t), sin(pi t) = cos(pi (1/2 - t))),
// the quotient formed exactly to double-float (FMA remainder), then the Taylor series at pi a.
__device__ __forceinline__ df df_sinpi_frac(int D, int den) {
  int a = D < 0 ? -D : D;
  if (2 * a > den) a = den - a;
  const bool use_cos = 4 * a > den;
  if (use_cos) a = den / 2 - a;
  const float fa = (float)a, fd = (float)den;
  const float q0 = __fdiv_rn(fa, fd);
  const float r = fmaf(-q0, fd, fa);
  df q;
  quick_two_sum(q0, __fdiv_rn(r, fd), q.hi, q.lo);
  constexpr df kPi = df_const(3.14159265358979323846);
  df s, c;
  df_sincos_taylor(df_mul(kPi, q), s, c);
  const df v = use_cos ? c : s;
  return D < 0 ? df_neg(v) : v;
}

// Complex compensated multiply-accumulate: acc += a * b with a, b complex df64 (float4 layout).
__device__ __forceinline__ void cdf_mac(dfacc& re, dfacc& im, float4 a, float4 b) {
  re.mac(a.x, a.y, b.x, b.y);
  re.mac(-a.z, -a.w, b.z, b.w);
  im.mac(a.x, a.y, b.z, b.w);
  im.mac(a.z, a.w, b.x, b.y);
}

}  // namespace fthms

namespace fthms {

// sqrt(a) for a > 0 in double-float: the FP32 root r corrected once by Newton's step with the exact
// residual a - r^2 (two-product), error about 2^-46.
__device__ __forceinline__ df df_sqrt(df a) {
  const float r = sqrtf(a.hi);
  const float p = __fmul_rn(r, r);
  const float pe = fmaf(r, r, -p);                    // r^2 = p + pe exactly
  const float d = __fadd_rn(__fadd_rn(__fsub_rn(a.hi, p), a.lo), -pe);
  df out;
  quick_two_sum(r, __fdiv_rn(d, __fmul_rn(2.f, r)), out.hi, out.lo);
  return out;
}

// 1 / sqrt(a) for a > 0 in double-float: y = rsqrt(a.hi) refined by one Newton step y (3 - a y^2) / 2
// with the product in double-float, error about 2^-46.
__device__ __forceinline__ df df_rsqrt(df a) {
  const float y = rsqrtf(a.hi);
  const df y2 = df_mul(df{y, 0.f}, df{y, 0.f});
  const df e = df_sub(df{1.f, 0.f}, df_mul(a, y2));   // 1 - a y^2, small
  df out;
  quick_two_sum(y, __fmul_rn(__fmul_rn(0.5f, y), e.hi), out.hi, out.lo);
  return out;
}


// a ~ hi + lo for a double a with 2^-60 <= |a| < 2^100 by integer operations only (no FP64 instruction):
// hi = a truncated to 24 significant bits, lo = the 29 fraction bits below them rounded to 24 bits (one
// integer-to-float conversion, its exponent then shifted by that of a), so |a - hi - lo| <= 2^-47 |a|.
// Outside that range (zero included) the FP64 conversions.
__device__ __forceinline__ void split_f64_bits(double a, float& hi, float& lo) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(a);
  const unsigned int uh = (unsigned int)(u >> 32), ul = (unsigned int)u;
  const int e = (int)((uh >> 20) & 0x7FFu);                   // biased FP64 exponent
  if (e < 1023 - 60 || e > 1023 + 100) {
    hi = __double2float_rn(a);
    lo = __double2float_rn(a - (double)hi);
    return;
  }
  const unsigned int sign = uh & 0x80000000u;
  const unsigned int frac23 = __funnelshift_l(ul, uh, 3) & 0x007FFFFFu;   // the top 23 fraction bits
  hi = __uint_as_float(sign | ((unsigned int)(e - 1023 + 127) << 23) | frac23);
  const unsigned int rem = ul & 0x1FFFFFFFu;                  // the 29 fraction bits below: rem 2^(e - 1075)
  const float r = __uint2float_rn(rem);
  lo = rem ? __uint_as_float(sign | (__float_as_uint(r) + ((unsigned int)(e - 1075) << 23))) : 0.f;
}

// acc += a * b for a = ah + al (double-float) and b a float: the exact error of ah b by the FMA
// two-product, al b added to the low word.
__device__ __forceinline__ void dfacc_mac1(dfacc& acc, float ah, float al, float b) {
  const float p = __fmul_rn(ah, b);
  float e = fmaf(ah, b, -p);
  e = fmaf(al, b, e);
  float s, t;
  two_sum(acc.hi, p, s, t);
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(t, e));
}

// a = a1 + a2 + a3 exactly for a double a with 2^-60 <= |a| < 2^100, by integer operations only: a1 = a truncated
// to 24 significant bits, a2 = the next 24 bits, a3 = the last 5 (integers below 2^24 convert to float exactly,
// then their exponents are shifted by that of a).  Outside that range (zero included; |a| below 2^128) by FP64
// operations.
__device__ __forceinline__ void split3_f64_bits(double a, float& a1, float& a2, float& a3) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(a);
  const unsigned int uh = (unsigned int)(u >> 32), ul = (unsigned int)u;
  const int e = (int)((uh >> 20) & 0x7FFu);
  if (e < 1023 - 60 || e > 1023 + 100) {
    a1 = __double2float_rn(a);
    const double r = a - (double)a1;
    a2 = __double2float_rn(r);
    a3 = __double2float_rn(r - (double)a2);
    return;
  }
  const unsigned int sign = uh & 0x80000000u;
  a1 = __uint_as_float(sign | ((unsigned int)(e - 1023 + 127) << 23) | (__funnelshift_l(ul, uh, 3) & 0x007FFFFFu));
  const unsigned int rem = ul & 0x1FFFFFFFu;            // the 29 fraction bits below a1: rem 2^(e - 1075)
  const unsigned int top = rem >> 5, low = rem & 31u;
  a2 = top ? __uint_as_float(sign | (__float_as_uint(__uint2float_rn(top)) + ((unsigned int)(e - 1070) << 23))) : 0.f;
  a3 = low ? __uint_as_float(sign | (__float_as_uint(__uint2float_rn(low)) + ((unsigned int)(e - 1075) << 23))) : 0.f;
}

// Anchored sums of products a x (a = a1 + a2 + a3 the exact three-float split, x a float) on the FP32 pipe,
// by error-free extraction against fixed power-of-two anchors (the "ExtractScalar" step of Rump, Ogita and
// Oishi's accurate summation, 2008).  With every partial sum of |a x| below 2^(kh-1), H starts at
// 1.5 2^kh and stays in [2^kh, 2^(kh+1)]: t = H + p1 and q = t - H are exact (Sterbenz), and p1 - q is the
// exact part of p1 below H's ulp (Fast2Sum, |H| >= |p1|).  Those parts, the product errors e1 (FMA
// two-product) and a2 x go the same way into M, anchored at 1.5 2^km (km = kh - 23 + ceil(log2(T + 4)) for
// T terms, so M too stays in its binade); a2 x through one FMA (M + a2 x rounded once, then the exact
// q and the rest a2 x - q rounded once more, ~2^(km-47)).  What falls below M's ulp, and a3 x, are added
// plainly in l, which renorm() folds back into M.  18 FP32 instructions a product instead of the 34 that
// exact three-level two-sums take; the error, about 2^-50 of the sum of |a x| (the anchors' scale), is of
// the order of an FP64 accumulation's.
struct aacc {
  float H, M, l, sh, sm;
  __device__ __forceinline__ void init(int kh, int km) {     // -126 < km < kh < 128
    H = sh = __uint_as_float(((unsigned)(127 + kh) << 23) | 0x400000u);   // 1.5 2^kh
    M = sm = __uint_as_float(((unsigned)(127 + km) << 23) | 0x400000u);
    l = 0.f;
  }
  __device__ __forceinline__ void put_m(float v) {      // |v| <= |M| / 2: exact split into M's grid and l
    const float t = __fadd_rn(M, v);
    l = __fadd_rn(l, __fsub_rn(v, __fsub_rn(t, M)));
    M = t;
  }
  __device__ __forceinline__ void add_prod(float a1, float a2, float a3, float x) {
    const float p1 = __fmul_rn(a1, x), e1 = fmaf(a1, x, -p1);
    const float t = __fadd_rn(H, p1);
    const float r1 = __fsub_rn(p1, __fsub_rn(t, H));
    H = t;
    put_m(r1);
    put_m(e1);
    const float u = fmaf(a2, x, M);
    const float q = __fsub_rn(u, M);
    l = __fadd_rn(l, fmaf(a2, x, -q));
    M = u;
    l = fmaf(a3, x, l);
  }
  __device__ __forceinline__ void renorm() {       // l's high part into M (exact), keeping l small
    const float t = __fadd_rn(M, l);
    l = __fsub_rn(l, __fsub_rn(t, M));
    M = t;
  }
  __device__ __forceinline__ double value() const {
    return ((double)__fsub_rn(H, sh) + (double)__fsub_rn(M, sm)) + (double)l;
  }
};

}  // namespace fthms
