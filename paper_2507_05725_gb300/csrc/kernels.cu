// CUDA kernels (sm_103a, FP64) of the FTH-MS open-arc hot path.
//
// Stages (one job):
//   tables         FFT twiddles, recentring phases, self log-weight tables, restriction tables
//   assemble_self  log-split Chebyshev Nystrom matrices A_j(omega_l)        (Section 4.2-4.3)
//   lu             A = P L U per (arc, omega), reused for every step and window (Algorithm 1)
//   cross_assemble stored S_Gamma_j rows at the other arcs' transfer nodes   (eq. FDsolk-interior)
//   incident       g_{k,1} = sign chi_k u^i on the transfer meshes, slow transform (eqs.
//                  criterion_int1, Fourierk)
//   restrict       transfer-mesh spectra -> data on the N_k(omega_l) solve nodes
//   per step m:
//     solve        phi = A^{-1} G                                             (eq. FDBIEk-interior)
//     cross_apply  W_k = sum_{j != k, masked} S_j[phi_j] (eq. vtilde) and the observation sum
//     synth_fwd    recentred inverse transform (eq. TDsol), g = -chi_k w (eq. criterion_int2),
//                  windowed slow transform (eq. Fourierk) -- one CTA per transfer node, in shared
//                  memory, with a radix-2 FFT
//   traces         u_M(z, t) at the output times (eq. mult-scatt-int)
#include <algorithm>
#include <cstdio>

#include "bessel.cuh"
#include "cplx.cuh"
#include "df64.cuh"
#include "kernels.h"
#include "lu_common.cuh"

namespace fthms {

cudaError_t init_constants() {
  double ha[20];
  ha[0] = 1.0;
  for (int k = 1; k < 20; ++k) ha[k] = ha[k - 1] * (double)((2 * k - 1) * (2 * k - 1)) / (8.0 * k);
  float2 hd[20];
  for (int k = 0; k < 20; ++k) {
    const float h = (float)ha[k];
    hd[k] = make_float2(h, (float)(ha[k] - (double)h));
  }
  cudaError_t e = cudaMemcpyToSymbol(c_hank_a, ha, sizeof ha);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(c_hank_df, hd, sizeof hd);
  if (e != cudaSuccess) return e;
  static double tj[kTaylorIntervals][kTaylorDegree + 1], ty[kTaylorIntervals][kTaylorDegree + 1];
  static float2 td[2][kTaylorIntervals][kTaylorDegree + 1];
  e = cudaMemcpyFromSymbol(tj, kTaylorJ0, sizeof tj);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyFromSymbol(ty, kTaylorYh, sizeof ty);
  if (e != cudaSuccess) return e;
  for (int k = 0; k < kTaylorIntervals; ++k)
    for (int n = 0; n <= kTaylorDegree; ++n) {
      const float a = (float)tj[k][n], c = (float)ty[k][n];
      td[0][k][n] = make_float2(a, (float)(tj[k][n] - (double)a));
      td[1][k][n] = make_float2(c, (float)(ty[k][n] - (double)c));
    }
  return cudaMemcpyToSymbol(c_taylor_df, td, sizeof td);
}

namespace {


// ---------------------------------------------------------------------------------------------
// Bessel test kernel
__global__ void k_bessel0(const double* __restrict__ z, double* j0, double* y0, double* yh, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double zz = z[i];
  Bessel0 b = bessel0(zz);
  double lg = kTwoOverPi * (log(0.5 * zz) + kEulerGamma);
  double Y0 = b.has_yhat ? fma(lg, b.j0, b.y) : b.y;
  double Yh = b.has_yhat ? b.y : fma(-lg, b.j0, b.y);
  if (j0) j0[i] = b.j0;
  if (y0) y0[i] = Y0;
  if (yh) yh[i] = Yh;
}

// ---------------------------------------------------------------------------------------------
// Tables

__global__ void k_fft_tw(double2* tw, float4* tw_df, int K) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= K / 2) return;
  double s, c;
  sincospi(2.0 * r / K, &s, &c);
  tw[r] = make_double2(c, -s);   // e^{-2 pi i r/K}
  if (tw_df) tw_df[r] = df_split2(make_double2(c, -s));
}

// syn_tw[q][l] = (w_l/pi) e^{-i l c_q} e^{-2 pi i (l nlo_q mod K)/K},  fwd_tw[q][l] = dt e^{i l c_q}
__global__ void k_freq_tw(DevJob J) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= J.Q * J.L) return;
  int q = idx / J.L, l = idx % J.L;
  double s, c;
  sincos((double)l * J.c_q[q], &s, &c);
  long long m = ((long long)l * J.nlo[q]) % J.K;
  double s2, c2;
  sincospi(2.0 * (double)m / J.K, &s2, &c2);
  double wl = J.wl[l] * kInvPi;
  double2 e1 = make_double2(c, -s), e2 = make_double2(c2, -s2);
  double2 sy = cmul(e1, e2);
  J.syn_tw[idx] = make_double2(wl * sy.x, wl * sy.y);
  J.fwd_tw[idx] = make_double2(J.dt * c, J.dt * s);
}

// Self log weights Rlog_il = -(pi/N) [ln 2 + F(|i-l|) + F(i+l+1)], F(m) = sum_{n=1}^{N-1} cos(n m pi/N)/n
// (the product-to-sum form of -(pi/N)[ln 2 + 2 sum_n T_n(t_i) T_n(t_l)/n]).
__global__ void k_rlog(DevJob J) {
  extern __shared__ double sh[];
  const int N = J.rlogN[blockIdx.x];
  double* cosr = sh;           // 2N
  double* F = sh + 2 * N;      // 2N
  double* invn = sh + 4 * N;   // N
  for (int r = threadIdx.x; r < 2 * N; r += blockDim.x) cosr[r] = cospi((double)r / N);
  for (int n = threadIdx.x; n < N; n += blockDim.x) invn[n] = n ? 1.0 / n : 0.0;
  __syncthreads();
  for (int m = threadIdx.x; m < 2 * N; m += blockDim.x) {
    double acc = 0.0;
    for (int n = 1; n < N; ++n) acc = fma(cosr[(n * m) % (2 * N)], invn[n], acc);
    F[m] = acc;
  }
  __syncthreads();
  double* out = J.rlog + J.rlog_off_N[blockIdx.x];
  const double ln2 = 0.69314718055994530941723212145817657;
  const double sc = -kPiD / N;
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    int i = e / N, l = e % N;
    int d = i > l ? i - l : l - i;
    out[e] = sc * (ln2 + F[d] + F[i + l + 1]);
  }
}

// Transposed restriction tables RT[x][i] = l_x(t_i): the Lagrange basis of the first-kind grid of
// size M evaluated at the first-kind nodes of size N, in the closed form
//   l_x(t_i) = T_M(t_i) sin(beta_x) (-1)^x / (M (t_i - tau_x))
// with the phases reduced exactly through D = (2i+1)M - (2x+1)N and S = (2i+1)M + (2x+1)N:
//   l_x(t_i) = sin(beta_x) sinpi(D/(2N)) / (2M sinpi(S/(4NM)) sinpi(D/(4NM))),  = 1 when D = 0,
// where sinpi(D/(2N)) = (-1)^(x+1) cospi((2i+1)M/(2N)) (the argument reduced mod 4N in integers) and
// sinpi(S/(4NM)) = sin(a_i + g_x), a_i = pi(2i+1)/(4N), g_x = pi(2x+1)/(4M), both in (0, pi/2), so
// only sinpi(D/(4NM)) is evaluated per entry.  One CTA per (N, M) pair; node tables in shared memory.
__global__ void k_restr(DevJob J) {
  extern __shared__ double shq[];
  const int t = blockIdx.x;
  const int N = J.restr_N[2 * t], M = J.restr_N[2 * t + 1];
  double* RT = J.restr + J.restr_off[t];
  double* cA = shq;          // N: cospi((2i+1)M / (2N))
  double* sa = cA + N;       // N: sin(a_i)
  double* ca = sa + N;       // N: cos(a_i)
  double* sb = ca + N;       // M: (-1)^(x+1) sin(beta_x)
  double* sg = sb + M;       // M: sin(g_x)
  double* cg = sg + M;       // M: cos(g_x)
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const long long A = ((long long)(2 * i + 1) * M) % (4LL * N);
    cA[i] = cospi((double)A / (2.0 * N));
    sincospi((double)(2 * i + 1) / (4.0 * N), &sa[i], &ca[i]);
  }
  for (int x = threadIdx.x; x < M; x += blockDim.x) {
    const double sbeta = sinpi((double)(2 * x + 1) / (2.0 * M));
    sb[x] = (x & 1) ? sbeta : -sbeta;
    sincospi((double)(2 * x + 1) / (4.0 * M), &sg[x], &cg[x]);
  }
  __syncthreads();
  const long long total = (long long)N * M;
  if (J.mixed) {
    // Mixed form: only the double-float table, computed on the FP32 pipe from the node tables
    // (converted in place, 8 bytes either way) with the exact fraction D / (4NM) for the sine.
    df* td = reinterpret_cast<df*>(shq);
    for (int k = threadIdx.x; k < 3 * (N + M); k += blockDim.x) td[k] = df_from(shq[k]);
    __syncthreads();
    const df *cAd = td, *sad = cAd + N, *cad = sad + N, *sbd = cad + N, *sgd = sbd + M, *cgd = sgd + M;
    const df m2d{(float)(2 * M), 0.f};
    const int den = 4 * N * M;
    float2* out = J.restr_df + J.restr_off[t];
    for (long long e = threadIdx.x; e < total; e += blockDim.x) {
      const int x = (int)(e / N), i = (int)(e % N);
      const int D = (2 * i + 1) * M - (2 * x + 1) * N;
      df v{1.f, 0.f};
      if (D != 0) {
        const df ssum = df_dot2(sad[i], cgd[x], cad[i], sgd[x]);
        v = df_div(df_mul(sbd[x], cAd[i]), df_mul(df_mul(m2d, ssum), df_sinpi_frac(D, den)));
      }
      out[e] = make_float2(v.hi, v.lo);
    }
    return;
  }
  const double nm4 = 4.0 * (double)N * (double)M, m2 = 2.0 * M;
  for (long long e = threadIdx.x; e < total; e += blockDim.x) {
    const int x = (int)(e / N), i = (int)(e % N);
    const long long D = (long long)(2 * i + 1) * M - (long long)(2 * x + 1) * N;
    double v = 1.0;
    if (D != 0) {
      const double ssum = fma(sa[i], cg[x], ca[i] * sg[x]);
      v = sb[x] * cA[i] / (m2 * ssum * sinpi((double)D / nm4));
    }
    RT[e] = v;
  }
}

// ---------------------------------------------------------------------------------------------
// Self assembly: A_ic = K1(t_i,t_c) Rlog_ic + K2(t_i,t_c) pi/N, symmetric in (i, c), for a band of
// consecutive frequencies sharing N (nodes, log table, |t - s| and its logarithm are shared).
// cos(theta - pi/4) and sin(theta - pi/4) as double-float pairs for a phase theta >= 0 given in FP64 (up
// to ~2e4): theta is reduced by n pi/2 in FP64 (pi/2 as the sum of two doubles, each product inside an
// FMA), the remainder |r| <= pi/4 is rounded to double-float (~3e-15 absolute) and its sine and cosine
// come from the double-float Taylor series; the quadrant n mod 4 permutes them.
__device__ __forceinline__ void df_phase_seed(double theta, df& cx, df& sx) {
  constexpr double kPio2Hi = 1.57079632679489661923, kPio2Lo = 6.123233995736766e-17;   // pi/2 = Hi + Lo
  const double n = rint(theta * kTwoOverPi);
  const double r = fma(-n, kPio2Lo, fma(-n, kPio2Hi, theta));
  df sr, cr;
  df_sincos_taylor(df_from(r), sr, cr);
  df s, c;
  switch (((long long)n) & 3) {
    case 0: s = sr; c = cr; break;
    case 1: s = cr; c = df_neg(sr); break;
    case 2: s = df_neg(sr); c = df_neg(cr); break;
    default: s = df_neg(cr); c = sr; break;
  }
  constexpr df kSqrtHalfD = df_const(0.70710678118654752440084436210484904);
  cx = df_mul(df_add(c, s), kSqrtHalfD);      // cos(theta - pi/4)
  sx = df_mul(df_sub(s, c), kSqrtHalfD);      // sin(theta - pi/4)
}

// A self-matrix entry: FP64, or (mixed form) the double-float pair the refinement reads plus its FP32
// rounding for the FP32 factorisation -- what a separate split of the FP64 matrix would give -- or (the
// FP64-kept form) the FP64 value the FP64 residual reads plus its FP32 rounding.
// Mixed forms: systems that keep FP64 matrices and residuals (all in the FP64-kept form; N >= f64_min_n in
// the mixed form, whose large systems' conditioning would amplify a double-float matrix's rounding).
__device__ __forceinline__ bool sys_f64(const DevJob& J, int N) { return J.fp64keep || N >= J.f64_min_n; }

__device__ __forceinline__ void store_self(const DevJob& J, long long off, double2 v, bool f64) {
  if (f64) {
    J.A[off] = v;
    J.LU32[off] = make_float2(__double2float_rn(v.x), __double2float_rn(v.y));
  } else if (J.mixed) {
    const float4 d = df_split2(v);
    reinterpret_cast<float4*>(J.A)[off] = d;
    J.LU32[off] = make_float2(d.x, d.z);
  } else {
    J.A[off] = v;
  }
}

// P and Q/w of the Hankel asymptotics (kmax + 1 terms each) by Horner's rule in w2 = -1/z^2 in
// double-float.  With |w2| <= 1/400 (z >= 20) the level-k term is below 2^(-8.6 k) of the sum, so the
// levels k >= 3 need only FP32 (22 bits) and the outer three double-float, where each product stays
// far below the coefficient it is added to (no cancellation).
__device__ __forceinline__ void hankel_pq_df(int kmax, df w2, df& P, df& Qa) {
  int k;
  if (kmax >= 3) {
    const float w2f = w2.hi;
    float pf = c_hank_df[2 * kmax].x, qf = c_hank_df[2 * kmax + 1].x;
    for (k = kmax - 1; k >= 3; --k) {
      pf = fmaf(pf, w2f, c_hank_df[2 * k].x);
      qf = fmaf(qf, w2f, c_hank_df[2 * k + 1].x);
    }
    P = df{pf, 0.f};
    Qa = df{qf, 0.f};
    k = 2;
  } else {
    const float2 cp = c_hank_df[2 * kmax], cq = c_hank_df[2 * kmax + 1];
    P = df{cp.x, cp.y};
    Qa = df{cq.x, cq.y};
    k = kmax - 1;
  }
  for (; k >= 0; --k) {
    const float2 cp = c_hank_df[2 * k], cq = c_hank_df[2 * k + 1];
    P = df_add_fast(df_mul(P, w2), df{cp.x, cp.y});
    Qa = df_add_fast(df_mul(Qa, w2), df{cq.x, cq.y});
  }
}

// J0 and Yhat0 for 0 <= z < 20 in double-float (mixed form): the piecewise Taylor expansions of
// bessel0_taylor with double-float coefficients, products and sums.
__device__ __forceinline__ void bessel0_taylor_df(df z, df& J0, df& Yh) {
  const int k = min((int)(2.f * z.hi), kTaylorIntervals - 1);
  const df d = df_add_fast(z, df{-(0.25f + 0.5f * (float)k), 0.f});
  const float2* cj = c_taylor_df[0][k];
  const float2* cy = c_taylor_df[1][k];
  float2 c = __ldg(&cj[kTaylorDegree]);
  df j{c.x, c.y};
  c = __ldg(&cy[kTaylorDegree]);
  df y{c.x, c.y};
#pragma unroll
  for (int n = kTaylorDegree - 1; n >= 0; --n) {
    c = __ldg(&cj[n]);
    j = df_add_fast(df_mul(j, d), df{c.x, c.y});
    c = __ldg(&cy[n]);
    y = df_add_fast(df_mul(y, d), df{c.x, c.y});
  }
  J0 = j;
  Yh = y;
}

__global__ void __launch_bounds__(256) k_assemble_self(DevJob J) {
  const SelfTile tile = J.tiles[blockIdx.x];
  const SysDesc s0 = J.sys[tile.sys];
  const int N = s0.N, nb = tile.nsys;
  // Mixed form: double-float assembly and storage, except for the systems that keep FP64 (sys_f64).
  const bool f64 = J.mixed && sys_f64(J, N);
  const bool df_asm = J.mixed && !f64;
  __shared__ double lnl[kSelfBand], invl[kSelfBand], rsql[kSelfBand];
  __shared__ df invl_d[kSelfBand], rsql_d[kSelfBand], lnl_d[kSelfBand], lh_d[kSelfBand];   // mixed form
  if (threadIdx.x < nb) {
    const double l = (double)(s0.l + threadIdx.x);
    lnl[threadIdx.x] = log(l);
    invl[threadIdx.x] = 1.0 / l;
    rsql[threadIdx.x] = rsqrt(l);
    if (J.mixed) {
      invl_d[threadIdx.x] = df_from(invl[threadIdx.x]);
      rsql_d[threadIdx.x] = df_from(rsql[threadIdx.x]);
      lnl_d[threadIdx.x] = df_from(lnl[threadIdx.x]);
      lh_d[threadIdx.x] = df_from(l * J.h);
    }
  }
  __syncthreads();
  const int i = tile.ti * kSelfTile + (threadIdx.x % kSelfTile);
  const int c = tile.tl * kSelfTile + (threadIdx.x / kSelfTile);
  if (i >= N || c >= N) return;
  if (tile.ti == tile.tl && i > c) return;
  const Panel pn = J.panels[s0.panel];
  const double rl = J.rlog[s0.rlog_off + (long long)i * N + c];
  const double w = kPiD / N;
  const long long e1 = (long long)c * N + i, e2 = (long long)i * N + c;
  if (i == c) {
    const double K1 = -0.5 * kInvPi;
    const double lsp = log(0.5 * J.h * J.node_sp[pn.off + i]);
    for (int b = 0; b < nb; ++b) {
      const double re = -0.5 * kInvPi * (kEulerGamma + lnl[b] + lsp);
      store_self(J, J.sys[tile.sys + b].mat_off + e1, make_double2(fma(K1, rl, re * w), 0.25 * w), f64);
    }
    return;
  }
  const double dx = J.node_x[pn.off + i] - J.node_x[pn.off + c];
  const double dy = J.node_y[pn.off + i] - J.node_y[pn.off + c];
  const double R = sqrt(fma(dx, dx, dy * dy));
  const double dts = fabs(J.node_t[pn.off + i] - J.node_t[pn.off + c]);
  const double hR = J.h * R;
  // A = K1 Rlog + K2 w with K1 = -J0/(2 pi):
  //   z < 20:  K2 = (i/4) J0 - (J0/(2 pi)) [ln l + ln(hR/(2|t-s|)) + gamma] - Yhat0/4
  //   z >= 20: K2 = (i/4) J0 - Y0/4 + (J0/(2 pi)) ln|t-s|
  // so Re A = J0 * alpha - (w/4) Y, with alpha depending on the entry (and on ln l below 20).
  const double lratio = log(hR / (2.0 * dts)) + kEulerGamma;
  const double alpha_a = -0.5 * kInvPi * (rl - w * log(dts));          // z >= 20
  const double qw = 0.25 * w;
  const double inv_u = 1.0 / hR, amp_u = sqrt(kTwoOverPi * inv_u);
  const int lsw = max(s0.l, (int)ceil(kBesselLarge * inv_u));         // first l with z >= 20
  const int lend = s0.l + nb;
  const double zmin = (lsw * J.h) * R;
  const int kmax = hankel_terms((float)zmin);
  if (df_asm) {
    // Mixed form, z < 20: the Taylor range in double-float, alpha = aw ln l + a0.
    const df R_d = df_from(R), qw_d = df_from(qw), aw_d = df_from(-0.5 * kInvPi * w),
             a0_d = df_from(-0.5 * kInvPi * fma(w, lratio, rl));
    for (int l = s0.l; l < min(lsw, lend); ++l) {
      const int b = l - s0.l;
      df J0, Yh;
      bessel0_taylor_df(df_mul(lh_d[b], R_d), J0, Yh);
      const df alpha = df_add_fast(df_mul(aw_d, lnl_d[b]), a0_d);
      const df re = df_dot2(alpha, J0, df_neg(qw_d), Yh);
      const df im = df_mul(qw_d, J0);
      const long long mo = J.sys[tile.sys + b].mat_off;
      const float4 d = make_float4(re.hi, re.lo, im.hi, im.lo);
      const float2 f = make_float2(re.hi, im.hi);
      reinterpret_cast<float4*>(J.A)[mo + e1] = d;
      reinterpret_cast<float4*>(J.A)[mo + e2] = d;
      J.LU32[mo + e1] = f;
      J.LU32[mo + e2] = f;
    }
  } else {
    for (int l = s0.l; l < min(lsw, lend); ++l) {
      const int b = l - s0.l;
      const double z = (l * J.h) * R;
      double J0, Yh;
      bessel0_taylor(z, J0, Yh);
      const double alpha = -0.5 * kInvPi * fma(w, lnl[b] + lratio, rl);
      const double2 v = make_double2(fma(alpha, J0, -qw * Yh), qw * J0);
      const long long mo = J.sys[tile.sys + b].mat_off;
      store_self(J, mo + e1, v, f64);
      store_self(J, mo + e2, v, f64);
    }
  }
  if (df_asm && lsw < lend) {
    // Mixed form: the recurrence above z = 20 in double-float on the FP32 pipe (about 48 bits), stored
    // as the pair and its FP32 rounding; FP64 only for the seeds.  (The FP64-kept form assembles the
    // whole self matrix in FP64, as the plain form does.)
    const df ampu_d = df_from(amp_u), invu_d = df_from(inv_u), alpha_d = df_from(alpha_a), qw_d = df_from(qw);
    df cu_d, su_d;
    if (hR <= 1.0) {
      df_sincos_taylor(df_from(hR), su_d, cu_d);
    } else {
      double su, cu;
      sincos(hR, &su, &cu);
      su_d = df_from(su);
      cu_d = df_from(cu);
    }
    df cx_d{0.f, 0.f}, sx_d{0.f, 0.f};
    int since_d = 16;
    for (int l = lsw; l < lend; ++l) {
      const int b = l - s0.l;
      if (since_d >= 16) {
        df_phase_seed((l * J.h) * R, cx_d, sx_d);
        since_d = 0;
      }
      const df wz = df_mul(invu_d, invl_d[b]);
      const df w2 = df_neg(df_mul(wz, wz));
      df P, Qa;
      hankel_pq_df(kmax, w2, P, Qa);
      Qa = df_mul(Qa, wz);
      const df amp = df_mul(ampu_d, rsql_d[b]);
      const df J0 = df_mul(amp, df_dot2(P, cx_d, Qa, sx_d));
      const df Y0 = df_mul(amp, df_dot2(P, sx_d, df_neg(Qa), cx_d));
      const df re = df_dot2(alpha_d, J0, df_neg(qw_d), Y0);
      const df im = df_mul(qw_d, J0);
      const long long mo = J.sys[tile.sys + b].mat_off;
      const float4 d = make_float4(re.hi, re.lo, im.hi, im.lo);
      const float2 f = make_float2(re.hi, im.hi);
      reinterpret_cast<float4*>(J.A)[mo + e1] = d;
      reinterpret_cast<float4*>(J.A)[mo + e2] = d;
      J.LU32[mo + e1] = f;
      J.LU32[mo + e2] = f;
      const df cn = df_dot2(cx_d, cu_d, df_neg(sx_d), su_d);   // rotation by e^{i h R}
      sx_d = df_dot2(sx_d, cu_d, cx_d, su_d);
      cx_d = cn;
      ++since_d;
    }
    return;
  }
  double su, cu;
  if (hR <= 1.0) sincos_taylor(hR, su, cu);
  else sincos(hR, &su, &cu);
  double cx = 0.0, sx = 0.0;
  int since = 16;
  for (int l = lsw; l < lend; ++l) {
    const int b = l - s0.l;
    if (since >= 16) {
      double sn, cs;
      sincos((l * J.h) * R, &sn, &cs);
      cx = (cs + sn) * kSqrtHalf;
      sx = (sn - cs) * kSqrtHalf;
      since = 0;
    }
    const double wz = inv_u * invl[b];
    const double w2 = -wz * wz;
    double P = c_hank_a[2 * kmax], Qa = c_hank_a[2 * kmax + 1];
    for (int k = kmax - 1; k >= 0; --k) {
      P = fma(P, w2, c_hank_a[2 * k]);
      Qa = fma(Qa, w2, c_hank_a[2 * k + 1]);
    }
    Qa *= wz;
    const double amp = amp_u * rsql[b];
    const double J0 = amp * fma(P, cx, Qa * sx);
    const double Y0 = amp * fma(P, sx, -Qa * cx);
    const double2 v = make_double2(fma(alpha_a, J0, -qw * Y0), qw * J0);
    const long long mo = J.sys[tile.sys + b].mat_off;
    store_self(J, mo + e1, v, f64);
    store_self(J, mo + e2, v, f64);
    const double cn = fma(cx, cu, -sx * su);
    sx = fma(sx, cu, cx * su);
    cx = cn;
    ++since;
  }
}

// ---------------------------------------------------------------------------------------------
// Blocked right-looking LU with partial pivoting (pivot: max |re| + |im|, first index on ties),
// one CTA of 256 threads per system, panel width 8 in shared memory, column-major factor in HBM.
constexpr int kNB = 8;
constexpr int kPS = kNB + 1;   // padded panel row stride (bank-conflict-free column access)
constexpr int kLuThreads = 256;

// C = double2 (plain form: factors J.A in place) or float2 (mixed form: factors J.LU32 in place).  One system
// by the whole CTA (kLuThreads threads); shl_raw: max(N (kNB + kPS), 2 kSB^2) elements of shared memory.
template <class C>
__device__ void lu_one(const DevJob& J, int sidx, unsigned char* shl_raw) {
  C* shl = reinterpret_cast<C*>(shl_raw);
  const SysDesc s = J.sys[sidx];
  const int N = s.N;
  C* A = (sizeof(C) == sizeof(double2) ? reinterpret_cast<C*>(J.A) : reinterpret_cast<C*>(J.LU32)) + s.mat_off;
  int* piv = J.piv + s.piv_off;
  C* Pn = shl;                       // [N][kPS] panel rows
  C* U = shl + (size_t)N * kPS;      // [kNB][N] U12 rows
  __shared__ int spiv[kNB];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int k0 = 0; k0 < N; k0 += kNB) {
    const int w = min(kNB, N - k0);
    const int nr = N - k0;
    for (int idx = tid; idx < nr * w; idx += kLuThreads) {
      int c = idx / nr, r = idx % nr;
      Pn[r * kPS + c] = A[(long long)(k0 + c) * N + k0 + r];
    }
    __syncthreads();
    // The panel's columns by one warp (warp barriers only).
    if (wid == 0) {
      panel_factor_warp<C>(Pn, kPS, nr, w, spiv, lane);
      __syncwarp();
      if (lane < w) piv[k0 + lane] = k0 + spiv[lane];
    }
    __syncthreads();
    for (int idx = tid; idx < nr * w; idx += kLuThreads) {
      int c = idx / nr, r = idx % nr;
      A[(long long)(k0 + c) * N + k0 + r] = Pn[r * kPS + c];
    }
    // Row interchanges on the columns outside the panel.
    for (int col = tid; col < N; col += kLuThreads) {
      if (col >= k0 && col < k0 + w) continue;
      C* Ac = A + (long long)col * N + k0;
      for (int c = 0; c < w; ++c) {
        int p = spiv[c];
        if (p != c) { C t = Ac[c]; Ac[c] = Ac[p]; Ac[p] = t; }
      }
    }
    __syncthreads();
    const int nc = N - k0 - w;
    if (nc > 0) {
      // U12 = L11^{-1} A12 (unit lower triangular solve), one column per thread.
      for (int j = tid; j < nc; j += kLuThreads) {
        C* Ac = A + (long long)(k0 + w + j) * N + k0;
        C xv[kNB];
#pragma unroll
        for (int r = 0; r < kNB; ++r) {
          if (r < w) {
            C v = Ac[r];
            for (int c = 0; c < r; ++c) v = cfms(Pn[r * kPS + c], xv[c], v);
            xv[r] = v;
            Ac[r] = v;
            U[r * N + j] = v;
          }
        }
      }
      __syncthreads();
      // A22 -= L21 U12.
      const int mr = nr - w;
      for (long long idx = tid; idx < (long long)mr * nc; idx += kLuThreads) {
        int j = (int)(idx / mr), r = (int)(idx % mr);
        C* a = A + (long long)(k0 + w + j) * N + k0 + w + r;
        C v = *a;
#pragma unroll
        for (int c = 0; c < kNB; ++c)
          if (c < w) v = cfms(Pn[(w + r) * kPS + c], U[c * N + j], v);
        *a = v;
      }
    }
    __syncthreads();
  }
  lu_finish<C, kLuThreads>(A, N,
                           (sizeof(C) == sizeof(double2) ? reinterpret_cast<C*>(J.dinv) : reinterpret_cast<C*>(J.dinv32)) +
                               s.piv_off,
                           shl);
}

template <class C>
__global__ void __launch_bounds__(kLuThreads) k_lu(DevJob J) {
  extern __shared__ __align__(16) unsigned char shl_raw[];
  lu_one<C>(J, J.lu_small[blockIdx.x], shl_raw);
}

// ---------------------------------------------------------------------------------------------
// Triangular solves, one warp per system, all Q right-hand sides together, in blocks of kSB = 32
// rows: x_b = T_b^{-1} b_b with the inverted diagonal block (a 32 x 32 GEMV, lane = row), then the
// rows beyond the block are updated with the block's columns (independent loads, lane = row).
// ceil(N/32) dependent steps per sweep instead of N.  Both factors have a unit diagonal (U was scaled
// and D^{-1} is applied between the sweeps).  C = double2 (FP64 factors) or float2 (FP32 factors).
constexpr int kSolveWarps = 4;

// Rows i0 and i0 + 32 of every window's b_q -= T[:, r0..r0+w) x_q with x_q = b_q[r0..r0+w), column-major T
// of leading dimension N: each factor entry is loaded once for all QT windows.  Each batch of columns
// issues the loads of both rows before their FMAs, so a lane has 2 x kCols independent loads in flight
// instead of walking its rows one after another.  A second row past `end` is computed on the first and
// not stored.
template <class C, int QT, bool kLean>
__device__ __forceinline__ void tri_update2(C* b, int N, const C* __restrict__ A, int r0, int w, int i0, int end) {
  const int i1 = i0 + 32 < end ? i0 + 32 : i0;
  // columns per load batch: 16 FP32 or 8 FP64 entries per row, halved for 3-4 windows and in lean builds
  // (registers)
  constexpr int kCols = (sizeof(C) == 8 ? 16 : 8) / (QT > 2 ? 2 : 1) / (kLean ? 2 : 1);
  C a0[QT], a1[QT];
#pragma unroll
  for (int q = 0; q < QT; ++q) {
    a0[q] = b[q * N + i0];
    a1[q] = b[q * N + i1];
  }
#pragma unroll 1
  for (int c0 = 0; c0 < kSB; c0 += kCols) {
    C v0[kCols], v1[kCols];
#pragma unroll
    for (int k = 0; k < kCols; ++k) {
      if (c0 + k < w) {
        const C* col = A + (long long)(r0 + c0 + k) * N;
        v0[k] = __ldg(&col[i0]);
        v1[k] = __ldg(&col[i1]);
      }
    }
#pragma unroll
    for (int k = 0; k < kCols; ++k) {
      if (c0 + k < w) {
#pragma unroll
        for (int q = 0; q < QT; ++q) {
          const C x = b[q * N + r0 + c0 + k];
          a0[q] = cfms(v0[k], x, a0[q]);
          a1[q] = cfms(v1[k], x, a1[q]);
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < QT; ++q) {
    b[q * N + i0] = a0[q];
    if (i0 + 32 < end) b[q * N + i0 + 32] = a1[q];
  }
}

// x_q = T_kk^{-1} b_q on the block rows r0 .. r0+w (the diagonal block stored inverted, so a GEMV): lane =
// row, the block's entries loaded once for all QT windows.  lower: the unit-lower block (entries left of
// the diagonal); else the unit-upper one (right of it).
template <class C, int QT, bool kLean>
__device__ __forceinline__ void tri_diag(C* b, int N, const C* __restrict__ A, int r0, int w, int lane, bool lower) {
  constexpr int kH = kLean ? 8 : 16;
  C x[QT];
  if (lane < w) {
#pragma unroll
    for (int q = 0; q < QT; ++q) x[q] = b[q * N + r0 + lane];
#pragma unroll 1
    for (int h = 0; h < kSB; h += kH) {        // kH loads in flight, then their FMAs
      C v[kH];
#pragma unroll
      for (int k = 0; k < kH; ++k) {
        const bool use = lower ? h + k < lane : (h + k > lane && h + k < w);
        if (use) v[k] = __ldg(&A[(long long)(r0 + h + k) * N + r0 + lane]);
      }
#pragma unroll
      for (int k = 0; k < kH; ++k) {
        const bool use = lower ? h + k < lane : (h + k > lane && h + k < w);
        if (use) {
#pragma unroll
          for (int q = 0; q < QT; ++q) x[q] = cfms(make_neg(v[k]), b[q * N + r0 + h + k], x[q]);
        }
      }
    }
  }
  __syncwarp();
  if (lane < w) {
#pragma unroll
    for (int q = 0; q < QT; ++q) b[q * N + r0 + lane] = x[q];
  }
  __syncwarp();
}

// Both triangular sweeps of one system for its QT windows b[q * N + i] (shared memory), one warp (kLean:
// smaller load batches, for kernels with a tighter register budget).
template <class C, int QT, bool kLean = false>
__device__ void tri_solve(C* b, int N, const C* __restrict__ A, const int* __restrict__ piv,
                          const C* __restrict__ dinv, int lane) {
  if (lane < QT) {
    C* bq = b + lane * N;
    for (int k = 0; k < N; ++k) {
      const int p = __ldg(&piv[k]);
      if (p != k) { C t = bq[k]; bq[k] = bq[p]; bq[p] = t; }
    }
  }
  __syncwarp();
  for (int r0 = 0; r0 < N; r0 += kSB) {           // forward, unit lower
    const int w = min(kSB, N - r0), r1 = r0 + w;
    tri_diag<C, QT, kLean>(b, N, A, r0, w, lane, true);
#pragma unroll 1
    for (int i0 = r1 + lane; i0 < N; i0 += 64) tri_update2<C, QT, kLean>(b, N, A, r0, w, i0, N);
    __syncwarp();
  }
  for (int e = lane; e < QT * N; e += 32) b[e] = cmul(b[e], __ldg(&dinv[e % N]));
  __syncwarp();
  for (int r0 = ((N - 1) / kSB) * kSB; r0 >= 0; r0 -= kSB) {   // backward, unit upper
    const int w = min(kSB, N - r0);
    tri_diag<C, QT, kLean>(b, N, A, r0, w, lane, false);
#pragma unroll 1
    for (int i0 = lane; i0 < r0; i0 += 64) tri_update2<C, QT, kLean>(b, N, A, r0, w, i0, r0);
    __syncwarp();
  }
}

// Both sweeps of one system's FP64 factors for all QT windows of step m, by one warp (b: QT x N double2 of
// shared memory), then its densities, their running sum and (kept densities) step m's copy.
template <int QT, bool kLean = false>
__device__ void solve_one(const DevJob& J, int sidx, int m, double2* b, int lane) {
  const SysDesc s = J.sys[sidx];
  const int N = s.N;
  const double2* G = J.G + s.vec_off;
  for (int e = lane; e < QT * N; e += 32) b[e] = G[e];
  __syncwarp();
  tri_solve<double2, QT, kLean>(b, N, J.A + s.mat_off, J.piv + s.piv_off, J.dinv + s.piv_off, lane);
  double2* out = J.phi + s.vec_off;
  double2* sum = J.phi_sum + s.vec_off;
  double2* all = J.phi_all ? J.phi_all + (long long)(m - 1) * J.vec_total + s.vec_off : nullptr;
  for (int e = lane; e < QT * N; e += 32) {
    double2 v = b[e];
    out[e] = v;
    sum[e] = m == 1 ? v : cadd(sum[e], v);
    if (all) all[e] = v;
  }
}

template <int QT>
__global__ void __launch_bounds__(32 * kSolveWarps) k_solve(DevJob J, int m) {
  extern __shared__ double2 shs[];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int slot = blockIdx.x * (blockDim.x >> 5) + wid;
  if (slot >= J.nsys) return;
  solve_one<QT>(J, J.sys_order[slot], m, shs + (size_t)wid * QT * J.max_n, lane);
}

// The FP64 self matrix of one system (plain form) by one CTA: every entry of the upper triangle (diagonal
// included) evaluated for the system's own frequency and stored at both mirror positions -- the same
// log-split rule, Taylor range below z = 20 and Hankel asymptotics above as k_assemble_self, without its
// sharing of the per-pair terms across a band of frequencies.
__device__ void assemble_one(const DevJob& J, int sidx) {
  const SysDesc s = J.sys[sidx];
  const int N = s.N;
  const Panel pn = J.panels[s.panel];
  const double l = (double)s.l, lnl = log(l);
  const double w = kPiD / N, qw = 0.25 * w;
  const long long ntri = (long long)N * (N + 1) / 2;
  for (long long t = threadIdx.x; t < ntri; t += blockDim.x) {
    // t -> (i, c) with i <= c, column by column: c (c + 1) / 2 <= t < (c + 1) (c + 2) / 2
    int c = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((long long)(c + 1) * (c + 2) / 2 <= t) ++c;
    while ((long long)c * (c + 1) / 2 > t) --c;
    const int i = (int)(t - (long long)c * (c + 1) / 2);
    const double rl = J.rlog[s.rlog_off + (long long)i * N + c];
    const long long e1 = (long long)c * N + i, e2 = (long long)i * N + c;
    double2 v;
    if (i == c) {
      const double lsp = log(0.5 * J.h * J.node_sp[pn.off + i]);
      v = make_double2(fma(-0.5 * kInvPi, rl, -0.5 * kInvPi * (kEulerGamma + lnl + lsp) * w), qw);
    } else {
      const double dx = J.node_x[pn.off + i] - J.node_x[pn.off + c];
      const double dy = J.node_y[pn.off + i] - J.node_y[pn.off + c];
      const double R = sqrt(fma(dx, dx, dy * dy));
      const double dts = fabs(J.node_t[pn.off + i] - J.node_t[pn.off + c]);
      const double hR = J.h * R, z = l * hR;
      if (z < kBesselLarge) {
        double J0, Yh;
        bessel0_taylor(z, J0, Yh);
        const double alpha = -0.5 * kInvPi * fma(w, lnl + log(hR / (2.0 * dts)) + kEulerGamma, rl);
        v = make_double2(fma(alpha, J0, -qw * Yh), qw * J0);
      } else {
        double J0, Y0;
        bessel0_asym(z, J0, Y0);
        const double alpha = -0.5 * kInvPi * (rl - w * log(dts));
        v = make_double2(fma(alpha, J0, -qw * Y0), qw * J0);
      }
    }
    J.A[s.mat_off + e1] = v;
    J.A[s.mat_off + e2] = v;
  }
}

// The fused kernel's step-1 solve, one window per warp (a single-window sweep needs few registers), as a
// separate call so that it keeps its own register allocation.
__device__ __noinline__ void fused_solve(const DevJob& J, int sidx, int q, double2* b, int lane) {
  const SysDesc s = J.sys[sidx];
  const int N = s.N;
  const long long o = s.vec_off + (long long)q * N;
  for (int e = lane; e < N; e += 32) b[e] = J.G[o + e];
  __syncwarp();
  tri_solve<double2, 1, true>(b, N, J.A + s.mat_off, J.piv + s.piv_off, J.dinv + s.piv_off, lane);
  double2* all = J.phi_all ? J.phi_all + o : nullptr;   // step 1's copy when densities are kept
  for (int e = lane; e < N; e += 32) {
    const double2 v = b[e];
    J.phi[o + e] = v;
    J.phi_sum[o + e] = v;
    if (all) all[e] = v;
  }
}

// Batching form, plain FP64: one persistent launch assembles, factors and solves (step 1) every (arc, omega)
// system.  Each CTA takes the next system from a work counter (systems by decreasing N, so the largest start
// first and the small ones fill the tail), assembles its matrix, factors it (lu_one) and solves its step-1
// windows, one warp per window; the counter is reset by the host before the launch.
template <int QT>
__global__ void __launch_bounds__(kLuThreads, 2) k_fused_asf(DevJob J, int* counter) {
  extern __shared__ __align__(16) unsigned char shf_raw[];
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= J.nsys) return;
    const int sidx = J.sys_order[item];
    assemble_one(J, sidx);
    __syncthreads();
    lu_one<double2>(J, sidx, shf_raw);
    __syncthreads();
    const int wid = threadIdx.x >> 5;
    if (wid < QT) fused_solve(J, sidx, wid, reinterpret_cast<double2*>(shf_raw) + (size_t)wid * J.max_n, threadIdx.x & 31);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------
// Cross assembly: stored rows of S_Gamma_j for one (pair, frequency band, 8-row chunk).
constexpr int kAsmThreads = 128;   // small blocks: an 8-row task leaves a short last pass
constexpr int kAsmMaxThreads = 256;   // largest cross-assembly block a tuned launch may use
constexpr int kAsmRows = 8;

// A stored cross entry: FP64, or double-float (float4, same 16 bytes) in the mixed-precision form.
__device__ __forceinline__ void store_entry(const DevJob& J, double2* p, double2 v) {
  if (J.mixed) *reinterpret_cast<float4*>(p) = df_split2(v);
  else *p = v;
}
constexpr int kAsmBand = 64;   // frequencies per assembly task (matches the planner's band cap)

// Near-rule product-integration weights of the rows of one task at N source nodes (block-wide, all
// threads call): Wn[r * N + i] = (lambda_0 + 2 sum_n lambda_n T_n(t_i)) / N for the near rows r, with
// lambda_n(t*) = int log|t* - s| T_n(s)/sqrt(1-s^2) ds for |t*| > 1, = -pi zeta^n / n (n >= 1); the sum
// stops where |zeta|^n < 1e-18 (the omitted terms are below 1e-17 of the weights).  ctab: 4N doubles,
// lam: kAsmRows x N doubles of shared memory; Wn may be shared or global memory.
__device__ void near_weights_block(const CrossTgt* tg, int nrows, int N, double* ctab, double* lam, double* Wn) {
  __shared__ int s_nlam[kAsmRows];
  for (int r = threadIdx.x; r < 4 * N; r += blockDim.x) ctab[r] = cospi((double)r / (2.0 * N));
  if (threadIdx.x < nrows && tg[threadIdx.x].near) {
    const double ts = tg[threadIdx.x].tstar;
    const double rt = sqrt(fma(ts, ts, -1.0));
    const double zeta = ts > 0 ? ts - rt : ts + rt;
    double* lr = lam + threadIdx.x * N;
    lr[0] = kPiD * log(0.5 * (fabs(ts) + rt));
    double pw = 1.0;
    int n = 1;
    for (; n < N; ++n) {
      pw *= zeta;
      if (fabs(pw) < 1e-18) break;
      lr[n] = -kPiD * pw / n;
    }
    s_nlam[threadIdx.x] = n;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nrows * N; e += blockDim.x) {
    int r = e / N, i = e % N;
    if (!tg[r].near) continue;
    const double* lr = lam + r * N;
    const int step = 2 * i + 1, mod = 4 * N, nlam = s_nlam[r];
    double acc = 0.0;
    int ph = 0;
    for (int n = 1; n < nlam; ++n) {
      ph += step;
      if (ph >= mod) ph -= mod;
      acc = fma(lr[n], ctab[ph], acc);
    }
    Wn[r * N + i] = (lr[0] + 2.0 * acc) / N;
  }
  __syncthreads();
}

// Quantities of one (target row, source node) pair shared by every frequency of a band.  Every entry,
// near or far, is E = (alpha J0 - (w/4) Y, (w/4) J0) with Y = Yhat0 below z = 20 and Y0 above;
// alpha = A0 + A1 ln l below 20 and beta w/4 above.
//   far rule:  A0 = -(w/(2 pi)) (ln(hR/2) + gamma),  beta = 0;
//   near rule: the log-singular part K1 ln|t* - s| is integrated with the weights wn instead of w,
//              so A0 = -(wn + w (ln(hR/2) + gamma - ln|t* - t_i|))/(2 pi) and
//              beta = -(2/pi)(wn/w - ln|t* - t_i|).
struct PairSetup {
  double R, hR, inv_u, A0, beta;
  int lsw;     // first frequency index with z = l h R >= 20
};

__device__ __forceinline__ PairSetup pair_setup(const DevJob& J, const CrossTgt& t, double xi, double yi, double ti,
                                                double wn, int l0, double w, double invw, double inv_h) {
  PairSetup s;
  const double dx = t.x - xi, dy = t.y - yi;
  const double R2 = fma(dx, dx, dy * dy);
  const double rinv = rsqrt(R2);
  const double R0 = R2 * rinv;
  s.R = fma(fma(-R0, R0, R2), 0.5 * rinv, R0);   // one Newton step on sqrt(R2)
  s.hR = J.h * s.R;
  s.inv_u = rinv * inv_h;                        // 1 / (h R)
  s.lsw = max(l0, (int)ceil(fmin(kBesselLarge * s.inv_u, 1.0e9)));
  s.A0 = 0.0;
  s.beta = 0.0;
  double lt = 0.0;
  if (t.near) {
    lt = log(fabs(t.tstar - ti));
    s.beta = -kTwoOverPi * fma(wn, invw, -lt);
  } else {
    wn = 0.0;
  }
  if (s.lsw > l0) s.A0 = -0.5 * kInvPi * fma(w, log(0.5 * s.hR) + kEulerGamma - lt, wn);
  return s;
}

// Entry at z = (l h) R < 20 from the Taylor tables (lh = l h, lnl = ln l).
__device__ __forceinline__ double2 taylor_entry(const PairSetup& s, double lh, double lnl, double A1, double qw) {
  double J0, Yh;
  bessel0_taylor(lh * s.R, J0, Yh);
  const double alpha = fma(A1, lnl, s.A0);
  return make_double2(fma(alpha, J0, -qw * Yh), qw * J0);
}

// Above z = 20 the Hankel expansion's phase advances by the fixed rotation e^{i h R} from one frequency
// to the next (re-seeded by sincos every 16 steps); 1/z = (1/(hR))(1/l) and sqrt(2/(pi z)) =
// sqrt(2/(pi hR))/sqrt(l); the number of terms follows the first (smallest) z of the run.
struct AsymState {
  double cx, sx;   // cos(z - pi/4), sin(z - pi/4) at the current frequency
  double cu, su;   // the step rotation e^{i h R}
  double ampw;     // sqrt(2/(pi h R)) w/4
  int since, kmax;
};

__device__ __forceinline__ AsymState asym_start(const PairSetup& s, double lh_first, double camp, bool step = true) {
  AsymState a;
  a.ampw = rsqrt(s.hR) * camp;
  a.su = 0.0;
  a.cu = 1.0;
  if (step) {
    if (s.hR <= 1.0) sincos_taylor(s.hR, a.su, a.cu);
    else sincos(s.hR, &a.su, &a.cu);
  }
  a.kmax = hankel_terms((float)(lh_first * s.R));
  a.cx = a.sx = 0.0;
  a.since = 16;
  return a;
}

__device__ __forceinline__ double2 asym_entry(AsymState& a, const PairSetup& s, double lh, double invl, double rsql) {
  if (a.since >= 16) {
    double sn, cs;
    sincos(lh * s.R, &sn, &cs);
    a.cx = (cs + sn) * kSqrtHalf;
    a.sx = (sn - cs) * kSqrtHalf;
    a.since = 0;
  }
  const double wz = s.inv_u * invl;
  const double w2 = -wz * wz;
  double P = c_hank_a[2 * a.kmax], Qa = c_hank_a[2 * a.kmax + 1];
  for (int k = a.kmax - 1; k >= 0; --k) {
    P = fma(P, w2, c_hank_a[2 * k]);
    Qa = fma(Qa, w2, c_hank_a[2 * k + 1]);
  }
  Qa *= wz;
  const double amp = a.ampw * rsql;
  const double t1 = fma(P, a.cx, Qa * a.sx);             // J0 / amp
  const double t2 = fma(P, a.sx, -Qa * a.cx);            // Y0 / amp
  const double cn = fma(a.cx, a.cu, -a.sx * a.su);
  a.sx = fma(a.sx, a.cu, a.cx * a.su);
  a.cx = cn;
  ++a.since;
  return make_double2(amp * fma(s.beta, t1, -t2), amp * t1);
}

// kNear: the launch over the tasks with near rows (shared memory for their product-integration weights);
// otherwise over the far-only tasks, which need only the band tables (more CTAs per SM).  Each launch skips
// the other kind of task.
template <bool kNear>
__global__ void __launch_bounds__(kAsmMaxThreads) k_cross_assemble(DevJob J) {
  extern __shared__ double sha[];
  const CrossAsm task = J.asms[blockIdx.x];
  const PairDesc pr = J.pairs[task.pair];
  const int N = task.N;
  const Panel pn = J.panels[task.panel];
  const CrossTgt* tg = J.tgts + pr.tgt_off + task.row0;
  double* ctab = sha;                                // 4N: cospi(r/(2N))
  double* lam = sha + 4 * N;                         // kAsmRows x N
  double* Wn = kNear ? lam + kAsmRows * N : sha;     // kAsmRows x N near weights (near launch only)
  __shared__ int any_near;
  if (threadIdx.x == 0) {
    int a = 0;
    for (int r = 0; r < task.nrows; ++r) a |= tg[r].near;
    any_near = a;
  }
  __syncthreads();
  if ((any_near != 0) != kNear) return;
  if (kNear) near_weights_block(tg, task.nrows, N, ctab, lam, Wn);
  const double w = kPiD / N, qw = 0.25 * w, invw = N * kInvPi;
  const double A1 = -0.5 * kInvPi * w;          // coefficient of ln l below z = 20
  const double camp = kSqrtTwoOverPi * qw;      // sqrt(2/pi) w/4
  const double inv_h = 1.0 / J.h;
  const int ld = pr.nrows;   // blocks are stored source-major: E[i * nrows + row]
  const int nl = task.l1 - task.l0 + 1;
  // per-band tables: 1/l, 1/sqrt(l), ln l and omega_l = l h
  double* invl = kNear ? Wn + kAsmRows * N : sha;    // <= kAsmBand each
  double* rsql = invl + kAsmBand;
  double* lnl = rsql + kAsmBand;
  double* lh = lnl + kAsmBand;
  df* invl_d = reinterpret_cast<df*>(lh + kAsmBand);      // the same as double-float (mixed form)
  df* rsql_d = invl_d + kAsmBand;
  df* lnl_d = rsql_d + kAsmBand;
  df* lh_d = lnl_d + kAsmBand;
  for (int b = threadIdx.x; b < nl; b += blockDim.x) {
    const int l = task.l0 + b;
    invl[b] = 1.0 / l;
    rsql[b] = rsqrt((double)l);
    lnl[b] = log((double)l);
    lh[b] = l * J.h;
    if (J.mixed) {
      invl_d[b] = df_from(invl[b]);
      rsql_d[b] = df_from(rsql[b]);
      lnl_d[b] = df_from(lnl[b]);
      lh_d[b] = df_from(lh[b]);
    }
  }
  __syncthreads();
  const long long* eo = J.e_off + (long long)task.pair * J.L;
  for (int e = threadIdx.x; e < task.nrows * N; e += blockDim.x) {
    const int r = e % task.nrows, i = e / task.nrows;
    const CrossTgt t = tg[r];
    const PairSetup ps = pair_setup(J, t, J.node_x[pn.off + i], J.node_y[pn.off + i], J.node_t[pn.off + i],
                                    kNear && t.near ? Wn[r * N + i] : 0.0, task.l0, w, invw, inv_h);
    double2* Ep = J.E + (long long)i * ld + task.row0 + r;
    const int lend = min(ps.lsw, task.l1 + 1);
    if (J.mixed && !J.fp64keep) {
      // Mixed form, z < 20: the Taylor range in double-float, stored as double-float pairs.
      const df R_d = df_from(ps.R), A0_d = df_from(ps.A0), A1_d = df_from(A1), qw_d = df_from(qw);
      for (int l = task.l0; l < lend; ++l) {
        const int b = l - task.l0;
        df J0, Yh;
        bessel0_taylor_df(df_mul(lh_d[b], R_d), J0, Yh);
        const df alpha = df_add_fast(df_mul(A1_d, lnl_d[b]), A0_d);
        const df re = df_dot2(alpha, J0, df_neg(qw_d), Yh);
        const df im = df_mul(qw_d, J0);
        *reinterpret_cast<float4*>(Ep + eo[l]) = make_float4(re.hi, re.lo, im.hi, im.lo);
      }
    } else {
      for (int l = task.l0; l < lend; ++l) {
        const int b = l - task.l0;
        store_entry(J, Ep + eo[l], taylor_entry(ps, lh[b], lnl[b], A1, qw));
      }
    }
    if (ps.lsw > task.l1) continue;
    const int lsw = ps.lsw;
    if (J.mixed) {
      // Mixed form: the same recurrence in double-float on the FP32 pipe (about 48 bits), stored as
      // the double-float pairs the mixed-form apply reads; FP64 only for the seeds (the step
      // rotation e^{i h R} itself is evaluated in double-float).
      const AsymState as = asym_start(ps, lh[lsw - task.l0], camp, false);
      const df ampw_d = df_from(as.ampw), invu_d = df_from(ps.inv_u), beta_d = df_from(ps.beta);
      df cu_d, su_d;
      if (ps.hR <= 1.0) {
        df_sincos_taylor(df_from(ps.hR), su_d, cu_d);
      } else {
        double su, cu;
        sincos(ps.hR, &su, &cu);
        su_d = df_from(su);
        cu_d = df_from(cu);
      }
      df cx_d{0.f, 0.f}, sx_d{0.f, 0.f};
      int since_d = 16;
      for (int l = lsw; l <= task.l1; ++l) {
        const int b = l - task.l0;
        if (since_d >= 16) {
          df_phase_seed(lh[b] * ps.R, cx_d, sx_d);
          since_d = 0;
        }
        const df wz = df_mul(invu_d, invl_d[b]);
        const df w2 = df_neg(df_mul(wz, wz));
        df P, Qa;
        hankel_pq_df(as.kmax, w2, P, Qa);
        Qa = df_mul(Qa, wz);
        const df a = df_mul(ampw_d, rsql_d[b]);
        const df t1 = df_dot2(P, cx_d, Qa, sx_d);
        const df t2 = df_dot2(P, sx_d, df_neg(Qa), cx_d);
        const df re = df_mul(a, df_dot2(beta_d, t1, df{-1.f, 0.f}, t2));
        const df im = df_mul(a, t1);
        *reinterpret_cast<float4*>(Ep + eo[l]) = make_float4(re.hi, re.lo, im.hi, im.lo);
        const df cn = df_dot2(cx_d, cu_d, df_neg(sx_d), su_d);   // rotation by e^{i h R}
        sx_d = df_dot2(sx_d, cu_d, cx_d, su_d);
        cx_d = cn;
        ++since_d;
      }
      continue;
    }
    AsymState as = asym_start(ps, lh[lsw - task.l0], camp);
    for (int l = lsw; l <= task.l1; ++l) {
      const int b = l - task.l0;
      store_entry(J, Ep + eo[l], asym_entry(as, ps, lh[b], invl[b], rsql[b]));
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Cross rows evaluated every step (cross_mode 1), nothing stored.  Near weights first, once per job,
// into a table (one slab of nrows x N per assembly task with near rows).
__global__ void __launch_bounds__(kAsmThreads) k_near_weights(DevJob J) {
  const long long off = J.wn_off[blockIdx.x];
  if (off < 0) return;
  extern __shared__ double shn[];
  const CrossAsm task = J.asms[blockIdx.x];
  const CrossTgt* tg = J.tgts + J.pairs[task.pair].tgt_off + task.row0;
  near_weights_block(tg, task.nrows, task.N, shn, shn + 4 * task.N, J.wn + off);
}

// One CTA per (assembly task, band of at most otf_band(Q) frequencies): thread (row r, source group g)
// evaluates the entries of its sources i = g, g + 16, ... for every frequency of the band exactly as
// k_cross_assemble does, multiplies them by the densities of the current step and adds them into its
// own slot of partial sums in shared memory; the 16 partial sums of a row are then added in group
// order (deterministic) into the per-row results, which k_cross_reduce adds per target in block order.
template <int Q>
__global__ void __launch_bounds__(kAsmThreads) k_cross_otf(DevJob J) {
  constexpr int B = OtfBand<Q>::value;
  constexpr int G = kAsmThreads / kAsmRows;          // source groups
  extern __shared__ double2 sho[];                    // [Q * B][G * kAsmRows] partial sums: slot-major, so
                                                      // a warp's read-modify-writes hit consecutive words
  __shared__ double tb[4][B];                         // 1/l, 1/sqrt(l), ln l, l h
  const CrossOtf ot = J.otf_tasks[blockIdx.x];
  const CrossAsm task = J.asms[ot.task];
  const PairDesc pr = J.pairs[task.pair];
  const int N = task.N, nl = ot.l1 - ot.l0 + 1;
  const Panel pn = J.panels[task.panel];
  const CrossTgt* tg = J.tgts + pr.tgt_off + task.row0;
  const long long woff = J.wn_off[ot.task];
  const double* Wn = woff >= 0 ? J.wn + woff : nullptr;
  if (threadIdx.x < nl) {
    const int l = ot.l0 + threadIdx.x;
    tb[0][threadIdx.x] = 1.0 / l;
    tb[1][threadIdx.x] = rsqrt((double)l);
    tb[2][threadIdx.x] = log((double)l);
    tb[3][threadIdx.x] = l * J.h;
  }
  double2* mine = sho + threadIdx.x;                  // slot e at mine[e * kAsmThreads]
  for (int e = 0; e < Q * B; ++e) mine[e * kAsmThreads] = make_double2(0.0, 0.0);
  __syncthreads();
  const double w = kPiD / N, qw = 0.25 * w, invw = N * kInvPi;
  const double A1 = -0.5 * kInvPi * w;
  const double camp = kSqrtTwoOverPi * qw;
  const double inv_h = 1.0 / J.h;
  const int r = threadIdx.x % kAsmRows, g = threadIdx.x / kAsmRows;
  if (r < task.nrows) {
    const CrossTgt t = tg[r];
    const SysDesc* sj = J.sys + (long long)pr.j * (J.L - 1) + (ot.l0 - 1);   // systems (j, l0..l1)
    for (int i = g; i < N; i += G) {
      const PairSetup ps = pair_setup(J, t, J.node_x[pn.off + i], J.node_y[pn.off + i], J.node_t[pn.off + i],
                                      t.near ? Wn[r * N + i] : 0.0, ot.l0, w, invw, inv_h);
      AsymState as{};
      bool started = false;
      for (int b = 0; b < nl; ++b) {
        const int l = ot.l0 + b;
        double2 E;
        if (l < ps.lsw) {
          E = taylor_entry(ps, tb[3][b], tb[2][b], A1, qw);
        } else {
          if (!started) {
            as = asym_start(ps, tb[3][b], camp);
            started = true;
          }
          E = asym_entry(as, ps, tb[3][b], tb[0][b], tb[1][b]);
        }
        const double2* ph = J.phi + sj[b].vec_off + i;
#pragma unroll
        for (int q = 0; q < Q; ++q)
          mine[(q * B + b) * kAsmThreads] = cfma(E, ph[q * N], mine[(q * B + b) * kAsmThreads]);
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < task.nrows * Q * nl; e += kAsmThreads) {
    const int rr = e / (Q * nl), q = (e / nl) % Q, b = e % nl;
    double2 sum = make_double2(0.0, 0.0);
    for (int gg = 0; gg < G; ++gg) sum = cadd(sum, sho[(q * B + b) * kAsmThreads + gg * kAsmRows + rr]);
    const long long row = J.otf_res_off[(long long)task.pair * J.L + ot.l0 + b] + task.row0 + rr;
    J.apply_res[row * Q + q] = sum;
  }
}

// Mixed forms, cross rows evaluated every step in double-float (on the FP32 pipe).  One CTA per (assembly
// task of kAsmRows target rows, band of at most kOtfBandDf frequencies), kOtfDfThreads threads, sources in
// tiles of kOtfDfSrc:
//  1. thread (row r, source i of the tile): the pair's FP64 set-up once (pair_setup), then the entries of
//     every frequency of the band -- below z = 20 the Taylor form (double-float; FP64 rounded to double-float
//     in the FP64-kept form), above it Hankel's expansion with its phase advanced by the double-float
//     rotation e^{i h R} (re-seeded every 16 steps), exactly as the mixed stored-row assembly -- into shared
//     memory; the tile's double-float densities phi(omega_l) are staged beside them;
//  2. thread (row, frequency): sum over the tile's sources of entry x density for every window, with
//     compensated double-float accumulation in source order (deterministic), carried across the tiles.
// The per-row sums go to the per-row results that k_cross_reduce adds per target in block order.
constexpr int kOtfDfSrc = 16;
constexpr int kOtfDfThreads = kAsmRows * kOtfDfSrc;   // 128
constexpr int kOtfDfPitch = kOtfBandDf + 1;           // float4 per shared-memory row (odd: no bank conflicts)

// sin and cos of theta >= 0 (FP64, up to ~2e4) as double-float: theta reduced by n pi/2 in FP64 (pi/2 as the
// sum of two doubles), the remainder's double-float Taylor series, the quadrant n mod 4.
__device__ __forceinline__ void df_sincos_reduced(double theta, df& s, df& c) {
  constexpr double kPio2Hi = 1.57079632679489661923, kPio2Lo = 6.123233995736766e-17;
  const double n = rint(theta * kTwoOverPi);
  const double r = fma(-n, kPio2Lo, fma(-n, kPio2Hi, theta));
  df sr, cr;
  df_sincos_taylor(df_from(r), sr, cr);
  switch (((long long)n) & 3) {
    case 0: s = sr; c = cr; break;
    case 1: s = cr; c = df_neg(sr); break;
    case 2: s = df_neg(sr); c = df_neg(cr); break;
    default: s = df_neg(cr); c = sr; break;
  }
}

// The per-pair quantities of pair_setup on the FP32 pipe (mixed forms, cross rows every step): the distance
// R from the FP64 coordinate differences by a double-float square root, 1/(hR) and the amplitude
// sqrt(2/(pi hR)) w/4 in double-float; FP64 only for the differences, the logarithms of the near rule and
// of the Taylor range (present in the low-frequency bands only) and R itself for the phase reductions.
struct PairDf {
  df R, invu, A0, beta, ampw;
  double R64;
  float hR;
  int lsw;
};

__device__ __forceinline__ PairDf pair_setup_df(const DevJob& J, const CrossTgt& t, double xi, double yi, double ti,
                                                double wn, int l0, double w, double invw, df h_d, df camp_d) {
  PairDf p;
  const double dx = t.x - xi, dy = t.y - yi;
  p.R = df_sqrt(df_from(fma(dx, dx, dy * dy)));
  p.R64 = (double)p.R.hi + (double)p.R.lo;
  const df hR = df_mul(h_d, p.R);
  p.hR = hR.hi;
  p.invu = df_div(df{1.f, 0.f}, hR);
  p.lsw = max(l0, (int)ceilf(fminf((float)kBesselLarge * p.invu.hi, 1.0e9f)));
  double lt = 0.0, beta = 0.0, A0 = 0.0;
  if (t.near) {
    lt = log(fabs(t.tstar - ti));
    beta = -kTwoOverPi * fma(wn, invw, -lt);
  } else {
    wn = 0.0;
  }
  if (p.lsw > l0) A0 = -0.5 * kInvPi * fma(w, log(0.5 * J.h * p.R64) + kEulerGamma - lt, wn);
  p.A0 = df_from(A0);
  p.beta = df_from(beta);
  p.ampw = df_mul(df_rsqrt(hR), camp_d);
  return p;
}

// Double-float state of Hankel's expansion along a band (the mixed stored-row assembly's recurrence).
struct AsymDf {
  df cx, sx, cu, su, ampw, invu, beta;
  int since, kmax;
};

__device__ __forceinline__ AsymDf asym_df_start(const PairDf& p, double lh_first, double h) {
  AsymDf a;
  a.ampw = p.ampw;
  a.invu = p.invu;
  a.beta = p.beta;
  a.kmax = hankel_terms((float)(lh_first * p.R64));
  if (p.hR <= 1.0f) df_sincos_taylor(df_from(h * p.R64), a.su, a.cu);
  else df_sincos_reduced(h * p.R64, a.su, a.cu);
  a.cx = a.sx = df{0.f, 0.f};
  a.since = 16;
  return a;
}

__device__ __forceinline__ float4 asym_df_entry(AsymDf& a, double lhR, df invl, df rsql) {
  if (a.since >= 16) {
    df_phase_seed(lhR, a.cx, a.sx);
    a.since = 0;
  }
  const df wz = df_mul(a.invu, invl);
  const df w2 = df_neg(df_mul(wz, wz));
  df P, Qa;
  hankel_pq_df(a.kmax, w2, P, Qa);
  Qa = df_mul(Qa, wz);
  const df amp = df_mul(a.ampw, rsql);
  const df t1 = df_dot2(P, a.cx, Qa, a.sx);
  const df t2 = df_dot2(P, a.sx, df_neg(Qa), a.cx);
  const df re = df_mul(amp, df_dot2(a.beta, t1, df{-1.f, 0.f}, t2));
  const df im = df_mul(amp, t1);
  const df cn = df_dot2(a.cx, a.cu, df_neg(a.sx), a.su);
  a.sx = df_dot2(a.sx, a.cu, a.cx, a.su);
  a.cx = cn;
  ++a.since;
  return make_float4(re.hi, re.lo, im.hi, im.lo);
}

template <int Q>
__global__ void __launch_bounds__(kOtfDfThreads) k_cross_otf_df(DevJob J) {
  constexpr int B = kOtfBandDf;
  extern __shared__ __align__(16) unsigned char sho_raw[];
  // entries [row][source][band] and densities [window][source][band], rows of kOtfDfPitch float4: a warp
  // of phase 2 (one row or window, 32 frequencies) reads 32 consecutive float4, a warp of phase 1 writes
  // with a 33-float4 stride (both at the minimum of 4 shared-memory wavefronts)
  float4* Et = reinterpret_cast<float4*>(sho_raw);                 // [kAsmRows * kOtfDfSrc][kOtfDfPitch]
  float4* Ps = Et + kAsmRows * kOtfDfSrc * kOtfDfPitch;            // [Q * kOtfDfSrc][kOtfDfPitch]
  __shared__ double tb[4][B];                                       // 1/l, 1/sqrt(l), ln l, l h
  __shared__ df tbd[4][B];                                          // the same as double-float
  __shared__ long long vo[B];                                       // density offsets of the band's systems
  const CrossOtf ot = J.otf_tasks[blockIdx.x];
  const CrossAsm task = J.asms[ot.task];
  const PairDesc pr = J.pairs[task.pair];
  const int N = task.N, nl = ot.l1 - ot.l0 + 1;
  const Panel pn = J.panels[task.panel];
  const CrossTgt* tg = J.tgts + pr.tgt_off + task.row0;
  const long long woff = J.wn_off[ot.task];
  const double* Wn = woff >= 0 ? J.wn + woff : nullptr;
  const int tid = threadIdx.x;
  if (tid < nl) {
    const int l = ot.l0 + tid;
    tb[0][tid] = 1.0 / l;
    tb[1][tid] = rsqrt((double)l);
    tb[2][tid] = log((double)l);
    tb[3][tid] = l * J.h;
    for (int k = 0; k < 4; ++k) tbd[k][tid] = df_from(tb[k][tid]);
    vo[tid] = J.sys[(long long)pr.j * (J.L - 1) + (l - 1)].vec_off;
  }
  __syncthreads();
  const double w = kPiD / N, qw = 0.25 * w, invw = N * kInvPi;
  const double A1 = -0.5 * kInvPi * w;
  const double camp = kSqrtTwoOverPi * qw;
  const double inv_h = 1.0 / J.h;
  const df A1_d = df_from(A1), qw_d = df_from(qw), h_d = df_from(J.h), camp_d = df_from(camp);
  // phase-2 accumulators: thread owns (row, band) pairs p = tid, tid + kOtfDfThreads (row = p / B)
  constexpr int kPairs = kAsmRows * B / kOtfDfThreads;
  dfacc acc_re[kPairs][Q], acc_im[kPairs][Q];
  const int r1 = tid / kOtfDfSrc, i1 = tid % kOtfDfSrc;            // phase-1 pair
  for (int s0 = 0; s0 < N; s0 += kOtfDfSrc) {
    const int i = s0 + i1;
    float4* Ep = Et + (r1 * kOtfDfSrc + i1) * kOtfDfPitch;          // + b
    if (r1 < task.nrows && i < N) {
      const CrossTgt t = tg[r1];
      const double xi = J.node_x[pn.off + i], yi = J.node_y[pn.off + i], ti = J.node_t[pn.off + i];
      const double wni = t.near ? Wn[r1 * N + i] : 0.0;
      const PairDf pd = pair_setup_df(J, t, xi, yi, ti, wni, ot.l0, w, invw, h_d, camp_d);
      const int lend = min(pd.lsw, ot.l1 + 1);
      if (lend > ot.l0) {                                           // z < 20: Taylor form
        PairSetup ps{};
        if (J.fp64keep) ps = pair_setup(J, t, xi, yi, ti, wni, ot.l0, w, invw, inv_h);
        for (int l = ot.l0; l < lend; ++l) {
          const int b = l - ot.l0;
          float4 e;
          if (J.fp64keep) {
            e = df_split2(taylor_entry(ps, tb[3][b], tb[2][b], A1, qw));
          } else {
            df J0, Yh;
            bessel0_taylor_df(df_mul(tbd[3][b], pd.R), J0, Yh);
            const df alpha = df_add_fast(df_mul(A1_d, tbd[2][b]), pd.A0);
            const df re = df_dot2(alpha, J0, df_neg(qw_d), Yh);
            const df im = df_mul(qw_d, J0);
            e = make_float4(re.hi, re.lo, im.hi, im.lo);
          }
          Ep[b] = e;
        }
      }
      if (lend <= ot.l1) {
        AsymDf as = asym_df_start(pd, tb[3][lend - ot.l0], J.h);
        for (int l = lend; l <= ot.l1; ++l) {
          const int b = l - ot.l0;
          Ep[b] = asym_df_entry(as, tb[3][b] * pd.R64, tbd[0][b], tbd[1][b]);
        }
      }
    } else {
      for (int b = 0; b < nl; ++b) Ep[b] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    // the tile's densities phi_q(omega_l)[s0 .. s0 + kOtfDfSrc) (zero past N)
    for (int e = tid; e < nl * Q * kOtfDfSrc; e += kOtfDfThreads) {
      const int ii = e % kOtfDfSrc, q = (e / kOtfDfSrc) % Q, b = e / (kOtfDfSrc * Q);
      Ps[(q * kOtfDfSrc + ii) * kOtfDfPitch + b] =
          s0 + ii < N ? J.phi_df[vo[b] + (long long)q * N + s0 + ii] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kPairs; ++k) {
      const int p = tid + k * kOtfDfThreads, r = p / B, b = p % B;
      if (b < nl) {
        const float4* Er = Et + r * kOtfDfSrc * kOtfDfPitch + b;
        const float4* Pb = Ps + b;
#pragma unroll 4
        for (int ii = 0; ii < kOtfDfSrc; ++ii) {
          const float4 e = Er[ii * kOtfDfPitch];
#pragma unroll
          for (int q = 0; q < Q; ++q) cdf_mac(acc_re[k][q], acc_im[k][q], e, Pb[(q * kOtfDfSrc + ii) * kOtfDfPitch]);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < kPairs; ++k) {
    const int p = tid + k * kOtfDfThreads, r = p / B, b = p % B;
    if (b < nl && r < task.nrows) {
      const long long row = J.otf_res_off[(long long)task.pair * J.L + ot.l0 + b] + task.row0 + r;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const df a = acc_re[k][q].value(), c = acc_im[k][q].value();
        J.apply_res[row * Q + q] = make_double2((double)a.hi + (double)a.lo, (double)c.hi + (double)c.lo);
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Cross apply: W_k(x, q, l) = sum_j sum_i E_{l,k,j}[i, r] phi_j[q, i]; observation sums accumulate.
// One thread per target row, the rows of all source blocks of the group concatenated so that warps
// stay full (on this GPU an FP64 instruction costs a full warp slot of the FP64 pipe whatever its
// active lanes); the source-major blocks make every load coalesced, the densities are shared-memory
// broadcasts, and the per-row sums are added per target in a fixed block order (deterministic).
// The window count is a template parameter so that no FMA is issued for absent windows.
constexpr int kApplyThreads = 256;
constexpr int kApplyMaxBlk = 64;   // receiving groups have at most P <= 64 source blocks

template <int Q>
__global__ void __launch_bounds__(kApplyThreads) k_cross_apply(DevJob J) {
  extern __shared__ double2 shc[];
  const CrossGrp g = J.grps[blockIdx.x];
  const int l = g.l;
  const bool obs = g.k == J.P;
  const int nout = obs ? J.n_obs : J.panels[J.tpanel[g.k]].N;
  const int nb = g.blk_end - g.blk_begin;
  __shared__ int s_row0[kApplyMaxBlk + 1], s_ph0[kApplyMaxBlk + 1];
  if (threadIdx.x == 0) {
    int r = 0, p = 0;
    for (int b = 0; b < nb; ++b) {
      s_row0[b] = r;
      s_ph0[b] = p;
      r += J.blks[g.blk_begin + b].nrows;
      p += Q * J.blks[g.blk_begin + b].N;
    }
    s_row0[nb] = r;
    s_ph0[nb] = p;
  }
  __syncthreads();
  const int nrow = s_row0[nb];
  double2* acc = shc;                              // [Q][nout]
  double2* res = acc + (size_t)Q * J.acc_cap;      // [Q][nrow]
  double2* ph = res + (size_t)Q * J.row_cap;       // concatenated [Q][N_b] densities
  for (int e = threadIdx.x; e < Q * nout; e += kApplyThreads) acc[e] = make_double2(0.0, 0.0);
  for (int b = 0; b < nb; ++b) {
    const CrossBlk B = J.blks[g.blk_begin + b];
    const double2* p = J.phi + J.sys[B.sys].vec_off;
    for (int e = threadIdx.x; e < Q * B.N; e += kApplyThreads) ph[s_ph0[b] + e] = p[e];
  }
  __syncthreads();
  int b = 0;
  for (int row = threadIdx.x; row < nrow; row += kApplyThreads) {
    while (row >= s_row0[b + 1]) ++b;
    const CrossBlk B = J.blks[g.blk_begin + b];
    const int N = B.N, nr = B.nrows, r = row - s_row0[b];
    const double2* phb = ph + s_ph0[b];
    double2 s[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) s[q] = make_double2(0.0, 0.0);
    const double2* __restrict__ Er = J.E + B.e_off + r;
#pragma unroll 4
    for (int i = 0; i < N; ++i) {
      const double2 ev = __ldg(&Er[(long long)i * nr]);
#pragma unroll
      for (int q = 0; q < Q; ++q) s[q] = cfma(ev, phb[q * N + i], s[q]);
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) res[q * nrow + row] = s[q];
  }
  __syncthreads();
  for (int bb = 0; bb < nb; ++bb) {
    const CrossBlk B = J.blks[g.blk_begin + bb];
    for (int r = threadIdx.x; r < B.nrows; r += kApplyThreads) {
      const int out = J.tgts[B.tgt_off + r].out;
#pragma unroll
      for (int q = 0; q < Q; ++q) acc[q * nout + out] = cadd(acc[q * nout + out], res[q * nrow + s_row0[bb] + r]);
    }
    __syncthreads();
  }
  if (obs) {
    for (int e = threadIdx.x; e < Q * nout; e += kApplyThreads) {
      int q = e / nout, z = e % nout;
      double2* v = J.Vobs + ((long long)z * Q + q) * J.L + l;
      *v = cadd(*v, acc[e]);
    }
  } else {
    const long long base = J.tr_off[g.k];
    for (int e = threadIdx.x; e < Q * nout; e += kApplyThreads) {
      int q = e / nout, x = e % nout;
      J.W[((base + x) * Q + q) * J.L + l] = acc[e];
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Mixed-precision solve: an FP32 blocked solve with the FP32 factors, then refinement steps, each a
// residual r = G - A phi (A kept as double-float, about 48 bits; the residual in double-float, or in FP64
// in the FP64-kept form) and an FP32 correction, until the error estimated to remain is below
// J.refine_tol, or J.refine_max steps.  Each step shrinks the error by a factor rho (the FP32 solve's
// relative accuracy), so what remains after a correction of relative size rel is about rho * rel; rho is
// estimated by the ratio of the last two corrections, or after the first step by kFirstRhoSafety * rel
// (that correction is the FP32 solution's own error, about rho times the solution for a generic
// right-hand side; the factor covers large systems, where one right-hand side underestimates rho by up
// to ~10x).  A system still above the tolerance after J.refine_max steps is counted as unconverged.
// A step is two launches over the
// systems still refining: k_mresid streams the double-float matrix with one thread per row (many
// warps in flight per SM), k_msolve runs the triangular solves with one warp per system and little
// register state.  Until a system finishes, its densities sit in its phi slots as double-float pairs
// (16 bytes, the size of the FP64 value written there at the end).
constexpr int kRefineCap = 16;          // largest refine_max accepted
constexpr double kFirstRhoSafety = 10.0;
constexpr int kResidThreads = 128;

// One thread per row (rows past N recompute the last row and store nothing), all Q windows of the row:
// r_q = G_q - A phi_q with compensated double-float sums over the columns in order.
template <int Q>
__global__ void __launch_bounds__(kResidThreads) k_mresid(DevJob J);

// Asynchronous 16-byte copies global -> shared (bypassing L1), for streams whose loads would otherwise
// occupy registers until they land.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int kPending>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(kPending) : "memory");
}

// Per row of the systems that keep FP64, upper bounds of the 1-norm and the 2-norm of the row's 2N real
// components (|Re a_ij|, |Im a_ij|) in FP32, once per job after the assembly: each |a| bounded from above by
// its 23 leading fraction bits times (1 + 2^-22), the sums of 2N such floats (or their squares) by (1 + 2^-10)
// for their roundings (2N 2^-24 < 2^-10), the square root by (1 + 2^-20).  The first-pass residual sizes the
// anchors of its FP32-pipe sums from them.
__device__ __forceinline__ float abs_bound_f32(double a) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(a) & 0x7FFFFFFFFFFFFFFFull;
  const int e = (int)(u >> 52);
  if (e >= 1023 + 127) return __uint_as_float(0x7F800000u);   // beyond FP32 (or not finite): +inf
  if (e < 1023 - 126) return 0x1p-126f;                       // below FP32's normal range
  const unsigned frac23 = (unsigned)(u >> 29) & 0x7FFFFFu;
  return __fmul_rn(__uint_as_float(((unsigned)(e - 1023 + 127) << 23) | frac23), 1.f + 0x1p-22f);
}
__global__ void __launch_bounds__(kResidThreads) k_arow_norms(DevJob J) {
  const int chunk = blockIdx.x * (kResidThreads / 32) + (threadIdx.x >> 5);
  if (chunk >= J.n_rchunks) return;
  const ResidChunk c = J.rchunks[chunk];
  const SysDesc s = J.sys[c.sys];
  const int N = s.N;
  if (!sys_f64(J, N)) return;
  const int i = c.row0 + (threadIdx.x & 31);
  if (i >= N) return;
  const double2* __restrict__ A64 = J.A + s.mat_off;
  float n1 = 0.f, n2 = 0.f;
#pragma unroll 4
  for (int j = 0; j < N; ++j) {
    const double2 a = __ldg(&A64[(long long)j * N + i]);
    const float br = abs_bound_f32(a.x), bi = abs_bound_f32(a.y);
    n1 = __fadd_rn(n1, __fadd_rn(br, bi));
    n2 = fmaf(br, br, fmaf(bi, bi, n2));
  }
  J.arow[s.piv_off + i] =
      make_float2(__fmul_rn(n1, 1.f + 0x1p-10f), __fmul_rn(__fsqrt_rn(__fmul_rn(n2, 1.f + 0x1p-10f)), 1.f + 0x1p-20f));
}

// The first-pass residual of the systems that keep FP64 (all in the FP64-kept form), to FP64 accuracy on both
// arithmetic pipes at once: phi_0 is the FP32 solution (exactly a float), so every product a_ij phi_j can be
// formed exactly from a three-float split of the FP64 entry.  A warp sums its rows either through FP64 FMAs
// (acc) or through those products and anchored sums on the FP32 pipe (aacc, anchors sized per window from
// the smaller of the row's 1-norm times max |phi_0| and its 2-norm times |phi_0|_2); the FP64 pipe, which
// alone would bound the kernel at 8 DFMA per entry and two windows, and the FP32 pipe then work side by
// side.  Either way G - A phi_0 comes out with an error of the order of an FP64 accumulation's (about 2^-50
// of sum_j |a_ij phi_j|).
template <int Q>
__global__ void __launch_bounds__(kResidThreads) k_mresid64(DevJob J) {
  const int chunk = blockIdx.x * (kResidThreads / 32) + (threadIdx.x >> 5);
  if (chunk >= J.n_rchunks) return;
  const ResidChunk c = J.rchunks[chunk];
  if (J.mdone[c.sys]) return;
  const SysDesc s = J.sys[c.sys];
  const int N = s.N;
  if (!sys_f64(J, N)) return;                 // double-float systems: k_mresid
  const int i = c.row0 + (threadIdx.x & 31);
  const int row = i < N ? i : N - 1;
  const double2* __restrict__ A64 = J.A + s.mat_off;
  const double2* __restrict__ ph = J.phi + s.vec_off;       // phi_0 as FP64 (exact)
  const float2* __restrict__ ph32 = J.dcorr + s.vec_off;    // the same values as floats (pass-0 solve)
  const double2* __restrict__ G = J.G + s.vec_off;
  const double isc = 1.0 / J.mscale[c.sys];   // a power of two: exact
  double2 acc[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const double2 g = G[q * N + row];
    acc[q] = make_double2(g.x * isc, g.y * isc);
  }
  // Anchors of the FP32-pipe sums, per window: every partial sum of |a phi_0| along the row (both the real
  // and the imaginary part's 2N terms) stays below bnd = min(|a_i|_1 max |phi_0|, |a_i|_2 |phi_0|_2) (Hoelder,
  // Cauchy-Schwarz; all bounded from above), so below 2^(kh-1) with kh = e + 2 for bnd in [2^e, 2^(e+1)).  A
  // chunk with a row outside the anchors' range sums in FP64.
  const float2 an = J.arow[s.piv_off + row];
  const int km_off = -23 + (32 - __clz(2 * N + 3));       // km = kh - 23 + ceil(log2(T + 4)), T = 2N terms a sum
  bool anchors_ok = true;
  aacc sr[Q], si[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const float2 ps = J.phistat[c.sys * 4 + q];
    const float bnd = __fmul_rn(fminf(__fmul_rn(an.x, ps.x), __fmul_rn(an.y, ps.y)), 1.f + 0x1p-20f);
    const int be = (int)((__float_as_uint(bnd) >> 23) & 0xFFu) - 127;
    const int kh = bnd > 0.f ? be + 2 : 0;                 // (bnd = 0: every product is zero)
    anchors_ok = anchors_ok && (bnd == 0.f || (be >= -40 && be <= 100));
    sr[q].init(kh, kh + km_off);
    si[q].init(kh, kh + km_off);
  }
  auto col64 = [&](const double2 a, int j) {
#pragma unroll
    for (int q = 0; q < Q; ++q) acc[q] = cfms(a, ph[q * N + j], acc[q]);
  };
  auto colx = [&](const double2 a, int j) {
    float r1, r2, r3, i1, i2, i3;
    split3_f64_bits(a.x, r1, r2, r3);
    split3_f64_bits(a.y, i1, i2, i3);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const float2 x = ph32[q * N + j];
      sr[q].add_prod(r1, r2, r3, x.x);          // Re a phi = ar phr - ai phi
      sr[q].add_prod(-i1, -i2, -i3, x.y);
      si[q].add_prod(r1, r2, r3, x.y);          // Im a phi = ar phi + ai phr
      si[q].add_prod(i1, i2, i3, x.x);
    }
  };
  // warps specialise: one of every six 32-row chunks sums in FP64, the rest on the FP32 pipe, so that warps
  // waiting on the FP64 pipe and warps issuing FP32 work share each SM (measured per job, N = 512: one chunk
  // in three on the FP64 pipe 91.6 ms, in four 79.9, in six 76.6, in eight 80.6)
  const bool on_fp32 = (chunk % 6) != 0 && __all_sync(0xffffffffu, anchors_ok);
  int j0 = 0;
  if (on_fp32) {
#pragma unroll 1
    for (; j0 + 4 <= N; j0 += 4) {             // four entries of the row loaded before their sums
      double2 a[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) a[k] = __ldg(&A64[(long long)(j0 + k) * N + row]);
#pragma unroll
      for (int k = 0; k < 4; ++k) colx(a[k], j0 + k);
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        sr[q].renorm();
        si[q].renorm();
      }
    }
    for (; j0 < N; ++j0) colx(__ldg(&A64[(long long)j0 * N + row]), j0);
  } else {
#pragma unroll 1
    for (; j0 + 8 <= N; j0 += 8) {
      double2 a[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) a[k] = __ldg(&A64[(long long)(j0 + k) * N + row]);
#pragma unroll
      for (int k = 0; k < 8; ++k) col64(a[k], j0 + k);
    }
    for (; j0 < N; ++j0) col64(__ldg(&A64[(long long)j0 * N + row]), j0);
  }
  if (i < N) {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const double2 r = make_double2(acc[q].x - sr[q].value(), acc[q].y - si[q].value());
      J.rres[s.vec_off + q * N + i] = make_float2(__double2float_rn(r.x), __double2float_rn(r.y));
      J.rres64[s.vec_off + q * N + i] = r;
    }
  }
}

// Later passes of the systems that keep FP64: the residual of the previous pass updated with its
// correction, r <- r - A d, instead of a new FP64 residual G - A phi (the same value: phi grew by d).  The
// FP64 matrix is split into two floats by integer operations (split_f64_bits) and d is an FP32 vector, so
// every product is formed to about 2^-47 on the FP32 pipe (FMA two-product) and summed with compensated
// double-float sums over the columns in order.  The update's error, about 2^-47 |A| |d|, stays far below
// the FP64 residual's 2^-53 |A| |phi| since the correction d is much smaller than phi; the FP64 pipe does
// one conversion per row.
template <int Q>
__global__ void __launch_bounds__(kResidThreads) k_mresid_upd(DevJob J) {
  const int chunk = blockIdx.x * (kResidThreads / 32) + (threadIdx.x >> 5);
  if (chunk >= J.n_rchunks) return;
  const ResidChunk c = J.rchunks[chunk];
  if (J.mdone[c.sys]) return;
  const SysDesc s = J.sys[c.sys];
  const int N = s.N;
  if (!sys_f64(J, N)) return;                 // double-float systems: k_mresid
  const int i = c.row0 + (threadIdx.x & 31);
  const int row = i < N ? i : N - 1;
  const double2* __restrict__ A64 = J.A + s.mat_off;
  const float2* __restrict__ d = J.dcorr + s.vec_off;
  double2* r64 = J.rres64 + s.vec_off;
  dfacc re[Q], im[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const float4 rd = df_split2(r64[q * N + row]);
    re[q].add(rd.x, rd.y);
    im[q].add(rd.z, rd.w);
  }
  // r -= a d:  Re -= ar dr - ai di,  Im -= ar di + ai dr; kB matrix entries of the row loaded before their sums
  constexpr int kB = Q <= 2 ? 8 : 4;
  auto step = [&](const double2 a, int j) {
    float arh, arl, aih, ail;
    split_f64_bits(a.x, arh, arl);
    split_f64_bits(a.y, aih, ail);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const float2 dv = d[q * N + j];
      dfacc_mac1(re[q], -arh, -arl, dv.x);
      dfacc_mac1(re[q], aih, ail, dv.y);
      dfacc_mac1(im[q], -arh, -arl, dv.y);
      dfacc_mac1(im[q], -aih, -ail, dv.x);
    }
  };
  int j0 = 0;
#pragma unroll 1
  for (; j0 + kB <= N; j0 += kB) {
    double2 a[kB];
#pragma unroll
    for (int k = 0; k < kB; ++k) a[k] = __ldg(&A64[(long long)(j0 + k) * N + row]);
#pragma unroll
    for (int k = 0; k < kB; ++k) step(a[k], j0 + k);
  }
  for (; j0 < N; ++j0) step(__ldg(&A64[(long long)j0 * N + row]), j0);
  if (i < N) {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const df rr = re[q].value(), ri = im[q].value();
      J.rres[s.vec_off + q * N + i] = make_float2(rr.hi + rr.lo, ri.hi + ri.lo);
      r64[q * N + i] = make_double2((double)rr.hi + (double)rr.lo, (double)ri.hi + (double)ri.lo);
    }
  }
}

template <int Q>
__global__ void __launch_bounds__(kResidThreads) k_mresid(DevJob J) {
  const int chunk = blockIdx.x * (kResidThreads / 32) + (threadIdx.x >> 5);
  if (chunk >= J.n_rchunks) return;
  const ResidChunk c = J.rchunks[chunk];
  if (J.mdone[c.sys]) return;
  const SysDesc s = J.sys[c.sys];
  const int N = s.N;
  if (sys_f64(J, N)) return;                  // FP64 systems: k_mresid64
  const int i = c.row0 + (threadIdx.x & 31);
  const int row = i < N ? i : N - 1;
  const float4* __restrict__ Adf = reinterpret_cast<const float4*>(J.A) + s.mat_off;
  const float4* __restrict__ ph = reinterpret_cast<const float4*>(J.phi + s.vec_off);
  const double2* __restrict__ G = J.G + s.vec_off;
  const double isc = 1.0 / J.mscale[c.sys];   // a power of two: exact
  dfacc re[Q], im[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const double2 g = G[q * N + row];
    const float4 gd = df_split2(make_double2(g.x * isc, g.y * isc));
    re[q].add(gd.x, gd.y);
    im[q].add(gd.z, gd.w);
  }
  int j0 = 0;
  if (Q == 1) {
    // 16 matrix entries of the row loaded before their sums; the 16 densities (the same for the whole
    // warp) loaded once by 16 lanes and handed round by shuffles.  Same order of sums as below.
    constexpr int kB = 16;
    const int lane = threadIdx.x & 31;
    for (; j0 + kB <= N; j0 += kB) {
      float4 a[kB];
#pragma unroll
      for (int k = 0; k < kB; ++k) a[k] = __ldg(&Adf[(long long)(j0 + k) * N + row]);
      const float4 pv = ph[j0 + (lane & (kB - 1))];
#pragma unroll
      for (int k = 0; k < kB; ++k) {
        const float4 x = make_float4(__shfl_sync(0xffffffffu, pv.x, k), __shfl_sync(0xffffffffu, pv.y, k),
                                     __shfl_sync(0xffffffffu, pv.z, k), __shfl_sync(0xffffffffu, pv.w, k));
        cdf_mac(re[0], im[0], make_float4(-a[k].x, -a[k].y, -a[k].z, -a[k].w), x);
      }
    }
  }
  constexpr int kUnroll = Q == 1 ? 8 : Q == 2 ? 4 : 2;   // loads in flight without spilling
#pragma unroll kUnroll
  for (int j = j0; j < N; ++j) {
    const float4 a = __ldg(&Adf[(long long)j * N + row]);
    const float4 na = make_float4(-a.x, -a.y, -a.z, -a.w);
#pragma unroll
    for (int q = 0; q < Q; ++q) cdf_mac(re[q], im[q], na, ph[q * N + j]);
  }
  if (i < N) {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const df rr = re[q].value(), ri = im[q].value();
      J.rres[s.vec_off + q * N + i] = make_float2(rr.hi + rr.lo, ri.hi + ri.lo);
    }
  }
}

// pass 0: solve with FP32 G, store phi as double-float (FP64 in the FP64-kept form, whose residual reads
// it), mark the system as refining.  pass p >= 1: solve for the correction from the residual, add it in
// double-float (FP64), and finish the system (FP64 densities, their double-float copy for the cross apply,
// their running sum, the statistics) once the correction is small enough or p = J.refine_max.
template <int QT>
__global__ void __launch_bounds__(32 * kSolveWarps, 3) k_msolve(DevJob J, int m, int pass) {
  extern __shared__ __align__(16) unsigned char shm_raw[];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
  const int slot = blockIdx.x * nw + wid;
  if (slot >= J.nsys) return;
  const int sidx = J.sys_order[slot];
  if (pass > 0 && J.mdone[sidx]) return;
  const SysDesc s = J.sys[sidx];
  const int N = s.N, Q = QT;
  const bool f64 = sys_f64(J, N);            // densities refined in FP64 (FP64 residual)
  float2* b = reinterpret_cast<float2*>(shm_raw) + (size_t)wid * Q * J.max_n;
  const float2* __restrict__ L32 = J.LU32 + s.mat_off;
  const int* __restrict__ piv = J.piv + s.piv_off;
  const float2* __restrict__ dinv = J.dinv32 + s.piv_off;
  float4* ph = reinterpret_cast<float4*>(J.phi + s.vec_off);
  double scale;
  if (pass == 0) {
    // the refinement runs in units of scale = 2^k >= max |G| (exact), so that no data underflow FP32
    const double2* __restrict__ G = J.G + s.vec_off;
    double gmax = 0.0;
    for (int e = lane; e < Q * N; e += 32) gmax = fmax(gmax, fmax(fabs(G[e].x), fabs(G[e].y)));
    for (int o = 16; o > 0; o >>= 1) gmax = fmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
    int ex = 0;
    frexp(gmax, &ex);
    scale = gmax > 0.0 ? ldexp(1.0, ex) : 1.0;
    if (lane == 0) J.mscale[sidx] = scale;
    const double isc = 1.0 / scale;
    for (int e = lane; e < Q * N; e += 32) {
      const double2 g = G[e];
      b[e] = make_float2(__double2float_rn(g.x * isc), __double2float_rn(g.y * isc));
    }
  } else {
    scale = J.mscale[sidx];
    const float2* __restrict__ r = J.rres + s.vec_off;
    for (int e = lane; e < Q * N; e += 32) b[e] = r[e];
  }
  __syncwarp();
  tri_solve<float2, QT>(b, N, L32, piv, dinv, lane);
  double2* ph64 = J.phi + s.vec_off;
  float2* dc = J.dcorr + s.vec_off;
  if (pass == 0) {
    if (f64) {
#pragma unroll
      for (int q = 0; q < QT; ++q) {
        float pm = 0.f, p2 = 0.f;
        for (int e = q * N + lane; e < (q + 1) * N; e += 32) {
          ph64[e] = make_double2(b[e].x, b[e].y);
          dc[e] = b[e];                       // phi_0 as floats for the first residual's FP32-pipe columns
          pm = fmaxf(pm, fmaxf(fabsf(b[e].x), fabsf(b[e].y)));
          p2 = fmaf(b[e].x, b[e].x, fmaf(b[e].y, b[e].y, p2));
        }
        for (int o = 16; o > 0; o >>= 1) {
          pm = fmaxf(pm, __shfl_xor_sync(0xffffffffu, pm, o));
          p2 = __fadd_rn(p2, __shfl_xor_sync(0xffffffffu, p2, o));
        }
        // the first residual's anchors: max |component| and an upper bound of the window's 2-norm
        if (lane == 0)
          J.phistat[sidx * 4 + q] =
              make_float2(pm, __fmul_rn(__fsqrt_rn(__fmul_rn(p2, 1.f + 0x1p-10f)), 1.f + 0x1p-20f));
      }
    } else {
      for (int e = lane; e < Q * N; e += 32) ph[e] = make_float4(b[e].x, 0.f, b[e].y, 0.f);
    }
    if (lane == 0) J.mdone[sidx] = 0;
    return;
  }
  float dmax = 0.f, pmax = 0.f;
  for (int e = lane; e < Q * N; e += 32) {
    const float2 d = b[e];
    if (f64) {
      dc[e] = d;                              // the next pass updates the residual with it
      double2 p = ph64[e];
      p.x += (double)d.x;
      p.y += (double)d.y;
      ph64[e] = p;
      pmax = fmaxf(pmax, fmaxf(fabsf((float)p.x), fabsf((float)p.y)));
    } else {
      float4 p = ph[e];
      float sh, sl;
      two_sum(p.x, d.x, sh, sl);
      quick_two_sum(sh, sl + p.y, p.x, p.y);
      two_sum(p.z, d.y, sh, sl);
      quick_two_sum(sh, sl + p.w, p.z, p.w);
      ph[e] = p;
      pmax = fmaxf(pmax, fmaxf(fabsf(p.x), fabsf(p.z)));
    }
    dmax = fmaxf(dmax, fmaxf(fabsf(d.x), fabsf(d.y)));
  }
  for (int o = 16; o > 0; o >>= 1) {
    dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    pmax = fmaxf(pmax, __shfl_xor_sync(0xffffffffu, pmax, o));
  }
  const double rel = pmax > 0.f ? (double)dmax / (double)pmax : 0.0;
  // contraction factor: after the first correction, twice the largest one measured for this system in an
  // earlier step, else kFirstRhoSafety x rel; later, the ratio of the last two corrections (remembered)
  double rho;
  if (pass == 1) {
    const float known = J.mrho[sidx];
    rho = known > 0.f ? 2.0 * (double)known : kFirstRhoSafety * rel;
  } else {
    rho = rel / fmax((double)J.mrel[sidx], 1e-300);
    if (lane == 0) J.mrho[sidx] = fmaxf(J.mrho[sidx], fminf((float)rho, 1.0f));
  }
  const double left = rel * rho;
  if (left >= J.refine_tol && pass < J.refine_max) {
    if (lane == 0) J.mrel[sidx] = (float)rel;
    return;
  }
  if (lane == 0) {
    J.mdone[sidx] = 1;
    // non-negative doubles and floats order like their bit patterns
    atomicMax(reinterpret_cast<unsigned long long*>(J.refine_resid), (unsigned long long)__double_as_longlong(left));
    atomicAdd(reinterpret_cast<unsigned long long*>(J.refine_resid) + 1, (unsigned long long)pass);
    if (!(left < J.refine_tol)) atomicAdd(reinterpret_cast<unsigned long long*>(J.refine_resid) + 2, 1ULL);
    atomicMax(reinterpret_cast<int*>(J.sys_err) + sidx, __float_as_int(fminf((float)left, 3.0e38f)));
  }
  // Each lane reads back the values it wrote itself (in units of scale) and replaces them by FP64.
  double2* out = J.phi + s.vec_off;
  double2* sum = J.phi_sum + s.vec_off;
  double2* all = J.phi_all ? J.phi_all + (long long)(m - 1) * J.vec_total + s.vec_off : nullptr;
  float4* pdf = J.phi_df + s.vec_off;
  for (int e = lane; e < Q * N; e += 32) {
    double2 v = f64 ? out[e] : df_join2(ph[e]);
    v = make_double2(v.x * scale, v.y * scale);
    pdf[e] = df_split2(v);
    out[e] = v;
    sum[e] = m == 1 ? v : cadd(sum[e], v);
    if (all) all[e] = v;
  }
}

// Entries of a row per batch of the mixed-form cross apply (even: two alternating accumulator sets).
__host__ __device__ constexpr int apply_batch(int Q) { return Q == 1 ? 8 : Q == 2 ? 6 : 4; }
constexpr int kApplyStages = 2;   // batches per thread in shared memory: one summed while the next lands

// Cross apply in double-float on the FP32 pipe (mixed form): E and phi as df64, compensated sums.
// Mixed form, first half: one CTA per slice of kApplySlice rows of a group, one thread per row, the
// row's double-float sum over its block's sources (E and phi as df64, two compensated sums).  The row's
// entries stream through a per-thread ring of kApplyStages batches in shared memory (cp.async): batch
// b + 1 is in flight while batch b is summed, so the loads never wait for the FP32 pipe and hold no
// registers.  A thread reads only the slots it filled itself (no barrier).
template <int Q>
__global__ void __launch_bounds__(kApplySlice, 3) k_cross_rows_df(DevJob J) {
  extern __shared__ __align__(16) float4 she[];     // [kApplyStages][kB][kApplySlice]
  const ApplySlice sl = J.slices[blockIdx.x];
  if ((int)threadIdx.x >= sl.nrows) return;
  const int row = sl.row0 + threadIdx.x;
  // the thread's source block: the slice's blocks hold consecutive rows of the group
  int b = sl.b0, r = row - sl.rowb0;
  while (r >= J.blks[b].nrows) {
    r -= J.blks[b].nrows;
    ++b;
  }
  const CrossBlk B = J.blks[b];
  const int N = B.N, nr = B.nrows;
  // the block's double-float densities, the same for every row: one cached load per warp and column
  const float4* __restrict__ phb = J.phi_df + J.sys[B.sys].vec_off;
  dfacc sr[Q], si[Q], tr[Q], ti[Q];
  const float4* __restrict__ Er = reinterpret_cast<const float4*>(J.E + B.e_off) + r;
  constexpr int kB = apply_batch(Q);
  const int nbat = N / kB;
  float4* mine = she + threadIdx.x;
  auto issue = [&](int bi) {
    float4* dst = mine + (bi % kApplyStages) * kB * kApplySlice;
    const float4* src = Er + (long long)bi * kB * nr;
#pragma unroll
    for (int k = 0; k < kB; ++k) cp_async16(dst + k * kApplySlice, src + (long long)k * nr);
  };
#pragma unroll
  for (int bi = 0; bi < kApplyStages - 1; ++bi) {
    if (bi < nbat) issue(bi);
    cp_async_commit();
  }
#pragma unroll 1
  for (int bi = 0; bi < nbat; ++bi) {
    if (bi + kApplyStages - 1 < nbat) issue(bi + kApplyStages - 1);
    cp_async_commit();                          // (empty near the end: keeps the group count uniform)
    cp_async_wait<kApplyStages - 1>();          // batch bi has landed
    const float4* src = mine + (bi % kApplyStages) * kB * kApplySlice;
    const int i = bi * kB;
#pragma unroll
    for (int k = 0; k < kB; k += 2) {
      const float4 e0 = src[k * kApplySlice], e1 = src[(k + 1) * kApplySlice];
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        cdf_mac(sr[q], si[q], e0, __ldg(&phb[q * N + i + k]));
        cdf_mac(tr[q], ti[q], e1, __ldg(&phb[q * N + i + k + 1]));
      }
    }
  }
  int i = nbat * kB;
  for (; i + 1 < N; i += 2) {
    const float4 e0 = __ldg(&Er[(long long)i * nr]);
    const float4 e1 = __ldg(&Er[(long long)(i + 1) * nr]);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      cdf_mac(sr[q], si[q], e0, __ldg(&phb[q * N + i]));
      cdf_mac(tr[q], ti[q], e1, __ldg(&phb[q * N + i + 1]));
    }
  }
  if (i < N) {
    const float4 e0 = __ldg(&Er[(long long)i * nr]);
#pragma unroll
    for (int q = 0; q < Q; ++q) cdf_mac(sr[q], si[q], e0, __ldg(&phb[q * N + i]));
  }
  double2* out = J.apply_res + (J.grp_res_off[sl.grp] + row) * Q;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    sr[q].add(tr[q].hi, tr[q].lo);
    si[q].add(ti[q].hi, ti[q].lo);
    const df a = sr[q].value(), c = si[q].value();
    out[q] = make_double2((double)a.hi + (double)a.lo, (double)c.hi + (double)c.lo);
  }
}

// Mixed form, second half: per group, the row sums of every source block added to their targets in
// the fixed block order (deterministic), then W (transfer nodes) or the observation spectra.
template <int Q>
__global__ void __launch_bounds__(kApplyThreads) k_cross_reduce(DevJob J) {
  extern __shared__ __align__(16) unsigned char shd_raw[];
  const CrossGrp g = J.grps[blockIdx.x];
  const int l = g.l;
  const bool obs = g.k == J.P;
  const int nout = obs ? J.n_obs : J.panels[J.tpanel[g.k]].N;
  double2* acc = reinterpret_cast<double2*>(shd_raw);      // [Q][nout]
  for (int e = threadIdx.x; e < Q * nout; e += kApplyThreads) acc[e] = make_double2(0.0, 0.0);
  __syncthreads();
  const double2* res = J.apply_res + J.grp_res_off[blockIdx.x] * Q;
  int row0 = 0;
  for (int bb = g.blk_begin; bb < g.blk_end; ++bb) {
    const CrossBlk B = J.blks[bb];
    for (int r = threadIdx.x; r < B.nrows; r += kApplyThreads) {
      const int o = J.tgts[B.tgt_off + r].out;
#pragma unroll
      for (int q = 0; q < Q; ++q) acc[q * nout + o] = cadd(acc[q * nout + o], res[(row0 + r) * Q + q]);
    }
    row0 += B.nrows;
    __syncthreads();
  }
  if (obs) {
    for (int e = threadIdx.x; e < Q * nout; e += kApplyThreads) {
      int q = e / nout, z = e % nout;
      double2* v = J.Vobs + ((long long)z * Q + q) * J.L + l;
      *v = cadd(*v, acc[e]);
    }
  } else {
    const long long base = J.tr_off[g.k];
    for (int e = threadIdx.x; e < Q * nout; e += kApplyThreads) {
      int q = e / nout, x = e % nout;
      J.W[((base + x) * Q + q) * J.L + l] = acc[e];
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Time-domain kernels: one CTA per active transfer node.
constexpr int kTimeThreads = 256;
constexpr int kTimeMaxThreads = 512;   // largest time-transform block a tuned launch may use

// In-place radix-2 decimation-in-time FFT, y_r = sum_b X_b e^{-2 pi i b r/K}; input in
// bit-reversed order.
__device__ void block_fft(double2* buf, int K, int logK, const double2* __restrict__ tw) {
  for (int s = 1; s <= logK; ++s) {
    const int half = 1 << (s - 1);
    const int tws = K >> s;   // twiddle stride
    for (int j = threadIdx.x; j < K / 2; j += blockDim.x) {
      const int pos = j & (half - 1);
      const int i0 = ((j >> (s - 1)) << s) + pos;
      const int i1 = i0 + half;
      const double2 wv = tw[pos * tws];
      const double2 a = buf[i0];
      const double2 bb = cmul(buf[i1], wv);
      buf[i0] = cadd(a, bb);
      buf[i1] = csub(a, bb);
    }
    __syncthreads();
  }
}

// The same FFT in double-float on the FP32 pipe (mixed form): complex values as float4 (re.hi,
// re.lo, im.hi, im.lo), twiddles from a double-float table.
__device__ void block_fft_df(float4* buf, int K, int logK, const float4* __restrict__ tw) {
  for (int s = 1; s <= logK; ++s) {
    const int half = 1 << (s - 1);
    const int tws = K >> s;
    for (int j = threadIdx.x; j < K / 2; j += blockDim.x) {
      const int pos = j & (half - 1);
      const int i0 = ((j >> (s - 1)) << s) + pos;
      const int i1 = i0 + half;
      const float4 a = buf[i0];
      const float4 bb = dfc_mul(buf[i1], tw[pos * tws]);
      buf[i0] = dfc_add(a, bb);
      buf[i1] = dfc_sub(a, bb);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int bitrev(int b, int logK) { return (int)(__brev((unsigned)b) >> (32 - logK)); }

// Transform of the bit-reversed spectrum in buf (FP64, or double-float for DF) and read-back of bin
// r as FP64.
template <bool DF>
__device__ __forceinline__ void fft_in_place(const DevJob& J, double2* buf) {
  if (DF) block_fft_df(reinterpret_cast<float4*>(buf), J.K, J.logK, J.fft_tw_df);
  else block_fft(buf, J.K, J.logK, J.fft_tw);
}
template <bool DF>
__device__ __forceinline__ void fft_put(double2* buf, int i, double2 v) {
  if (DF) reinterpret_cast<float4*>(buf)[i] = df_split2(v);
  else buf[i] = v;
}
template <bool DF>
__device__ __forceinline__ double2 fft_get(const double2* buf, int i) {
  if (DF) return df_join2(reinterpret_cast<const float4*>(buf)[i]);
  return buf[i];
}

// Windowed slow transforms of g[0..NT) into out[q*L + l] (eq. Fourierk with the exact phase split).
template <bool DF>
__device__ void forward_all(const DevJob& J, const double* g, double2* buf, double2* out) {
  const int K = J.K, NT = J.NT, L = J.L;
  for (int q = 0; q < J.Q; ++q) {
    const double* wq = J.win + (long long)q * NT;
    for (int b = threadIdx.x; b < K; b += blockDim.x) {
      double acc = 0.0;
      for (int n = b; n < NT; n += K) acc = fma(g[n], wq[n], acc);
      fft_put<DF>(buf, bitrev(b, J.logK), make_double2(acc, 0.0));
    }
    __syncthreads();
    fft_in_place<DF>(J, buf);
    for (int l = threadIdx.x; l < L; l += blockDim.x) {
      double2 v = make_double2(0.0, 0.0);
      if (l > 0) {
        double2 y = fft_get<DF>(buf, l & (K - 1));
        v = cmul(J.fwd_tw[q * L + l], make_double2(y.x, -y.y));
      }
      out[q * L + l] = v;
    }
    __syncthreads();
  }
}

// Sampled signal: the degree-7 Lagrange interpolant through the samples i0 .. i0 + 7, i0 = floor(s) - 3,
// s = (t - t0)/dt (missing samples count as zero), and 0 outside [t0, t0 + (n_t - 1) dt].  With x = s - i0
// in [3, 4), the weight of sample i0 + k is prod_{m != k} (x - m) / prod_{m != k} (k - m), the numerator
// from prefix and suffix products.
__device__ double sampled_f(const DevJob& J, double t) {
  const double tend = J.sig_t0 + (double)(J.sig_nt - 1) * J.sig_dt;
  if (!(t >= J.sig_t0 && t <= tend)) return 0.0;
  const double s = (t - J.sig_t0) / J.sig_dt;
  const double fl = floor(s);
  const int i0 = (int)fl - 3;
  const double x = s - fl + 3.0;
  constexpr double kDen[8] = {-5040.0, 720.0, -240.0, 144.0, -144.0, 240.0, -720.0, 5040.0};
  double pre[8], suf[8];
  pre[0] = 1.0;
#pragma unroll
  for (int k = 1; k < 8; ++k) pre[k] = pre[k - 1] * (x - (double)(k - 1));
  suf[7] = 1.0;
#pragma unroll
  for (int k = 6; k >= 0; --k) suf[k] = suf[k + 1] * (x - (double)(k + 1));
  double acc = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int i = i0 + k;
    const double fi = (i >= 0 && i < J.sig_nt) ? __ldg(&J.sig_f[i]) : 0.0;
    acc = fma(pre[k] * suf[k] / kDen[k], fi, acc);
  }
  return acc;
}

__device__ __forceinline__ double signal_f(const DevJob& J, double t) {
  if (J.sig_nt > 0) return sampled_f(J, t);
  const double a = (t - J.centre) / J.width;
  return J.amp * sin(J.carrier * t) * exp(-a * a);
}

// u^i at (X, Y) and time t (plane wave, or point source by the trapezoid rule in v).
__device__ double incident_u(const DevJob& J, double X, double Y, double t) {
  if (J.sig_kind == 1) return signal_f(J, t - fma(Y, J.diry, X * J.dirx));
  const double dx = X - J.z0x, dy = Y - J.z0y;
  const double r = sqrt(fma(dx, dx, dy * dy));
  // f(t - tau) can be nonzero for tau in [t - (end of f), t - (start of f)]
  const bool smp = J.sig_nt > 0;
  const double tau_hi = smp ? t - J.sig_t0 : t - J.centre + 8.0 * J.width;
  if (tau_hi <= r) return 0.0;
  const double tau_lo = fmax(r, smp ? t - (J.sig_t0 + (double)(J.sig_nt - 1) * J.sig_dt)
                                    : t - J.centre - 8.0 * J.width);
  if (tau_lo >= tau_hi) return 0.0;
  const double v_lo = acosh(tau_lo / r), v_hi = acosh(tau_hi / r);
  const double band = smp ? J.sig_band : fabs(J.carrier) + 8.0 / J.width;
  const double rate = band * r * sinh(v_hi) + 1.0;
  const int n = (int)ceil((v_hi - v_lo) * (1.25 * rate + 24.0) / (2.0 * kPiD) * 2.0) + 16;
  const double dv = (v_hi - v_lo) / n;
  double acc = 0.5 * (signal_f(J, t - r * cosh(v_lo)) + signal_f(J, t - r * cosh(v_hi)));
  for (int k = 1; k < n; ++k) acc += signal_f(J, t - r * cosh(v_lo + k * dv));
  return acc * dv * (0.5 * kInvPi);
}

// Incident time samples g[a][n] = sign chi_k u^i(x, t_n) at the active transfer nodes, t_n = -H + n dt.
// One thread per run of kIncRun consecutive samples.  Point source with the analytic signal: the
// trapezoid rule in v on the run's common range [v_lo(t_first), v_hi(t_last)] (it contains every sample's
// own range, outside of which f < e^{-64}) with the step of the run's largest rate, and each term of the
// sum advanced from sample to sample by an exact recurrence: with rho = r cosh v and d = t - centre - rho,
// T(t) = e^{i carrier (t - rho)} e^{-(d/width)^2} (so f = amp Im T) satisfies
//   T(t_{j+1}) = T(t_j) u g_j,  u = e^{i carrier dt} e^{-(dt^2 + 2 dt d_0)/width^2},  g_j = e^{-2 j dt^2/width^2}
// from the run's first sample (d_0 = t_first - centre - rho; |d_0| <= 10 width keeps u within e^{+-3}),
// so a term costs one seed (sincos, exp) per run and a complex product per sample.  Runs whose Gaussian
// factor could change by more than e^{-64} within the run (dt kIncRun > 2 width) and sampled signals
// evaluate every sample directly (incident_u).
constexpr int kIncRun = 16;
constexpr int kIncThreads = 128;

__global__ void __launch_bounds__(kIncThreads) k_incident_u(DevJob J) {
  const int a = blockIdx.x;
  const int n0 = (blockIdx.y * kIncThreads + threadIdx.x) * kIncRun;
  if (n0 >= J.NT) return;
  const int nr = min(kIncRun, J.NT - n0);
  const int k = J.act_arc[a], x = J.act_idx[a];
  const Panel pn = J.panels[J.tpanel[k]];
  const double X = J.node_x[pn.off + x], Y = J.node_y[pn.off + x];
  const double pref = J.sign * J.chi[J.tr_off[k] + x];
  double* g = J.ginc + (long long)a * J.NT + n0;
  const bool rec = J.sig_kind == 0 && J.sig_nt == 0 && J.dt * kIncRun <= 2.0 * J.width;
  if (!rec) {
    for (int j = 0; j < nr; ++j) g[j] = pref * incident_u(J, X, Y, -J.H + (n0 + j) * J.dt);
    return;
  }
  const double dx = X - J.z0x, dy = Y - J.z0y;
  const double r = sqrt(fma(dx, dx, dy * dy));
  const double t_first = -J.H + n0 * J.dt, t_last = -J.H + (n0 + nr - 1) * J.dt;
  double acc[kIncRun];
#pragma unroll
  for (int j = 0; j < kIncRun; ++j) acc[j] = 0.0;
  const double tau_hi = t_last - J.centre + 8.0 * J.width;
  const double tau_lo = fmax(r, t_first - J.centre - 8.0 * J.width);
  if (tau_hi > r && tau_lo < tau_hi) {
    const double v_lo = acosh(tau_lo / r), v_hi = acosh(tau_hi / r);
    const double rate = (fabs(J.carrier) + 8.0 / J.width) * r * sinh(v_hi) + 1.0;
    const int n = (int)ceil((v_hi - v_lo) * (1.25 * rate + 24.0) / (2.0 * kPiD) * 2.0) + 16;
    const double dv = (v_hi - v_lo) / n;
    const double iw2 = 1.0 / (J.width * J.width);
    double sa, ca;
    sincos(J.carrier * J.dt, &sa, &ca);
    const double gam = exp(-2.0 * J.dt * J.dt * iw2);
    for (int kk = 0; kk <= n; ++kk) {
      const double rho = r * cosh(fma((double)kk, dv, v_lo));
      const double wgt = (kk == 0 || kk == n) ? 0.5 : 1.0;
      const double d0 = t_first - J.centre - rho;
      double sp, cp;
      sincos(J.carrier * (t_first - rho), &sp, &cp);
      const double e0 = wgt * exp(-d0 * d0 * iw2);
      double2 z = make_double2(e0 * cp, e0 * sp);
      const double b = exp(-(J.dt * J.dt + 2.0 * J.dt * d0) * iw2);
      const double2 u = make_double2(ca * b, sa * b);
      double gj = 1.0;
#pragma unroll
      for (int j = 0; j < kIncRun; ++j) {
        acc[j] += z.y;
        z = cmul(z, make_double2(u.x * gj, u.y * gj));
        gj *= gam;
      }
    }
    const double sc = pref * J.amp * dv * (0.5 * kInvPi);
#pragma unroll
    for (int j = 0; j < kIncRun; ++j) acc[j] *= sc;
  }
  for (int j = 0; j < nr; ++j) g[j] = acc[j];
}

// Slow transforms of the incident samples of one active transfer node (eq. Fourierk per window).
template <bool DF>
__global__ void __launch_bounds__(kTimeMaxThreads) k_incident(DevJob J) {
  extern __shared__ double2 sht[];
  const int a = blockIdx.x;
  const int k = J.act_arc[a], x = J.act_idx[a];
  double2* buf = sht;                               // K
  double* g = reinterpret_cast<double*>(sht + J.K); // NT
  const double* src = J.ginc + (long long)a * J.NT;
  for (int n = threadIdx.x; n < J.NT; n += blockDim.x) g[n] = src[n];
  __syncthreads();
  forward_all<DF>(J, g, buf, J.Gt + (J.tr_off[k] + x) * J.Q * J.L);
}

// PART = 0: the whole step at one transfer node (synthesis, -chi_k, windowed forward transforms).  In a
// frequency-partitioned job the synthesis sums only this rank's frequencies: PART = 1 writes those partial
// samples to J.ginc, the ranks add them, and PART = 2 reads the sums back and finishes the step.
template <bool DF, int PART>
__global__ void __launch_bounds__(kTimeMaxThreads) k_synth_fwd(DevJob J) {
  extern __shared__ double2 sht[];
  const int a = blockIdx.x;
  const int k = J.act_arc[a], x = J.act_idx[a];
  const int K = J.K, L = J.L, NT = J.NT;
  double2* buf = sht;
  double* g = reinterpret_cast<double*>(sht + K);
  const long long base = (J.tr_off[k] + x) * J.Q * L;
  double* gpart = J.ginc + (long long)a * NT;
  if (PART == 2) {
    for (int n = threadIdx.x; n < NT; n += blockDim.x) g[n] = gpart[n];
  } else {
    for (int n = threadIdx.x; n < NT; n += blockDim.x) g[n] = 0.0;
    for (int q = 0; q < J.Q; ++q) {
      const double2* Wq = J.W + base + (long long)q * L;
      const double2* st = J.syn_tw + (long long)q * L;
      for (int b = threadIdx.x; b < K; b += blockDim.x) {
        double2 acc = make_double2(0.0, 0.0);
        for (int l = (b == 0 ? K : b); l < L; l += K) acc = cfma(st[l], Wq[l], acc);
        fft_put<DF>(buf, bitrev(b, J.logK), acc);
      }
      __syncthreads();
      fft_in_place<DF>(J, buf);
      const int n0 = J.nlo[q];
      for (int r = threadIdx.x; r < K; r += blockDim.x) {
        const int n = n0 + r;
        if (n < NT) g[n] += fft_get<DF>(buf, r).x;
      }
      __syncthreads();
    }
    if (PART == 1) {
      for (int n = threadIdx.x; n < NT; n += blockDim.x) gpart[n] = g[n];
      return;
    }
  }
  const double mchi = -J.chi[J.tr_off[k] + x];
  for (int n = threadIdx.x; n < NT; n += blockDim.x) g[n] *= mchi;
  __syncthreads();
  forward_all<DF>(J, g, buf, J.Gt + base);
}

// ---------------------------------------------------------------------------------------------
// Restriction of transfer-mesh spectra to the solve nodes of every system.
constexpr int kRestrThreads = 128;
constexpr int kRestrMaxThreads = 256;   // largest restriction block a tuned launch may use

template <bool DF>
__global__ void __launch_bounds__(kRestrMaxThreads) k_restrict(DevJob J) {
  extern __shared__ double2 shr[];
  const int sidx = J.sys_order[blockIdx.x];
  const SysDesc s = J.sys[sidx];
  const int k = s.arc, l = s.l, N = s.N, Q = J.Q, L = J.L;
  const long long base = J.tr_off[k];
  double2* G = J.G + s.vec_off;
  const long long off = J.restr_of_sys[sidx];
  if (off < 0) {
    for (int e = threadIdx.x; e < Q * N; e += blockDim.x) {
      int q = e / N, i = e % N;
      G[e] = J.Gt[((base + i) * Q + q) * L + l];
    }
    return;
  }
  const int a0 = J.act_off[k], na = J.act_off[k + 1] - a0;
  if constexpr (DF) {
    // Mixed form: the same sums in double-float (spectra split once, compensated sums).
    float4* sh4 = reinterpret_cast<float4*>(shr);
    for (int e = threadIdx.x; e < Q * na; e += blockDim.x) {
      int q = e / na, a = e % na;
      sh4[e] = df_split2(J.Gt[((base + J.act_idx[a0 + a]) * Q + q) * L + l]);
    }
    __syncthreads();
    const float2* RTd = J.restr_df + off;
    for (int e = threadIdx.x; e < Q * N; e += blockDim.x) {
      int q = e / N, i = e % N;
      dfacc re, im;
      for (int a = 0; a < na; ++a) {
        const float2 rv = RTd[(long long)J.act_idx[a0 + a] * N + i];
        const float4 gv = sh4[q * na + a];
        re.mac(rv.x, rv.y, gv.x, gv.y);
        im.mac(rv.x, rv.y, gv.z, gv.w);
      }
      const df vr = re.value(), vi = im.value();
      G[e] = make_double2((double)vr.hi + (double)vr.lo, (double)vi.hi + (double)vi.lo);
    }
  } else {
    for (int e = threadIdx.x; e < Q * na; e += blockDim.x) {
      int q = e / na, a = e % na;
      shr[e] = J.Gt[((base + J.act_idx[a0 + a]) * Q + q) * L + l];
    }
    __syncthreads();
    const double* RT = J.restr + off;
    for (int e = threadIdx.x; e < Q * N; e += blockDim.x) {
      int q = e / N, i = e % N;
      double2 acc = make_double2(0.0, 0.0);
      for (int a = 0; a < na; ++a) {
        const double rv = RT[(long long)J.act_idx[a0 + a] * N + i];
        const double2 gv = shr[q * na + a];
        acc.x = fma(rv, gv.x, acc.x);
        acc.y = fma(rv, gv.y, acc.y);
      }
      G[e] = acc;
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Output traces u_M(z, t) = sum_q [valid] (1/pi) Re sum_l w_l Vobs(z, q, l) e^{-i l h (t - s_q)}.
constexpr int kTraceThreads = 128;

// One block per (observation point, output time): the threads split the frequencies, then a
// fixed-order tree sums their partial sums (deterministic).
__global__ void __launch_bounds__(kTraceThreads) k_traces(DevJob J) {
  __shared__ double part[kTraceThreads];
  const int idx = blockIdx.x;
  const int z = idx / J.n_tout, it = idx % J.n_tout;
  const double t = J.tout[it];
  double acc = 0.0;
  for (int q = 0; q < J.Q; ++q) {
    const double rel = t - J.s_q[q];
    if (!(rel >= -J.H && rel < J.period - J.H)) continue;
    const double c = J.h * (t - J.s_q[q]);
    const double2* V = J.Vobs + ((long long)z * J.Q + q) * J.L;
    for (int l = 1 + threadIdx.x; l < J.L; l += kTraceThreads) {
      double sn, cs;
      sincos((double)l * c, &sn, &cs);
      acc = fma(J.wl[l], fma(V[l].x, cs, V[l].y * sn), acc);
    }
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kTraceThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) J.traces[idx] = part[0] * kInvPi;
}

inline int cdiv(long long a, int b) { return (int)((a + b - 1) / b); }

}  // namespace

// ---------------------------------------------------------------------------------------------
// Launch wrappers

cudaError_t launch_bessel0(const double* z, double* j0, double* y0, double* yh, int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_bessel0<<<cdiv(n, 256), 256, 0, st>>>(z, j0, y0, yh, n);
  return cudaGetLastError();
}

cudaError_t launch_tables(const DevJob& J, cudaStream_t st, int* launches) {
  k_fft_tw<<<cdiv(J.K / 2, 256), 256, 0, st>>>(J.fft_tw, J.fft_tw_df, J.K);
  k_freq_tw<<<cdiv((long long)J.Q * J.L, 256), 256, 0, st>>>(J);
  *launches += 2;
  if (J.n_rlogN > 0) {
    size_t sh = (size_t)5 * J.max_n * sizeof(double);
    cudaFuncSetAttribute(k_rlog, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
    k_rlog<<<J.n_rlogN, 256, sh, st>>>(J);
    *launches += 1;
  }
  if (J.n_restr > 0) {
    const size_t sh = (size_t)3 * (J.max_n + J.max_nmax) * sizeof(double);   // <= 38 KB
    k_restr<<<J.n_restr, 256, sh, st>>>(J);
    *launches += 1;
  }
  return cudaGetLastError();
}

cudaError_t launch_tables_rlog_only(const DevJob& J, cudaStream_t st, int* launches) {
  size_t sh = (size_t)5 * J.max_n * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_rlog, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  k_rlog<<<J.n_rlogN, 256, sh, st>>>(J);
  *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_assemble_self(const DevJob& J, cudaStream_t st, int* launches) {
  if (J.n_tiles > 0) {
    k_assemble_self<<<J.n_tiles, 256, 0, st>>>(J);
    *launches += 1;
  }
  // the row bounds of the FP64 matrices, for the first-pass residual's anchors
  const bool any64 = J.mixed && (J.fp64keep || J.max_n >= J.f64_min_n);
  const int rgrid = cdiv(J.n_rchunks, kResidThreads / 32);
  if (any64 && J.arow && rgrid > 0) {
    k_arow_norms<<<rgrid, kResidThreads, 0, st>>>(J);
    *launches += 1;
  }
  return cudaGetLastError();
}

cudaError_t launch_lu(const DevJob& J, cudaStream_t st, int* launches) {
  cudaError_t e = launch_lu_small(J, st, launches);
  if (e != cudaSuccess || !J.mixed) return e;
  return launch_lu_large(J, st, launches);
}

cudaError_t launch_lu_small(const DevJob& J, cudaStream_t st, int* launches) {
  if (J.mixed) {
    // k_assemble_self already wrote the FP32 matrix and the double-float pairs (or FP64 values)
    if (J.n_lu_small > 0) {
      int small_max = 0;   // systems above kLuBigMin go to the tensor-core path; J.max_n bounds the rest
      small_max = std::min(J.max_n, kLuBigMin - 1);
      size_t sh = std::max((size_t)small_max * (kNB + kPS), (size_t)2 * kSB * kSB) * sizeof(float2);
      cudaError_t e = cudaFuncSetAttribute(k_lu<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
      if (e != cudaSuccess) return e;
      k_lu<float2><<<J.n_lu_small, kLuThreads, sh, st>>>(J);
      *launches += 1;
      return cudaGetLastError();
    }
    return cudaSuccess;
  }
  if (J.n_lu_small == 0) return cudaSuccess;
  size_t sh = std::max((size_t)J.max_n * (kNB + kPS), (size_t)2 * kSB * kSB) * sizeof(double2);
  cudaError_t e = cudaFuncSetAttribute(k_lu<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  k_lu<double2><<<J.n_lu_small, kLuThreads, sh, st>>>(J);
  *launches += 1;
  return cudaGetLastError();
}

template <int QT>
static cudaError_t launch_fused_q(const DevJob& J, int* counter, size_t sh, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_fused_asf<QT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused_asf<QT>, kLuThreads, sh);
  if (e != cudaSuccess) return e;
  const int grid = std::max(1, std::min(J.nsys, sms * std::max(per_sm, 1)));
  e = cudaMemsetAsync(counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  k_fused_asf<QT><<<grid, kLuThreads, sh, st>>>(J, counter);
  return cudaGetLastError();
}

cudaError_t launch_fused_asf(const DevJob& J, int* counter, cudaStream_t st, int* launches) {
  if (J.nsys == 0) return cudaSuccess;
  const size_t sh = std::max((size_t)J.max_n * (kNB + kPS), (size_t)2 * kSB * kSB) * sizeof(double2);
  *launches += 1;
  switch (J.Q) {
    case 1: return launch_fused_q<1>(J, counter, sh, st);
    case 2: return launch_fused_q<2>(J, counter, sh, st);
    case 3: return launch_fused_q<3>(J, counter, sh, st);
    default: return launch_fused_q<4>(J, counter, sh, st);
  }
}

cudaError_t launch_cross_assemble(const DevJob& J, cudaStream_t st, int* launches) {
  if (J.n_asm == 0) return cudaSuccess;
  // Shared layout of k_cross_assemble, in 8-byte words: ctab 4N, lam kAsmRows N, Wn kAsmRows N, then
  // band tables invl, rsql, lnl, lh (doubles) and invl_d, rsql_d, lnl_d, lh_d (double-float pairs),
  // kAsmBand each.
  // (the far-only launch: the band tables alone)
  const size_t sh = ((size_t)(4 + 2 * kAsmRows) * J.max_n + 8 * kAsmBand) * sizeof(double);
  const size_t sh_far = (size_t)8 * kAsmBand * sizeof(double);
  const int nt = J.shape_asm > 0 ? J.shape_asm : kAsmThreads;
  cudaError_t e = cudaFuncSetAttribute(k_cross_assemble<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  k_cross_assemble<true><<<J.n_asm, nt, sh, st>>>(J);
  k_cross_assemble<false><<<J.n_asm, nt, sh_far, st>>>(J);
  *launches += 2;
  return cudaGetLastError();
}

static size_t time_smem(const DevJob& J) { return (size_t)J.K * sizeof(double2) + (size_t)J.NT * sizeof(double); }

cudaError_t launch_incident(const DevJob& J, cudaStream_t st, int* launches) {
  if (J.n_act == 0) return cudaSuccess;
  const int runs = (J.NT + kIncRun - 1) / kIncRun;
  k_incident_u<<<dim3(J.n_act, (runs + kIncThreads - 1) / kIncThreads), kIncThreads, 0, st>>>(J);
  size_t sh = time_smem(J);
  const int nt = J.shape_time > 0 ? J.shape_time : kTimeThreads;
  const bool df = J.mixed && !J.fp64keep;   // double-float FFT butterflies
  cudaError_t e = cudaFuncSetAttribute(df ? k_incident<true> : k_incident<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  if (df) k_incident<true><<<J.n_act, nt, sh, st>>>(J);
  else k_incident<false><<<J.n_act, nt, sh, st>>>(J);
  *launches += 2;
  return cudaGetLastError();
}

template <int PART>
static cudaError_t launch_synth_part(const DevJob& J, cudaStream_t st, int* launches) {
  if (J.n_act == 0) return cudaSuccess;
  size_t sh = time_smem(J);
  const int nt = J.shape_time > 0 ? J.shape_time : kTimeThreads;
  const bool df = J.mixed && !J.fp64keep;   // double-float FFT butterflies
  cudaError_t e = cudaFuncSetAttribute(df ? k_synth_fwd<true, PART> : k_synth_fwd<false, PART>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  if (df) k_synth_fwd<true, PART><<<J.n_act, nt, sh, st>>>(J);
  else k_synth_fwd<false, PART><<<J.n_act, nt, sh, st>>>(J);
  *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_synth_fwd(const DevJob& J, cudaStream_t st, int* launches) {
  return launch_synth_part<0>(J, st, launches);
}
cudaError_t launch_synth_partial(const DevJob& J, cudaStream_t st, int* launches) {
  return launch_synth_part<1>(J, st, launches);
}
cudaError_t launch_fwd_after_sum(const DevJob& J, cudaStream_t st, int* launches) {
  return launch_synth_part<2>(J, st, launches);
}

cudaError_t launch_restrict(const DevJob& J, cudaStream_t st, int* launches) {
  size_t sh = (size_t)J.Q * J.max_nmax * sizeof(double2);
  const int nt = J.shape_restr > 0 ? J.shape_restr : kRestrThreads;
  cudaError_t e = cudaFuncSetAttribute(J.mixed ? k_restrict<true> : k_restrict<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  if (J.nsys == 0) return cudaSuccess;
  if (J.mixed) k_restrict<true><<<J.nsys, nt, sh, st>>>(J);
  else k_restrict<false><<<J.nsys, nt, sh, st>>>(J);
  *launches += 1;
  return cudaGetLastError();
}

// Warps (systems) per solve block: kSolveWarps, fewer when their right-hand sides would not fit in the
// 227 KB of shared memory a block may use (large Q x N).
static int solve_warps(size_t bytes_per_warp, int wanted) {
  const size_t cap = 227 * 1024;
  int nw = wanted > 0 && wanted < kSolveWarps ? wanted : kSolveWarps;
  while (nw > 1 && (size_t)nw * bytes_per_warp > cap) --nw;
  return nw;
}

int refine_passes(const DevJob& J) {
  return J.mixed && J.n_rchunks > 0 ? std::min(std::max(J.refine_max, 1), kRefineCap) : 0;
}

// Mixed forms: the triangular solves of refinement pass `pass` (0: the FP32 solution) for every system
// still refining.
template <int QT>
static cudaError_t launch_msolve_q(const DevJob& J, int m, int pass, cudaStream_t st, int* launches) {
  const size_t per = (size_t)QT * J.max_n * sizeof(float2);
  const int nw = solve_warps(per, J.shape_solve);
  const size_t sh = (size_t)nw * per;
  cudaError_t e = cudaFuncSetAttribute(k_msolve<QT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  k_msolve<QT><<<cdiv(J.nsys, nw), 32 * nw, sh, st>>>(J, m, pass);
  *launches += 1;
  return cudaGetLastError();
}

// Mixed forms: the residuals before refinement pass `pass` >= 1: FP64 for the systems that keep FP64 at
// the first pass, updated with the last correction at later ones (reading of the FP64 residual), double-float
// for the others.
template <int QT>
static cudaError_t launch_resid_q(const DevJob& J, int pass, cudaStream_t st, int* launches) {
  const int rgrid = cdiv(J.n_rchunks, kResidThreads / 32);
  if (rgrid == 0) return cudaSuccess;
  const bool any64 = J.fp64keep || J.max_n >= J.f64_min_n, anydf = !J.fp64keep;
  if (any64 && pass == 1) k_mresid64<QT><<<rgrid, kResidThreads, 0, st>>>(J);
  else if (any64) k_mresid_upd<QT><<<rgrid, kResidThreads, 0, st>>>(J);
  if (anydf) k_mresid<QT><<<rgrid, kResidThreads, 0, st>>>(J);
  *launches += (int)any64 + (int)anydf;
  return cudaGetLastError();
}

template <int QT>
static cudaError_t launch_solve_q(const DevJob& J, int m, cudaStream_t st, int* launches) {
  if (J.mixed) {
    cudaError_t e = launch_msolve_q<QT>(J, m, 0, st, launches);
    for (int pass = 1; pass <= refine_passes(J) && e == cudaSuccess; ++pass) {
      e = launch_resid_q<QT>(J, pass, st, launches);
      if (e == cudaSuccess) e = launch_msolve_q<QT>(J, m, pass, st, launches);
    }
    return e;
  }
  const size_t per = (size_t)QT * J.max_n * sizeof(double2);
  const int nw = solve_warps(per, J.shape_solve);
  size_t sh = (size_t)nw * per;
  cudaError_t e = cudaFuncSetAttribute(k_solve<QT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  k_solve<QT><<<cdiv(J.nsys, nw), 32 * nw, sh, st>>>(J, m);
  *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_solve(const DevJob& J, int m, cudaStream_t st, int* launches) {
  switch (J.Q) {
    case 1: return launch_solve_q<1>(J, m, st, launches);
    case 2: return launch_solve_q<2>(J, m, st, launches);
    case 3: return launch_solve_q<3>(J, m, st, launches);
    default: return launch_solve_q<4>(J, m, st, launches);
  }
}

cudaError_t launch_msolve(const DevJob& J, int m, int pass, cudaStream_t st, int* launches) {
  switch (J.Q) {
    case 1: return launch_msolve_q<1>(J, m, pass, st, launches);
    case 2: return launch_msolve_q<2>(J, m, pass, st, launches);
    case 3: return launch_msolve_q<3>(J, m, pass, st, launches);
    default: return launch_msolve_q<4>(J, m, pass, st, launches);
  }
}

cudaError_t launch_resid(const DevJob& J, int pass, cudaStream_t st, int* launches) {
  switch (J.Q) {
    case 1: return launch_resid_q<1>(J, pass, st, launches);
    case 2: return launch_resid_q<2>(J, pass, st, launches);
    case 3: return launch_resid_q<3>(J, pass, st, launches);
    default: return launch_resid_q<4>(J, pass, st, launches);
  }
}

template <int Q>
static cudaError_t launch_cross_apply_q(const DevJob& J, size_t sh, cudaStream_t st) {
  if (J.mixed) {
    // the row kernel's ring of entry batches (the densities come through the L1 cache)
    const size_t sh_rows = (size_t)kApplyStages * apply_batch(Q) * kApplySlice * sizeof(float4);
    const size_t sh_red = (size_t)Q * J.acc_cap * sizeof(double2);
    cudaError_t e = cudaFuncSetAttribute(k_cross_rows_df<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh_rows);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_cross_reduce<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh_red);
    if (e != cudaSuccess) return e;
    if (J.n_slices > 0) k_cross_rows_df<Q><<<J.n_slices, kApplySlice, sh_rows, st>>>(J);
    k_cross_reduce<Q><<<J.n_grp, kApplyThreads, sh_red, st>>>(J);
    return cudaGetLastError();
  }
  cudaError_t e = cudaFuncSetAttribute(k_cross_apply<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  k_cross_apply<Q><<<J.n_grp, kApplyThreads, sh, st>>>(J);
  return cudaGetLastError();
}

cudaError_t launch_cross_apply(const DevJob& J, cudaStream_t st, int* launches) {
  if (J.n_grp == 0) return cudaSuccess;
  size_t sh = (size_t)J.Q * (J.acc_cap + J.row_cap + J.ph_cap) * sizeof(double2);
  *launches += J.mixed ? 2 : 1;
  switch (J.Q) {
    case 1: return launch_cross_apply_q<1>(J, sh, st);
    case 2: return launch_cross_apply_q<2>(J, sh, st);
    case 3: return launch_cross_apply_q<3>(J, sh, st);
    default: return launch_cross_apply_q<4>(J, sh, st);
  }
}

cudaError_t launch_near_weights(const DevJob& J, cudaStream_t st, int* launches) {
  if (J.n_asm == 0) return cudaSuccess;
  const size_t sh = (size_t)(4 + kAsmRows) * J.max_n * sizeof(double);   // ctab 4N, lam kAsmRows N
  cudaError_t e = cudaFuncSetAttribute(k_near_weights, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  k_near_weights<<<J.n_asm, kAsmThreads, sh, st>>>(J);
  *launches += 1;
  return cudaGetLastError();
}

template <int Q>
static cudaError_t launch_cross_otf_q(const DevJob& J, cudaStream_t st) {
  constexpr int B = OtfBand<Q>::value;
  const size_t sh_red = (size_t)Q * J.acc_cap * sizeof(double2);
  cudaError_t e = cudaFuncSetAttribute(k_cross_reduce<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh_red);
  if (e != cudaSuccess) return e;
  if (J.n_otf > 0) {
    if (J.mixed) {
      const size_t sh = (size_t)kOtfDfPitch * (kAsmRows + Q) * kOtfDfSrc * sizeof(float4);
      e = cudaFuncSetAttribute(k_cross_otf_df<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
      if (e != cudaSuccess) return e;
      k_cross_otf_df<Q><<<J.n_otf, kOtfDfThreads, sh, st>>>(J);
    } else {
      const size_t sh = (size_t)kAsmThreads * Q * B * sizeof(double2);
      k_cross_otf<Q><<<J.n_otf, kAsmThreads, sh, st>>>(J);
    }
  }
  k_cross_reduce<Q><<<J.n_grp, kApplyThreads, sh_red, st>>>(J);
  return cudaGetLastError();
}

cudaError_t launch_cross_otf(const DevJob& J, cudaStream_t st, int* launches) {
  if (J.n_grp == 0) return cudaSuccess;
  *launches += 2;
  switch (J.Q) {
    case 1: return launch_cross_otf_q<1>(J, st);
    case 2: return launch_cross_otf_q<2>(J, st);
    case 3: return launch_cross_otf_q<3>(J, st);
    default: return launch_cross_otf_q<4>(J, st);
  }
}

cudaError_t launch_traces(const DevJob& J, cudaStream_t st, int* launches) {
  int n = J.n_obs * J.n_tout;
  if (n == 0) return cudaSuccess;
  k_traces<<<n, kTraceThreads, 0, st>>>(J);
  *launches += 1;
  return cudaGetLastError();
}

}  // namespace fthms
