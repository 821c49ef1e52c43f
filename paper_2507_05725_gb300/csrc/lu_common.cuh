// Pieces of the blocked LU factorisation shared by the one-CTA-per-system kernel (N <= 800) and the
// large-system path (tensor-core trailing updates): the pivoted factorisation of an 8-column panel by one
// warp, and the finishing pass that prepares a factor for the blocked triangular solves.
#pragma once
#include "cplx.cuh"

namespace fthms {

constexpr int kSB = 32;   // diagonal block of the blocked triangular solves

// Factor the w <= 8 columns of the panel Pn (nr rows, row stride ps, shared memory) in place with partial
// pivoting, by one warp (lane = 0..31; warp barriers only): the pivot of column c is the largest
// |re| + |im| among rows c..nr-1, the lowest row on ties; the rows are swapped inside the panel, the
// column is scaled by the pivot's reciprocal and the panel's remaining columns get the rank-1 update.
// spiv[c] receives the pivot's panel row.
template <class C>
__device__ void panel_factor_warp(C* Pn, int ps, int nr, int w, int* spiv, int lane) {
  using Real = typename CTraits<C>::R;
  for (int c = 0; c < w; ++c) {
    Real best = -1;
    int bi = 0x7fffffff;
    for (int r = c + lane; r < nr; r += 32) {
      C v = Pn[r * ps + c];
      Real m = fabs(v.x) + fabs(v.y);
      if (m > best) { best = m; bi = r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      Real ov = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    const int p = bi == 0x7fffffff ? c : bi;
    if (lane == 0) spiv[c] = p;
    if (p != c && lane < w) {
      C t = Pn[c * ps + lane];
      Pn[c * ps + lane] = Pn[p * ps + lane];
      Pn[p * ps + lane] = t;
    }
    __syncwarp();
    const C inv = crecip(Pn[c * ps + c]);
    for (int r = c + 1 + lane; r < nr; r += 32) {
      C lr = cmul(Pn[r * ps + c], inv);
      Pn[r * ps + c] = lr;
      for (int cc = c + 1; cc < w; ++cc) Pn[r * ps + cc] = cfms(lr, Pn[c * ps + cc], Pn[r * ps + cc]);
    }
    __syncwarp();
  }
}

// The same factorisation by a whole block of NT threads (the same pivots, the same arithmetic per entry, so
// the same factor bit for bit): per column, the pivot search over rows split across the threads (warp
// shuffles, then the NT / 32 warp results in red_m / red_i, reduced by every thread), the swap, then the
// scaling and rank-1 update with rows split across the threads; three block barriers per column.
template <class C, int NT>
__device__ void panel_factor_block(C* Pn, int ps, int nr, int w, int* spiv,
                                   typename CTraits<C>::R* red_m, int* red_i) {
  using Real = typename CTraits<C>::R;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int c = 0; c < w; ++c) {
    Real best = -1;
    int bi = 0x7fffffff;
    for (int r = c + tid; r < nr; r += NT) {
      C v = Pn[r * ps + c];
      Real m = fabs(v.x) + fabs(v.y);
      if (m > best) { best = m; bi = r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      Real ov = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) {
      red_m[wid] = best;
      red_i[wid] = bi;
    }
    __syncthreads();
    best = red_m[0];
    bi = red_i[0];
#pragma unroll
    for (int k = 1; k < NT / 32; ++k) {
      const Real ov = red_m[k];
      const int oi = red_i[k];
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    const int p = bi == 0x7fffffff ? c : bi;
    if (tid == 0) spiv[c] = p;
    if (p != c && tid < w) {
      C t = Pn[c * ps + tid];
      Pn[c * ps + tid] = Pn[p * ps + tid];
      Pn[p * ps + tid] = t;
    }
    __syncthreads();
    const C inv = crecip(Pn[c * ps + c]);
    for (int r = c + 1 + tid; r < nr; r += NT) {
      C lr = cmul(Pn[r * ps + c], inv);
      Pn[r * ps + c] = lr;
      for (int cc = c + 1; cc < w; ++cc) Pn[r * ps + cc] = cfms(lr, Pn[c * ps + cc], Pn[r * ps + cc]);
    }
    __syncthreads();
  }
}

// Finish the factor P A = L U (column-major N x N in A, unit lower L below the diagonal, U on and above)
// for the blocked triangular solves, by all NT threads of a block: U = D U' with unit-diagonal U' (dinv
// receives 1/U_kk, the rows of U right of the diagonal are scaled), then the kSB x kSB diagonal blocks of
// L and of U' are inverted in place.  shl: 2 kSB^2 elements of shared memory.
template <class C, int NT>
__device__ void lu_finish(C* A, int N, C* dinv, C* shl) {
  const int tid = threadIdx.x;
  for (int k = tid; k < N; k += NT) dinv[k] = crecip(A[(long long)k * N + k]);
  __syncthreads();
  for (long long e = tid; e < (long long)N * N; e += NT) {
    const int col = (int)(e / N), row = (int)(e % N);
    if (col > row) A[e] = cmul(A[e], dinv[row]);
  }
  __syncthreads();
  // Invert the kSB x kSB diagonal blocks of the unit-lower L and of the unit-upper U' in place (the
  // strictly lower part of a block holds L^{-1}'s, the strictly upper part U'^{-1}'s), so that the
  // triangular solves take ceil(N/kSB) dependent block steps.  Column c of the inverse of a unit
  // triangular T: X[c][c] = 1, X[i][c] = -sum_k T[i][k] X[k][c] over k between c and i.
  C* T = shl;                      // kSB x kSB block, column-major
  C* Xi = shl + kSB * kSB;
  for (int r0 = 0; r0 < N; r0 += kSB) {
    const int w = min(kSB, N - r0);
    for (int e = tid; e < kSB * kSB; e += NT) {
      const int c = e / kSB, i = e % kSB;
      T[e] = (c < w && i < w) ? A[(long long)(r0 + c) * N + r0 + i] : C{};
    }
    __syncthreads();
    // Xi <- identity; then step k: X[i][c] -= T[i][k] X[k][c] for i > k, c <= k (lower part) and,
    // from the bottom, X[i][c] -= T[i][k'] X[k'][c] for i < k', c >= k' (upper part), k' = w-1-k:
    // all (i, c) pairs of a step in parallel.
    for (int e = tid; e < kSB * kSB; e += NT) Xi[e] = (e / kSB == e % kSB) ? C{1} : C{};
    __syncthreads();
    for (int kk = 0; kk < w - 1; ++kk) {
      const int ku = w - 1 - kk;
      for (int e = tid; e < 2 * kSB * kSB; e += NT) {
        const int half = e / (kSB * kSB), f = e % (kSB * kSB), c = f / kSB, i = f % kSB;
        if (half == 0) {
          if (i > kk && i < w && c <= kk) Xi[c * kSB + i] = cfms(T[kk * kSB + i], Xi[c * kSB + kk], Xi[c * kSB + i]);
        } else {
          if (i < ku && c >= ku && c < w) Xi[c * kSB + i] = cfms(T[ku * kSB + i], Xi[c * kSB + ku], Xi[c * kSB + i]);
        }
      }
      __syncthreads();
    }
    for (int e = tid; e < w * w; e += NT) {
      const int c = e / w, i = e % w;
      if (i != c) A[(long long)(r0 + c) * N + r0 + i] = Xi[c * kSB + i];
    }
    __syncthreads();
  }
}

}  // namespace fthms
