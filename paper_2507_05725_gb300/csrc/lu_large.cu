// FP32 LU factorisation of the large (arc, omega) systems of the mixed forms (N up to 2048): blocked
// right-looking LU with partial pivoting in 32-column outer panels.  Per outer panel, one CTA per system
// factors the panel (8-column inner panels by one warp, as the one-CTA LU does), applies the row
// interchanges to the other columns and computes U12 = L11^{-1} A12; then the trailing update
// A22 -= L21 U12 runs on the tensor cores (tcgen05.mma, kind::tf32, accumulators in tensor memory).
// Algorithm 1 factors each (arc, omega) matrix once and reuses it for every step and window; the FP32
// factor is refined back to FP64 accuracy against the kept matrix (k_msolve / k_mresid).
//
// Trailing update, one CTA per (system, 128 x 128 complex output tile), K = 32 (the outer panel):
//  - complex as real products: Re D = Ar Br - Ai Bi, Im D = Ar Bi + Ai Br (A = L21 tile, B = U12 tile), the
//    minus sign by the instruction descriptor's B negation;
//  - FP32 accuracy from TF32 by the three-term split x = x_hi + x_lo (x_hi = tf32(x), x_lo = tf32(x - x_hi)):
//    A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi, FP32 accumulation;
//  - 8 operand parts (Ar, Ai, Br, Bi) x (hi, lo) of 128 rows x 32 K in shared memory, K-major without
//    swizzle: element (r, k) at byte (r % 8) 16 + (r / 8) 1024 + (k % 4) 4 + (k / 4) 128, so a core matrix
//    (8 rows x 16 bytes) is contiguous, K-adjacent core matrices are 128 bytes apart (leading byte offset)
//    and 8-row groups 1024 bytes apart (stride byte offset); 48 MMAs of 128 x 128 x 8 per tile;
//  - Re D and Im D in TMEM columns [0, 128) and [128, 256) (the CTA holds all 512 columns: one CTA per SM);
//    lane = tile row; the epilogue reads 16 columns at a time and subtracts them from the FP32 factor in
//    HBM (a warp's rows are contiguous there);
//  - the wait for the MMAs is bounded: when it runs out the CTA flags J.dev_err (fthms_wait reports it),
//    frees its tensor memory and returns, and later CTAs return at once.
#include <cstdint>

#include "cplx.cuh"
#include "kernels.h"
#include "lu_common.cuh"
#include "tc.cuh"

namespace fthms {
namespace {

constexpr int kOuter = 32;          // outer panel width = K of the tensor-core update
constexpr int kInner = 8;           // inner panel width (one warp)
constexpr int kInnerPS = kInner + 1;
constexpr int kPanelThreads = 256;
constexpr int kTile = 128;          // complex rows and columns of an update tile
constexpr int kPartBytes = kTile * kOuter * 4;   // 128 x 32 TF32 = 16 KB per operand part
constexpr int kUpdThreads = 256;
constexpr long long kMaxPolls = 1ll << 18;      // bounded wait for the tensor core (well under a second)
constexpr uint32_t kTmemCols = 512;             // the whole tensor memory of the SM (one CTA per SM)
constexpr int kLuThreadsFinish = 256;

// Byte offset of element (r, k) of a 128 x 32 K-major part (see the file comment).
__device__ __forceinline__ int part_off(int r, int k) {
  return (r & 7) * 16 + (r >> 3) * 1024 + (k & 3) * 4 + (k >> 2) * 128;
}

// Outer panel k0 of every large system with N > k0 (kPanelThreads threads per system).
__global__ void __launch_bounds__(kPanelThreads) k_lu_big_panel(DevJob J, int k0) {
  extern __shared__ __align__(16) unsigned char sh_raw[];
  float2* Pn = reinterpret_cast<float2*>(sh_raw);   // [N - k1][kInnerPS] inner panel rows
  __shared__ float2 U[kInner][kOuter];              // inner U12 rows within the outer panel
  __shared__ float2 L11[kOuter][kOuter + 1];        // unit-lower block of the outer panel (row-major)
  __shared__ int spiv[kInner];
  const SysDesc s = J.sys[J.lu_big[blockIdx.x]];
  const int N = s.N;
  if (k0 >= N) return;
  float2* A = J.LU32 + s.mat_off;
  int* piv = J.piv + s.piv_off;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nbo = min(kOuter, N - k0), kend = k0 + nbo;
  for (int k1 = k0; k1 < kend; k1 += kInner) {
    const int w = min(kInner, kend - k1), nr = N - k1;
    for (int idx = tid; idx < nr * w; idx += kPanelThreads) {
      const int c = idx / nr, r = idx % nr;
      Pn[r * kInnerPS + c] = A[(long long)(k1 + c) * N + k1 + r];
    }
    __syncthreads();
    if (wid == 0) {
      panel_factor_warp<float2>(Pn, kInnerPS, nr, w, spiv, lane);
      __syncwarp();
      if (lane < w) piv[k1 + lane] = k1 + spiv[lane];
    }
    __syncthreads();
    for (int idx = tid; idx < nr * w; idx += kPanelThreads) {
      const int c = idx / nr, r = idx % nr;
      A[(long long)(k1 + c) * N + k1 + r] = Pn[r * kInnerPS + c];
    }
    // Row interchanges on the outer panel's other columns (the columns outside it get the panel's
    // interchanges all at once below).
    for (int col = k0 + tid; col < kend; col += kPanelThreads) {
      if (col >= k1 && col < k1 + w) continue;
      float2* Ac = A + (long long)col * N + k1;
      for (int c = 0; c < w; ++c) {
        const int p = spiv[c];
        if (p != c) {
          const float2 t = Ac[c];
          Ac[c] = Ac[p];
          Ac[p] = t;
        }
      }
    }
    __syncthreads();
    // The outer panel's remaining columns: U12 rows of this inner panel, then the rank-w update.
    const int j0 = k1 + w, nc = kend - j0;
    if (nc > 0) {
      for (int j = tid; j < nc; j += kPanelThreads) {
        float2* Ac = A + (long long)(j0 + j) * N + k1;
        float2 x[kInner];
#pragma unroll
        for (int r = 0; r < kInner; ++r) {
          if (r < w) {
            float2 v = Ac[r];
            for (int c = 0; c < r; ++c) v = cfms(Pn[r * kInnerPS + c], x[c], v);
            x[r] = v;
            Ac[r] = v;
            U[r][j] = v;
          }
        }
      }
      __syncthreads();
      const int mr = nr - w;
      for (long long idx = tid; idx < (long long)mr * nc; idx += kPanelThreads) {
        const int j = (int)(idx / mr), r = (int)(idx % mr);
        float2* a = A + (long long)(j0 + j) * N + j0 + r;
        float2 v = *a;
#pragma unroll
        for (int c = 0; c < kInner; ++c)
          if (c < w) v = cfms(Pn[(w + r) * kInnerPS + c], U[c][j], v);
        *a = v;
      }
    }
    __syncthreads();
  }
  // The panel's interchanges on every column outside it, in order (rows k and piv[k], k = k0 .. kend-1): a
  // column's rows k0 .. kend-1 in a per-thread segment of shared memory (the inner-panel buffer, free
  // now; element r of thread t at seg[r * kPanelThreads + t], conflict-free), pivot rows below them in
  // HBM; then, right of the panel, U12 = L11^{-1} A12 on those rows in registers (static indices only).
  __shared__ int pv[kOuter];
  for (int e = tid; e < nbo * nbo; e += kPanelThreads) {
    const int c = e / nbo, r = e % nbo;
    L11[r][c] = A[(long long)(k0 + c) * N + k0 + r];
  }
  if (tid < nbo) pv[tid] = piv[k0 + tid] - k0;
  __syncthreads();
  float2* seg = Pn;
  for (int col = tid; col < N - nbo; col += kPanelThreads) {
    const int cc = col < k0 ? col : col + nbo;        // skip the panel's own columns
    float2* Ac = A + (long long)cc * N + k0;
    for (int r = 0; r < nbo; ++r) seg[r * kPanelThreads + tid] = Ac[r];
    for (int c = 0; c < nbo; ++c) {
      const int p = pv[c];
      if (p == c) continue;
      const float2 t = p < nbo ? seg[p * kPanelThreads + tid] : Ac[p];
      if (p < nbo) seg[p * kPanelThreads + tid] = seg[c * kPanelThreads + tid];
      else Ac[p] = seg[c * kPanelThreads + tid];
      seg[c * kPanelThreads + tid] = t;
    }
    if (cc >= kend) {
      float2 x[kOuter];
#pragma unroll
      for (int r = 0; r < kOuter; ++r) x[r] = r < nbo ? seg[r * kPanelThreads + tid] : make_float2(0.f, 0.f);
#pragma unroll
      for (int r = 1; r < kOuter; ++r) {
#pragma unroll
        for (int c = 0; c < r; ++c) x[r] = cfms(L11[r][c], x[c], x[r]);
      }
#pragma unroll
      for (int r = 0; r < kOuter; ++r)
        if (r < nbo) Ac[r] = x[r];
    } else {
      for (int r = 0; r < nbo; ++r) Ac[r] = seg[r * kPanelThreads + tid];
    }
  }
}

// One operand part element: the TF32 value and its TF32 remainder.
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  hi = tc::to_tf32(x);
  lo = tc::to_tf32(x - hi);
}

// Trailing update A22 -= L21 U12 after outer panel k0: blockIdx.x = large system, blockIdx.y = tile.
__global__ void __launch_bounds__(kUpdThreads, 1) k_lu_big_update(DevJob J, int k0) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_base;
  const SysDesc s = J.sys[J.lu_big[blockIdx.x]];
  const int N = s.N;
  const int T = N - k0 - kOuter;                  // trailing size
  if (T <= 0) return;
  const int tm = (T + kTile - 1) / kTile;
  if ((int)blockIdx.y >= tm * tm) return;
  if (*(volatile int*)J.dev_err) return;         // an earlier wait ran out: the factor is void anyway
  const int R0 = k0 + kOuter + kTile * ((int)blockIdx.y / tm), C0 = k0 + kOuter + kTile * ((int)blockIdx.y % tm);
  float2* A = J.LU32 + s.mat_off;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // parts: 0 Ar_hi, 1 Ar_lo, 2 Ai_hi, 3 Ai_lo, 4 Br_hi, 5 Br_lo, 6 Bi_hi, 7 Bi_lo
  unsigned char* part = sm;
  if (wid == 0) tc::tmem_alloc(&tmem_base, kTmemCols);
  if (tid == 0) tc::mbar_init(&bar, 1);
  // L21 tile: rows R0 .. R0+127 of columns k0 .. k0+31 (thread = row and half of K; zero beyond N), the 16
  // loads of a thread issued before their splits.
  {
    const int r = tid & (kTile - 1), kh = (tid >> 7) * (kOuter / 2), row = R0 + r;
    float2 v[kOuter / 2];
#pragma unroll
    for (int k = 0; k < kOuter / 2; ++k)
      v[k] = row < N ? A[(long long)(k0 + kh + k) * N + row] : make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < kOuter / 2; ++k) {
      float h, l;
      const int o = part_off(r, kh + k);
      split_tf32(v[k].x, h, l);
      *reinterpret_cast<float*>(part + 0 * kPartBytes + o) = h;
      *reinterpret_cast<float*>(part + 1 * kPartBytes + o) = l;
      split_tf32(v[k].y, h, l);
      *reinterpret_cast<float*>(part + 2 * kPartBytes + o) = h;
      *reinterpret_cast<float*>(part + 3 * kPartBytes + o) = l;
    }
  }
  // U12 tile: rows k0 .. k0+31 of columns C0 .. C0+127 as a 128 (column) x 32 (k) K-major operand
  // (warp = column, lane = k: each column's 32 values are contiguous in HBM), 4 columns in flight per warp.
  for (int n0 = wid; n0 < kTile; n0 += 4 * (kUpdThreads / 32)) {
    float2 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int col = C0 + n0 + u * (kUpdThreads / 32);
      v[u] = col < N ? A[(long long)col * N + k0 + lane] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      float h, l;
      const int o = part_off(n0 + u * (kUpdThreads / 32), lane);
      split_tf32(v[u].x, h, l);
      *reinterpret_cast<float*>(part + 4 * kPartBytes + o) = h;
      *reinterpret_cast<float*>(part + 5 * kPartBytes + o) = l;
      split_tf32(v[u].y, h, l);
      *reinterpret_cast<float*>(part + 6 * kPartBytes + o) = h;
      *reinterpret_cast<float*>(part + 7 * kPartBytes + o) = l;
    }
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  if (tid == 0) {
    const uint32_t base = tc::smem_addr(part);
    constexpr uint32_t id_pos = tc::idesc_tf32(kTile, kTile, false), id_neg = tc::idesc_tf32(kTile, kTile, true);
    const uint32_t d_re = tmem, d_im = tmem + kTile;
    // (A part, B part) pairs of the three-term split: hi hi, hi lo, lo hi
    const int xa[3] = {0, 0, 1}, xb[3] = {0, 1, 0};
    bool first = true;
    for (int t = 0; t < 3; ++t) {
      for (int ks = 0; ks < kOuter / 8; ++ks) {
        const uint32_t ko = ks * 256;    // 8 TF32 of K = two 16-byte core-matrix columns
        auto desc = [&](int p) { return tc::smem_desc(base + p * kPartBytes + ko, 128, 1024); };
        const uint64_t ar = desc(0 + xa[t]), ai = desc(2 + xa[t]), br = desc(4 + xb[t]), bi = desc(6 + xb[t]);
        tc::mma_tf32(d_re, ar, br, id_pos, !first);
        tc::mma_tf32(d_re, ai, bi, id_neg, true);
        tc::mma_tf32(d_im, ar, bi, id_pos, !first);
        tc::mma_tf32(d_im, ai, br, id_pos, true);
        first = false;
      }
    }
    tc::mma_commit(&bar);
  }
  const bool ok = tc::mbar_wait(&bar, 0, kMaxPolls);
  tc::fence_after_sync();
  if (ok) {
    // warp w reads TMEM lanes 32 (w % 4) .. + 31 (its lane quarter); warps 0-3 take columns 0-63, 4-7 64-127
    const int quarter = wid & 3, row = R0 + 32 * quarter + lane;
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * quarter) << 16);
    for (int c = (wid >> 2) * (kTile / 2); c < (wid >> 2) * (kTile / 2) + kTile / 2; c += 16) {
      float re[16], im[16];
      tc::tmem_ld16(lane_addr + c, re);
      tc::tmem_ld16(lane_addr + kTile + c, im);
      if (row < N) {
        float2 v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = C0 + c + j;
          v[j] = col < N ? A[(long long)col * N + row] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = C0 + c + j;
          if (col < N) A[(long long)col * N + row] = make_float2(v[j].x - re[j], v[j].y - im[j]);
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(J.dev_err, 1);       // the tensor core did not complete: reported by fthms_wait
  }
  tc::fence_before_sync();
  __syncthreads();
  if (wid == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

__global__ void __launch_bounds__(kLuThreadsFinish) k_lu_big_finish(DevJob J) {
  __shared__ float2 shl[2 * kSB * kSB];
  const SysDesc s = J.sys[J.lu_big[blockIdx.x]];
  lu_finish<float2, kLuThreadsFinish>(J.LU32 + s.mat_off, s.N, J.dinv32 + s.piv_off, shl);
}

}  // namespace

// The inner-panel rows (maxN x kInnerPS) or, later in the same buffer, the threads' 32-row column segments.
size_t lu_big_panel_smem(int maxN) {
  const size_t pn = (size_t)maxN * kInnerPS, segs = (size_t)kOuter * kPanelThreads;
  return (pn > segs ? pn : segs) * sizeof(float2);
}

// Kernel attributes of the large-system LU (once per launch sequence).
static cudaError_t lu_big_attributes(const DevJob& J) {
  const size_t sh_p = lu_big_panel_smem(J.big_max_n);
  cudaError_t e = cudaFuncSetAttribute(k_lu_big_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh_p);
  if (e != cudaSuccess) return e;
  // the largest shared-memory carveout, so that two panel CTAs (128 registers a thread) share an SM
  e = cudaFuncSetAttribute(k_lu_big_panel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_lu_big_update, cudaFuncAttributeMaxDynamicSharedMemorySize, 8 * kPartBytes);
}

int lu_big_panels(const DevJob& J) { return J.n_lu_big > 0 ? (J.big_max_n + kOuter - 1) / kOuter : 0; }

cudaError_t launch_lu_big_panel(const DevJob& J, int panel, cudaStream_t st, int* launches) {
  if (J.n_lu_big == 0) return cudaSuccess;
  cudaError_t e = panel == 0 ? lu_big_attributes(J) : cudaSuccess;
  if (e != cudaSuccess) return e;
  k_lu_big_panel<<<J.n_lu_big, kPanelThreads, lu_big_panel_smem(J.big_max_n), st>>>(J, panel * kOuter);
  *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_lu_big_update(const DevJob& J, int panel, cudaStream_t st, int* launches) {
  const int k0 = panel * kOuter, T = J.big_max_n - k0 - kOuter;
  if (J.n_lu_big == 0 || T <= 0) return cudaSuccess;
  const int tm = (T + kTile - 1) / kTile;
  k_lu_big_update<<<dim3(J.n_lu_big, tm * tm), kUpdThreads, 8 * kPartBytes, st>>>(J, k0);
  *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_lu_big_finish(const DevJob& J, cudaStream_t st, int* launches) {
  if (J.n_lu_big == 0) return cudaSuccess;
  k_lu_big_finish<<<J.n_lu_big, kLuThreadsFinish, 0, st>>>(J);
  *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_lu_large(const DevJob& J, cudaStream_t st, int* launches) {
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < lu_big_panels(J) && e == cudaSuccess; ++k) {
    e = launch_lu_big_panel(J, k, st, launches);
    if (e == cudaSuccess) e = launch_lu_big_update(J, k, st, launches);
  }
  return e == cudaSuccess ? launch_lu_big_finish(J, st, launches) : e;
}

}  // namespace fthms
