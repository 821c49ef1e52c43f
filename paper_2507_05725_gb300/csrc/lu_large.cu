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
//  - K in two stages of 16: 8 operand parts (Ar, Ai, Br, Bi) x (hi, lo) of 128 rows x 16 K in 64 KB of shared
//    memory, K-major without swizzle: element (r, k) at byte (r % 8) 16 + (r / 8) 512 + (k % 4) 4 + (k / 4) 128,
//    so a core matrix (8 rows x 16 bytes) is contiguous, K-adjacent core matrices are 128 bytes apart (leading
//    byte offset) and 8-row groups 512 bytes apart (stride byte offset); 24 MMAs of 128 x 128 x 8 per stage;
//    the second stage's HBM loads are in flight while the first stage's MMAs run;
//  - Re D and Im D in TMEM columns [0, 128) and [128, 256) of the CTA's 256 (two CTAs per SM); lane = tile
//    row; the epilogue reads 16 columns at a time and subtracts them from the FP32 factor in HBM (a warp's rows
//    are contiguous there);
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
constexpr int kStageK = 16;                       // K per operand stage (two stages per 32-column panel)
constexpr int kPartBytes = kTile * kStageK * 4;   // 128 x 16 TF32 = 8 KB per operand part and stage
constexpr int kSBO = (kStageK / 4) * 128;         // bytes between 8-row groups of a part (K-major, no swizzle)
constexpr int kUpdThreads = 256;
constexpr long long kMaxPolls = 1ll << 18;      // bounded wait for the tensor core (well under a second)
constexpr uint32_t kTmemCols = 256;             // Re and Im accumulators, 128 columns each (two CTAs per SM)
constexpr int kLuThreadsFinish = 256;

// Byte offset of element (r, k) of a 128 x 16 K-major part (see the file comment).
__device__ __forceinline__ int part_off(int r, int k) {
  return (r & 7) * 16 + (r >> 3) * kSBO + (k & 3) * 4 + (k >> 2) * 128;
}

// Outer panel k0 of every large system with N > k0 (kPanelThreads threads per system; the 8-column inner
// panels factored by the whole block).
__global__ void __launch_bounds__(kPanelThreads) k_lu_big_panel(DevJob J, int k0) {
  extern __shared__ __align__(16) unsigned char sh_raw[];
  float2* Pn = reinterpret_cast<float2*>(sh_raw);   // [N - k1][kInnerPS] inner panel rows
  __shared__ float2 U[kInner][kOuter];              // inner U12 rows within the outer panel
  __shared__ float2 L11[kOuter][kOuter + 1];        // unit-lower block of the outer panel (row-major)
  __shared__ int spiv[kInner];
  __shared__ float red_m[kPanelThreads / 32];
  __shared__ int red_i[kPanelThreads / 32];
  const SysDesc s = J.sys[J.lu_big[blockIdx.x]];
  const int N = s.N;
  if (k0 >= N) return;
  float2* A = J.LU32 + s.mat_off;
  int* piv = J.piv + s.piv_off;
  const int tid = threadIdx.x;
  const int nbo = min(kOuter, N - k0), kend = k0 + nbo;
  for (int k1 = k0; k1 < kend; k1 += kInner) {
    const int w = min(kInner, kend - k1), nr = N - k1;
    for (int idx = tid; idx < nr * w; idx += kPanelThreads) {
      const int c = idx / nr, r = idx % nr;
      Pn[r * kInnerPS + c] = A[(long long)(k1 + c) * N + k1 + r];
    }
    __syncthreads();
    panel_factor_block<float2, kPanelThreads>(Pn, kInnerPS, nr, w, spiv, red_m, red_i);
    if (tid < w) piv[k1 + tid] = k1 + spiv[tid];
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

// One operand stage (K = 16 of the panel, from column k0 + kk0): the L21 tile (rows R0 .. R0+127) and the U12
// tile (columns C0 .. C0+127), both read from HBM into registers (zero beyond N).
struct StageRegs {
  float2 l[8];   // L21: row tid % 128, k = kk0 + 8 (tid / 128) + 0..7
  float2 u[8];   // U12: k = kk0 + tid % 16, column tid / 16 + 16 j, j = 0..7
};

__device__ __forceinline__ void load_stage(const float2* A, int N, int k0, int kk0, int R0, int C0, int tid,
                                           StageRegs& g) {
  const int r = tid & (kTile - 1), kh = (tid >> 7) * 8, row = R0 + r;
#pragma unroll
  for (int k = 0; k < 8; ++k)
    g.l[k] = row < N ? A[(long long)(k0 + kk0 + kh + k) * N + row] : make_float2(0.f, 0.f);
  const int kk = tid & 15;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int col = C0 + (tid >> 4) + 16 * j;
    g.u[j] = col < N ? A[(long long)col * N + k0 + kk0 + kk] : make_float2(0.f, 0.f);
  }
}

// One operand element: the TF32 value and its TF32 remainder.
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  hi = tc::to_tf32(x);
  lo = tc::to_tf32(x - hi);
}

// The stage's registers as the 8 K-major parts 0 Ar_hi, 1 Ar_lo, 2 Ai_hi, 3 Ai_lo, 4 Br_hi, 5 Br_lo,
// 6 Bi_hi, 7 Bi_lo in shared memory.
__device__ __forceinline__ void store_stage(unsigned char* part, int tid, const StageRegs& g) {
  const int r = tid & (kTile - 1), kh = (tid >> 7) * 8;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    float h, l;
    const int o = part_off(r, kh + k);
    split_tf32(g.l[k].x, h, l);
    *reinterpret_cast<float*>(part + 0 * kPartBytes + o) = h;
    *reinterpret_cast<float*>(part + 1 * kPartBytes + o) = l;
    split_tf32(g.l[k].y, h, l);
    *reinterpret_cast<float*>(part + 2 * kPartBytes + o) = h;
    *reinterpret_cast<float*>(part + 3 * kPartBytes + o) = l;
  }
  const int kk = tid & 15;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    float h, l;
    const int o = part_off((tid >> 4) + 16 * j, kk);
    split_tf32(g.u[j].x, h, l);
    *reinterpret_cast<float*>(part + 4 * kPartBytes + o) = h;
    *reinterpret_cast<float*>(part + 5 * kPartBytes + o) = l;
    split_tf32(g.u[j].y, h, l);
    *reinterpret_cast<float*>(part + 6 * kPartBytes + o) = h;
    *reinterpret_cast<float*>(part + 7 * kPartBytes + o) = l;
  }
}

// The MMAs of one stage (issued by one thread): complex as four real products, each as the three TF32 products
// hi hi, hi lo, lo hi; the first stage's first products overwrite the accumulators.
__device__ __forceinline__ void mma_stage(uint32_t base, uint32_t d_re, uint32_t d_im, bool first) {
  constexpr uint32_t id_pos = tc::idesc_tf32(kTile, kTile, false), id_neg = tc::idesc_tf32(kTile, kTile, true);
  const int xa[3] = {0, 0, 1}, xb[3] = {0, 1, 0};
  for (int t = 0; t < 3; ++t) {
    for (int ks = 0; ks < kStageK / 8; ++ks) {
      const uint32_t ko = ks * 256;    // 8 TF32 of K = two 16-byte core-matrix columns
      auto desc = [&](int p) { return tc::smem_desc(base + p * kPartBytes + ko, 128, kSBO); };
      const uint64_t ar = desc(0 + xa[t]), ai = desc(2 + xa[t]), br = desc(4 + xb[t]), bi = desc(6 + xb[t]);
      tc::mma_tf32(d_re, ar, br, id_pos, !first);
      tc::mma_tf32(d_re, ai, bi, id_neg, true);
      tc::mma_tf32(d_im, ar, bi, id_pos, !first);
      tc::mma_tf32(d_im, ai, br, id_pos, true);
      first = false;
    }
  }
}

// Trailing update A22 -= L21 U12 after outer panel k0: blockIdx.x = large system, blockIdx.y = tile.  K = 32 in
// two stages of 16 through one 64 KB operand buffer: the second stage's HBM loads are issued before the wait for
// the first stage's MMAs (which read the buffer), then written over it.  64 KB of shared memory and 256 tensor-
// memory columns per CTA, so two CTAs share an SM and overlap one's epilogue with the other's loads.
__global__ void __launch_bounds__(kUpdThreads, 2) k_lu_big_update(DevJob J, int k0) {
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
  unsigned char* part = sm;
  if (wid == 0) tc::tmem_alloc(&tmem_base, kTmemCols);
  if (tid == 0) tc::mbar_init(&bar, 1);
  StageRegs g;
  load_stage(A, N, k0, 0, R0, C0, tid, g);
  store_stage(part, tid, g);
  load_stage(A, N, k0, kStageK, R0, C0, tid, g);  // in flight during the first stage's MMAs
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t base = tc::smem_addr(part);
  if (tid == 0) {
    mma_stage(base, tmem, tmem + kTile, true);
    tc::mma_commit(&bar);
  }
  bool ok = tc::mbar_wait(&bar, 0, kMaxPolls);   // the buffer is free once the first stage's MMAs are done
  tc::fence_after_sync();
  if (ok) {
    store_stage(part, tid, g);
    tc::fence_proxy_async();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  ok = __syncthreads_and(ok) != 0;
  if (ok) {
    if (tid == 0) {
      mma_stage(base, tmem, tmem + kTile, false);
      tc::mma_commit(&bar);
    }
    ok = tc::mbar_wait(&bar, 1, kMaxPolls);
    tc::fence_after_sync();
  }
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
  e = cudaFuncSetAttribute(k_lu_big_update, cudaFuncAttributeMaxDynamicSharedMemorySize, 8 * kPartBytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_lu_big_update, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
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
