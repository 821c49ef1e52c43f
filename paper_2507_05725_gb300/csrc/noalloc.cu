// fthms_assemble_self_noalloc: the self-matrix assembly of fthms_assemble_self without any device
// allocation.  Its temporary device data (node coordinates, the log-weight table, the tile and system
// descriptors) live in one file-scope device array that every GPU loading the library holds until the
// process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "fthms.h"
#include "kernels.h"

namespace {

using namespace fthms;

constexpr int kNoallocMaxN = 256;                       // largest N accepted
constexpr int kNoallocMaxTiles = 136;                   // (16 * 17) / 2 tiles at N = 256
constexpr size_t kAlign = 256;

constexpr size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Scratch layout (byte offsets inside the array).
constexpr size_t kOffNodes = 0;                                                   // 4 x N doubles
constexpr size_t kOffRlog = align_up(kOffNodes + 4 * kNoallocMaxN * sizeof(double));  // N x N doubles
constexpr size_t kOffSys = align_up(kOffRlog + (size_t)kNoallocMaxN * kNoallocMaxN * sizeof(double));
constexpr size_t kOffPanel = align_up(kOffSys + sizeof(SysDesc));
constexpr size_t kOffRlogN = align_up(kOffPanel + sizeof(Panel));
constexpr size_t kOffRlogOff = align_up(kOffRlogN + sizeof(int));
constexpr size_t kOffTiles = align_up(kOffRlogOff + sizeof(long long));
constexpr size_t kScratchBytes = align_up(kOffTiles + kNoallocMaxTiles * sizeof(SelfTile));   // ~534 KB

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
unsigned char* g_scratch_dev[64] = {};   // device address of g_scratch per device (set-up once)

fthms_status fail_msg(fthms_status s, const char* msg) {
  set_last_error(msg);
  return s;
}

fthms_status cuda_msg(cudaError_t e, const char* what) {
  char buf[256];
  std::snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  set_last_error(buf);
  return FTHMS_ECUDA;
}

// Per-device set-up, done by the first call on each device with that device current: the device
// address of g_scratch (host code only has a host-side stand-in for the symbol) and the Bessel tables.
fthms_status scratch_address(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (dev < 0 || dev >= 64) return fail_msg(FTHMS_EINVAL, "fthms_assemble_self_noalloc: device index >= 64");
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return cuda_msg(e, "cudaGetSymbolAddress(no-alloc scratch)");
    e = init_constants();
    if (e != cudaSuccess) return cuda_msg(e, "init_constants");
    g_scratch_dev[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_dev[dev];
  return FTHMS_OK;
}

void curve_eval(const fthms_curve* c, double th, double& x, double& y, double& dx, double& dy) {
  x = y = dx = dy = 0.0;
  for (int k = 0; k <= c->degree; ++k) {
    const double cs = std::cos(k * th), sn = std::sin(k * th);
    x += c->ax[k] * cs + c->bx[k] * sn;
    y += c->ay[k] * cs + c->by[k] * sn;
    dx += k * (-c->ax[k] * sn + c->bx[k] * cs);
    dy += k * (-c->ay[k] * sn + c->by[k] * cs);
  }
}

}  // namespace

extern "C" fthms_status fthms_assemble_self_noalloc(const fthms_curve* curve, const fthms_arc* arc, int N,
                                                    double kappa, double* A_dev, void* cuda_stream) {
  if (!curve || !arc || !A_dev || !curve->ax || !curve->bx || !curve->ay || !curve->by || curve->degree < 1 ||
      !(kappa > 0) || !(arc->theta_b > arc->theta_a))
    return fail_msg(FTHMS_EINVAL, "fthms_assemble_self_noalloc: bad arguments");
  if (N < 2 || N > kNoallocMaxN)
    return fail_msg(FTHMS_EINVAL, "fthms_assemble_self_noalloc: N must be in [2, 256] (size of the static scratch)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_msg(e, "cudaGetDevice");
  unsigned char* base = nullptr;
  fthms_status s = scratch_address(dev, &base);
  if (s != FTHMS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

  // Host-side tables on the stack (no heap, no device allocation).  A copy from pageable host memory
  // has been staged by the time cudaMemcpyAsync returns, so these buffers may go out of scope after
  // the loop below; the kernels stay queued on the stream.
  double nodes[4 * kNoallocMaxN];
  const double tc = 0.5 * (arc->theta_a + arc->theta_b), half = 0.5 * (arc->theta_b - arc->theta_a);
  for (int i = 0; i < N; ++i) {
    const double t = std::cos((2.0 * i + 1.0) * 3.14159265358979323846 / (2.0 * N));
    double x, y, dx, dy;
    curve_eval(curve, tc + half * t, x, y, dx, dy);
    nodes[i] = t;
    nodes[N + i] = x;
    nodes[2 * N + i] = y;
    nodes[3 * N + i] = std::hypot(dx, dy) * half;
  }
  SysDesc sys{};
  sys.arc = 0; sys.l = 1; sys.N = N; sys.panel = 0; sys.mat_off = 0; sys.vec_off = 0; sys.piv_off = 0;
  sys.rlog_off = 0; sys.kappa = kappa;
  Panel pn{0, N, 0};
  int rlogN = N;
  long long rlog_off = 0;
  SelfTile tiles[kNoallocMaxTiles];
  int nt = (N + kSelfTile - 1) / kSelfTile, ntile = 0;
  for (int a = 0; a < nt; ++a)
    for (int b = a; b < nt; ++b) tiles[ntile++] = SelfTile{0, 1, a, b};

  // Every region the kernels read is overwritten here and every entry of A is written by the
  // kernel, so nothing carried over from an earlier call is used and nothing needs clearing.
  const struct { size_t off; const void* src; size_t n; } ups[] = {
      {kOffNodes, nodes, 4 * (size_t)N * sizeof(double)}, {kOffSys, &sys, sizeof sys},
      {kOffPanel, &pn, sizeof pn}, {kOffRlogN, &rlogN, sizeof rlogN}, {kOffRlogOff, &rlog_off, sizeof rlog_off},
      {kOffTiles, tiles, ntile * sizeof(SelfTile)}};
  for (const auto& u : ups) {
    e = cudaMemcpyAsync(base + u.off, u.src, u.n, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_msg(e, "cudaMemcpyAsync(no-alloc scratch)");
  }
  DevJob J{};
  const double* nd = reinterpret_cast<const double*>(base + kOffNodes);
  J.node_t = nd;
  J.node_x = nd + N;
  J.node_y = nd + 2 * N;
  J.node_sp = nd + 3 * N;
  J.rlog = reinterpret_cast<double*>(base + kOffRlog);
  J.sys = reinterpret_cast<const SysDesc*>(base + kOffSys);
  J.panels = reinterpret_cast<const Panel*>(base + kOffPanel);
  J.rlogN = reinterpret_cast<const int*>(base + kOffRlogN);
  J.rlog_off_N = reinterpret_cast<const long long*>(base + kOffRlogOff);
  J.tiles = reinterpret_cast<const SelfTile*>(base + kOffTiles);
  J.A = reinterpret_cast<double2*>(A_dev);
  J.h = kappa;
  J.n_rlogN = 1;
  J.n_tiles = ntile;
  J.max_n = N;
  J.K = 16;
  int nl = 0;
  e = launch_tables_rlog_only(J, st, &nl);
  if (e == cudaSuccess) e = launch_assemble_self(J, st, &nl);
  if (e != cudaSuccess) return cuda_msg(e, "fthms_assemble_self_noalloc launch");
  return FTHMS_OK;
}
