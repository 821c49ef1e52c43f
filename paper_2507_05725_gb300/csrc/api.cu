// C ABI of the FTH-MS library (declared in include/fthms.h): contexts, jobs, device memory and the
// order in which the pipeline stages of kernels.cu are enqueued.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <functional>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <vector>

#include "fthms.h"
#include "kernels.h"
#include "plan.h"

using namespace fthms;

namespace {

thread_local std::string g_last_error = "no error";

fthms_status fail(fthms_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

fthms_status cuda_fail(cudaError_t e, const char* what) {
  char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  g_last_error = buf;
  return FTHMS_ECUDA;
}

#define CK(call)                                              \
  do {                                                        \
    cudaError_t e__ = (call);                                 \
    if (e__ != cudaSuccess) return cuda_fail(e__, #call);     \
  } while (0)

std::mutex g_init_mu;
bool g_init_done[64] = {};

fthms_status ensure_device(int dev) {
  CK(cudaSetDevice(dev));
  std::lock_guard<std::mutex> lk(g_init_mu);
  if (dev >= 0 && dev < 64 && !g_init_done[dev]) {
    CK(init_constants());
    // Job memory comes from the device's stream-ordered pool (cudaMallocAsync); keep what released
    // jobs free there for the next job instead of returning it to the driver at every synchronisation
    // (a per-process pool attribute; the HBM budget still admits jobs by its own accounting).
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      unsigned long long keep = ~0ULL;   // the attribute is a 64-bit unsigned byte count
      if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) cudaGetLastError();
    } else {
      cudaGetLastError();
    }
    g_init_done[dev] = true;
  }
  return FTHMS_OK;
}

}  // namespace

void fthms::set_last_error(const char* msg) { g_last_error = msg; }

struct fthms_ctx {
  int device = 0;
  size_t budget = 0;
  size_t in_use = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;         // created by fthms_create (no stream was given)
  std::mutex mu;
  std::set<fthms_req*> live;       // prepared and not yet released jobs
};

struct ProfMark {
  int stage;
  int launches;
  cudaEvent_t a, b;
};

struct fthms_req {
  fthms_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;   // stream of all of this job's work (the context's, or a server slot's)
  Plan plan;
  DevJob J{};
  std::vector<void*> allocs;
  size_t bytes = 0;
  size_t h2d = 0;
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<ProfMark> marks;
  double stage_ms[FTHMS_NSTAGES] = {};
  long long stage_launches[FTHMS_NSTAGES] = {};
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool ran = false;
  int launches = 0;
  double setup_ms = 0.0;
  bool use_graph = false;          // replay the captured pipeline instead of launching stage by stage
  bool use_fused = false;          // FP64 form: assembly + LU + step-1 solve in one persistent launch
  cudaGraphExec_t graph = nullptr;
  bool conv_checked = false;       // the last run's refinement counters have been read
  fthms_status conv_status = FTHMS_OK;
  std::string conv_msg;
  int fallback_runs = 0;           // runs repeated in FP64 after a refinement that did not converge
  bool plain_apply_fits = true;    // the FP64 stored-row apply fits shared memory (FP64 fallback possible)
  int lu_min = kLuBigMin;          // smallest N factored with tensor-core updates (mixed forms)
  fthms_allreduce_fn allreduce = nullptr;   // sum across the ranks of a frequency-partitioned job
  void* allreduce_user = nullptr;
};

namespace {

template <class T>
fthms_status dev_upload(fthms_req* r, const std::vector<T>& v, const T** out) {
  *out = nullptr;
  if (v.empty()) return FTHMS_OK;
  void* p = nullptr;
  size_t b = v.size() * sizeof(T);
  CK(cudaMallocAsync(&p, b, r->stream));
  r->allocs.push_back(p);
  r->bytes += b;
  CK(cudaMemcpyAsync(p, v.data(), b, cudaMemcpyHostToDevice, r->stream));
  r->h2d += b;
  *out = static_cast<const T*>(p);
  return FTHMS_OK;
}

template <class T>
fthms_status dev_alloc(fthms_req* r, size_t count, T** out) {
  *out = nullptr;
  if (count == 0) return FTHMS_OK;
  void* p = nullptr;
  size_t b = count * sizeof(T);
  CK(cudaMallocAsync(&p, b, r->stream));
  r->allocs.push_back(p);
  r->bytes += b;
  *out = static_cast<T*>(p);
  return FTHMS_OK;
}

void free_req(fthms_req* r) {
  if (r->graph) {
    cudaGraphExecDestroy(r->graph);
    r->graph = nullptr;
  }
  for (void* p : r->allocs) cudaFreeAsync(p, r->stream);
  r->allocs.clear();
  for (cudaEvent_t e : r->ev_pool) cudaEventDestroy(e);
  r->ev_pool.clear();
  if (r->ev0) cudaEventDestroy(r->ev0);
  if (r->ev1) cudaEventDestroy(r->ev1);
}

#define TRY(x)                         \
  do {                                 \
    fthms_status s__ = (x);            \
    if (s__ != FTHMS_OK) return s__;   \
  } while (0)

// The first n_big systems of sys_order (the largest) take the tensor-core LU, the rest the one-CTA LU.
void set_lu_split(fthms_req* r, int n_big) {
  DevJob& J = r->J;
  const Plan& p = r->plan;
  n_big = std::max(0, std::min(n_big, (int)p.sys_order.size()));
  J.lu_big = J.sys_order;
  J.n_lu_big = n_big;
  J.lu_small = J.sys_order ? J.sys_order + n_big : nullptr;
  J.n_lu_small = (int)p.sys_order.size() - n_big;
  J.big_max_n = n_big > 0 ? p.sys[p.sys_order[0]].N : 0;
}

// Launch shapes and LU split from five choices (validated): 0 keeps the built-in default.
void apply_shapes(fthms_req* r, const int* shapes) {
  DevJob& J = r->J;
  J.shape_solve = shapes[0];
  J.shape_asm = shapes[1];
  J.shape_time = shapes[2];
  J.shape_restr = shapes[3];
  if (r->plan.opt.precision >= 1) {
    const int lu_min = shapes[4] ? shapes[4] : kLuBigMin;
    int nb = 0;
    while (nb < (int)r->plan.sys_order.size() && r->plan.sys[r->plan.sys_order[nb]].N >= lu_min) ++nb;
    set_lu_split(r, nb);
    r->lu_min = lu_min;
  }
}

fthms_status upload_job(fthms_req* r) {
  Plan& p = r->plan;
  DevJob& J = r->J;
  J.P = p.P; J.L = p.L; J.Q = p.Q; J.K = p.K; J.NT = p.NT; J.M = p.M;
  J.n_obs = p.n_obs; J.n_tout = p.n_tout;
  J.nsys = (int)p.sys_order.size();   // systems of this rank's frequencies (all, unpartitioned)
  J.n_act = (int)p.act_idx.size();
  J.n_grp = (int)p.grps.size();
  J.n_asm = (int)p.asms.size();
  J.n_tiles = (int)p.self_tiles.size();
  J.n_rlogN = (int)p.rlogN.size();
  J.n_restr = (int)p.restr_pairs.size();
  J.logK = 0;
  while ((1 << J.logK) < p.K) ++J.logK;
  J.max_n = p.maxN;
  J.max_nmax = 0;
  for (int k = 0; k < p.P; ++k) J.max_nmax = std::max(J.max_nmax, p.Nmax[k]);
  J.acc_cap = std::max(J.max_nmax, p.n_obs);
  J.row_cap = 0;
  J.ph_cap = 0;
  for (const CrossGrp& g : p.grps) {
    int rows = 0, nsum = 0;
    for (int b = g.blk_begin; b < g.blk_end; ++b) {
      rows += p.blks[b].nrows;
      nsum += p.blks[b].N;
    }
    J.row_cap = std::max(J.row_cap, rows);
    J.ph_cap = std::max(J.ph_cap, nsum);
  }
  // The FP64 stored-row apply keeps a whole group in shared memory (the mixed form works in row slices).
  r->plain_apply_fits = p.opt.cross_mode != 0 ||
                        (size_t)J.Q * (J.acc_cap + J.row_cap + J.ph_cap) * 16 <= (size_t)227 * 1024;
  if (p.opt.precision == 0 && !r->plain_apply_fits)
    return fail(FTHMS_EINVAL, "fthms_prepare: the stored cross rows of one (arc, frequency) group do not fit the "
                              "apply's shared memory; use cross_mode 1");
  J.h = p.h; J.dt = p.dt; J.sign = p.sig.sign;
  J.sig_kind = p.sig.kind;
  J.z0x = p.sig.z0[0]; J.z0y = p.sig.z0[1];
  J.dirx = p.sig.dir[0]; J.diry = p.sig.dir[1];
  J.amp = p.sig.amp; J.carrier = p.sig.carrier; J.centre = p.sig.centre; J.width = p.sig.width;
  J.sig_nt = (int)p.sig_f.size();
  J.sig_t0 = p.sig.t0; J.sig_dt = p.sig.dt; J.sig_band = p.sig.band;
  J.H = p.H; J.period = p.period;
  J.vec_total = p.vec_total;
  J.mixed = p.opt.precision >= 1 ? 1 : 0;
  J.fp64keep = p.opt.precision == 2 ? 1 : 0;
  J.refine_tol = p.opt.refine_tol;
  J.refine_max = p.opt.refine_max;
  J.mat_total = p.mat_total;
  TRY(dev_upload(r, p.sig_f, &J.sig_f));

  TRY(dev_upload(r, p.sys, &J.sys));
  TRY(dev_upload(r, p.sys_order, &J.sys_order));
  set_lu_split(r, p.n_lu_big);
  TRY(dev_alloc(r, 1, &J.dev_err));
  TRY(dev_alloc(r, 1, &J.work_counter));
  TRY(dev_upload(r, p.panels, &J.panels));
  TRY(dev_upload(r, p.node_t, &J.node_t));
  TRY(dev_upload(r, p.node_x, &J.node_x));
  TRY(dev_upload(r, p.node_y, &J.node_y));
  TRY(dev_upload(r, p.node_sp, &J.node_sp));
  TRY(dev_upload(r, p.rlogN, &J.rlogN));
  TRY(dev_upload(r, p.rlog_off_N, &J.rlog_off_N));
  TRY(dev_alloc(r, (size_t)p.rlog_total, &J.rlog));
  std::vector<int> rn;
  for (auto& pr : p.restr_pairs) { rn.push_back(pr.first); rn.push_back(pr.second); }
  TRY(dev_upload(r, rn, &J.restr_N));
  TRY(dev_upload(r, p.restr_off, &J.restr_off));
  TRY(dev_alloc(r, (size_t)p.restr_total, &J.restr));
  J.restr_df = nullptr;
  if (p.opt.precision >= 1) TRY(dev_alloc(r, (size_t)p.restr_total, &J.restr_df));
  TRY(dev_upload(r, p.restr_of_sys, &J.restr_of_sys));
  TRY(dev_upload(r, p.self_tiles, &J.tiles));
  TRY(dev_upload(r, p.tgts, &J.tgts));
  TRY(dev_upload(r, p.pairs, &J.pairs));
  TRY(dev_upload(r, p.e_off, &J.e_off));
  TRY(dev_upload(r, p.asms, &J.asms));
  TRY(dev_upload(r, p.grps, &J.grps));
  TRY(dev_upload(r, p.blks, &J.blks));
  J.n_slices = 0;
  J.slice_ph_cap = p.slice_ph_cap;
  J.slices = nullptr;
  J.grp_res_off = nullptr;
  J.apply_res = nullptr;
  J.otf = p.opt.cross_mode == 1 ? 1 : 0;
  J.n_otf = 0;
  J.otf_tasks = nullptr;
  J.wn_off = nullptr;
  J.wn = nullptr;
  J.otf_res_off = nullptr;
  if (J.mixed || J.otf) {
    TRY(dev_upload(r, p.grp_res_off, &J.grp_res_off));
    TRY(dev_alloc(r, (size_t)std::max(1LL, p.res_total) * p.Q, &J.apply_res));
  }
  if (J.mixed && !J.otf) {
    TRY(dev_upload(r, p.slices, &J.slices));
    J.n_slices = (int)p.slices.size();
  }
  if (J.otf) {
    TRY(dev_upload(r, p.otf, &J.otf_tasks));
    TRY(dev_upload(r, p.wn_off, &J.wn_off));
    TRY(dev_upload(r, p.otf_res_off, &J.otf_res_off));
    TRY(dev_alloc(r, (size_t)p.wn_total, &J.wn));
    J.n_otf = (int)p.otf.size();
  }
  apply_shapes(r, p.opt.shapes);       // launch shapes and LU split (fthms_options.shapes; 0 = default)
  TRY(dev_upload(r, p.tpanel, &J.tpanel));
  TRY(dev_upload(r, p.tr_off, &J.tr_off));
  TRY(dev_upload(r, p.chi, &J.chi));
  TRY(dev_upload(r, p.act_off, &J.act_off));
  TRY(dev_upload(r, p.act_idx, &J.act_idx));
  TRY(dev_upload(r, p.act_arc, &J.act_arc));
  TRY(dev_upload(r, p.win, &J.win));
  TRY(dev_upload(r, p.wl, &J.wl));
  TRY(dev_upload(r, p.c_q, &J.c_q));
  TRY(dev_upload(r, p.nlo, &J.nlo));
  TRY(dev_upload(r, p.tout, &J.tout));
  TRY(dev_upload(r, p.s_q, &J.s_q));
  TRY(dev_alloc(r, (size_t)p.mat_total, &J.A));
  TRY(dev_alloc(r, (size_t)p.piv_total, &J.piv));
  TRY(dev_alloc(r, (size_t)p.piv_total, &J.dinv));
  J.LU32 = nullptr;
  J.dinv32 = nullptr;
  J.rres = nullptr;
  J.rres64 = nullptr;
  J.dcorr = nullptr;
  J.mdone = nullptr;
  J.mrel = nullptr;
  J.mrho = nullptr;
  J.mscale = nullptr;
  J.arow = nullptr;
  J.phistat = nullptr;
  J.f64_min_n = J.fp64keep ? 0 : (J.mixed ? kLuBigMin : 1 << 30);
  J.rchunks = nullptr;
  J.n_rchunks = 0;
  TRY(dev_alloc(r, 3, &J.refine_resid));          // [0] max estimated error left, [1] passes, [2] unconverged
  J.sys_err = nullptr;
  if (J.mixed) {
    TRY(dev_alloc(r, p.sys.size(), &J.sys_err));
    TRY(dev_alloc(r, (size_t)p.mat_total, &J.LU32));
    TRY(dev_alloc(r, (size_t)p.piv_total, &J.dinv32));
    TRY(dev_alloc(r, (size_t)p.vec_total, &J.rres));
    TRY(dev_alloc(r, (size_t)p.vec_total, &J.rres64));
    TRY(dev_alloc(r, (size_t)p.vec_total, &J.dcorr));
    TRY(dev_alloc(r, p.sys.size(), &J.mdone));
    TRY(dev_alloc(r, p.sys.size(), &J.mrel));
    TRY(dev_alloc(r, p.sys.size(), &J.mrho));
    TRY(dev_alloc(r, p.sys.size(), &J.mscale));
    TRY(dev_alloc(r, (size_t)p.piv_total, &J.arow));
    TRY(dev_alloc(r, p.sys.size() * 4, &J.phistat));
    TRY(dev_upload(r, p.rchunks, &J.rchunks));
    J.n_rchunks = (int)p.rchunks.size();
  }
  TRY(dev_alloc(r, (size_t)p.vec_total, &J.G));
  TRY(dev_alloc(r, (size_t)p.vec_total, &J.phi));
  J.phi_df = nullptr;
  if (J.mixed) TRY(dev_alloc(r, (size_t)p.vec_total, &J.phi_df));
  TRY(dev_alloc(r, (size_t)p.vec_total, &J.phi_sum));
  J.phi_all = nullptr;
  if (p.opt.keep_densities) TRY(dev_alloc(r, (size_t)p.vec_total * p.M, &J.phi_all));
  TRY(dev_alloc(r, (size_t)p.spec_total, &J.W));
  TRY(dev_alloc(r, (size_t)p.spec_total, &J.Gt));
  TRY(dev_alloc(r, (size_t)p.act_idx.size() * p.NT, &J.ginc));
  J.E = nullptr;
  if (!J.otf) TRY(dev_alloc(r, (size_t)p.e_total, &J.E));
  TRY(dev_alloc(r, (size_t)std::max(1, p.n_obs * p.Q * p.L), &J.Vobs));
  TRY(dev_alloc(r, (size_t)std::max(1, p.n_obs * p.n_tout), &J.traces));
  TRY(dev_alloc(r, (size_t)p.K / 2, &J.fft_tw));
  J.fft_tw_df = nullptr;
  if (J.mixed) TRY(dev_alloc(r, (size_t)p.K / 2, &J.fft_tw_df));
  TRY(dev_alloc(r, (size_t)p.Q * p.L, &J.syn_tw));
  TRY(dev_alloc(r, (size_t)p.Q * p.L, &J.fwd_tw));
  return FTHMS_OK;
}

fthms_status next_event(fthms_req* r, cudaEvent_t* e) {
  if (r->ev_used == r->ev_pool.size()) {
    cudaEvent_t ev;
    CK(cudaEventCreate(&ev));
    r->ev_pool.push_back(ev);
  }
  *e = r->ev_pool[r->ev_used++];
  return FTHMS_OK;
}

// Fold the stage timers of a finished run into the totals.
fthms_status flush_marks(fthms_req* r) {
  if (r->marks.empty()) return FTHMS_OK;
  CK(cudaEventSynchronize(r->marks.back().b));
  for (const ProfMark& m : r->marks) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, m.a, m.b));
    r->stage_ms[m.stage] += ms;
    r->stage_launches[m.stage] += m.launches;
  }
  r->marks.clear();
  r->ev_used = 0;
  return FTHMS_OK;
}

// One pipeline stage, bracketed by profiling events when enabled.
template <class F>
fthms_status stage(fthms_req* r, int st_id, cudaStream_t st, int* nl, F&& launch) {
  ProfMark m{st_id, 0, nullptr, nullptr};
  if (r->profiling) {
    TRY(next_event(r, &m.a));
    CK(cudaEventRecord(m.a, st));
  }
  int before = *nl;
  cudaError_t e = launch();
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  if (r->profiling) {
    TRY(next_event(r, &m.b));
    CK(cudaEventRecord(m.b, st));
    m.launches = *nl - before;
    r->marks.push_back(m);
  }
  return FTHMS_OK;
}

fthms_status enqueue_stages(fthms_req* r, bool bracket = true);

// Run the pipeline: directly, or (use_graph, profiling off) through a CUDA graph captured on the first
// run and replayed afterwards (one launch for the whole job).
fthms_status enqueue(fthms_req* r) {
  if (r->plan.ranks > 1 && !r->allreduce)
    return fail(FTHMS_EINVAL, "fthms_run: a frequency-partitioned job needs fthms_set_allreduce");
  if (!r->use_graph || r->profiling || r->plan.ranks > 1) return enqueue_stages(r);
  TRY(flush_marks(r));
  cudaStream_t st = r->stream;
  if (!r->graph) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    // An event recorded on a capturing stream only marks a dependency inside the graph, so the
    // job's start and end events are recorded around each replay instead.
    fthms_status s = enqueue_stages(r, false);
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (s != FTHMS_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&r->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  }
  CK(cudaEventRecord(r->ev0, st));
  CK(cudaGraphLaunch(r->graph, st));
  CK(cudaEventRecord(r->ev1, st));
  r->ran = true;
  r->conv_checked = false;
  return FTHMS_OK;
}

fthms_status enqueue_stages(fthms_req* r, bool bracket) {
  const DevJob& J = r->J;
  cudaStream_t st = r->stream;
  int nl = 0;
  r->conv_checked = false;
  TRY(flush_marks(r));
  if (bracket) CK(cudaEventRecord(r->ev0, st));
  // Per-run flags and refinement state, cleared before the first kernel: the tensor-core LU reads
  // dev_err (job memory may come back from the pool holding an earlier job's values).
  CK(cudaMemsetAsync(J.dev_err, 0, sizeof(int), st));
  CK(cudaMemsetAsync(J.refine_resid, 0, 3 * sizeof(double), st));
  if (J.sys_err) CK(cudaMemsetAsync(J.sys_err, 0, r->plan.sys.size() * sizeof(float), st));
  if (J.mrho) CK(cudaMemsetAsync(J.mrho, 0, r->plan.sys.size() * sizeof(float), st));   // measured per run
  const bool fused = r->use_fused && !J.mixed;   // assembly, LU and step-1 solve in the fused launch below
  TRY(stage(r, FTHMS_STAGE_TABLES, st, &nl, [&] { return launch_tables(J, st, &nl); }));
  if (!fused) {
    TRY(stage(r, FTHMS_STAGE_ASSEMBLE, st, &nl, [&] { return launch_assemble_self(J, st, &nl); }));
    TRY(stage(r, FTHMS_STAGE_LU, st, &nl, [&] { return launch_lu_small(J, st, &nl); }));
  }
  if (J.mixed) {              // large systems: panels (LU stage) and tensor-core trailing updates, in turn
    for (int k = 0; k < lu_big_panels(J); ++k) {
      TRY(stage(r, FTHMS_STAGE_LU, st, &nl, [&] { return launch_lu_big_panel(J, k, st, &nl); }));
      TRY(stage(r, FTHMS_STAGE_LU_UPDATE, st, &nl, [&] { return launch_lu_big_update(J, k, st, &nl); }));
    }
    TRY(stage(r, FTHMS_STAGE_LU, st, &nl, [&] { return launch_lu_big_finish(J, st, &nl); }));
  }
  TRY(stage(r, FTHMS_STAGE_CROSS_ASM, st, &nl, [&] {
    return J.otf ? launch_near_weights(J, st, &nl) : launch_cross_assemble(J, st, &nl);
  }));
  CK(cudaMemsetAsync(J.Gt, 0, (size_t)r->plan.spec_total * sizeof(double2), st));
  CK(cudaMemsetAsync(J.W, 0, (size_t)r->plan.spec_total * sizeof(double2), st));
  CK(cudaMemsetAsync(J.Vobs, 0, (size_t)std::max(1, J.n_obs * J.Q * J.L) * sizeof(double2), st));
  TRY(stage(r, FTHMS_STAGE_INCIDENT, st, &nl, [&] { return launch_incident(J, st, &nl); }));
  TRY(stage(r, FTHMS_STAGE_RESTRICT, st, &nl, [&] { return launch_restrict(J, st, &nl); }));
  for (int m = 1; m <= J.M; ++m) {
    if (J.mixed) {            // the FP32 solve, then refinement passes (residuals, correction solves)
      TRY(stage(r, FTHMS_STAGE_SOLVE, st, &nl, [&] { return launch_msolve(J, m, 0, st, &nl); }));
      for (int pass = 1; pass <= refine_passes(J); ++pass) {
        TRY(stage(r, pass == 1 ? FTHMS_STAGE_RESID : FTHMS_STAGE_RESID_UPD, st, &nl,
                  [&] { return launch_resid(J, pass, st, &nl); }));
        TRY(stage(r, FTHMS_STAGE_SOLVE, st, &nl, [&] { return launch_msolve(J, m, pass, st, &nl); }));
      }
    } else if (fused && m == 1) {
      TRY(stage(r, FTHMS_STAGE_FUSED, st, &nl, [&] { return launch_fused_asf(J, J.work_counter, st, &nl); }));
    } else {
      TRY(stage(r, FTHMS_STAGE_SOLVE, st, &nl, [&] { return launch_solve(J, m, st, &nl); }));
    }
    TRY(stage(r, FTHMS_STAGE_CROSS_APPLY, st, &nl, [&] {
      return J.otf ? launch_cross_otf(J, st, &nl) : launch_cross_apply(J, st, &nl);
    }));
    if (m < J.M) {
      if (r->plan.ranks > 1) {
        // partial synthesis over this rank's frequencies, the ranks' sum, then the rest of the step
        TRY(stage(r, FTHMS_STAGE_SYNTH_FWD, st, &nl, [&] { return launch_synth_partial(J, st, &nl); }));
        if (J.n_act > 0) r->allreduce(J.ginc, (size_t)J.n_act * J.NT, st, r->allreduce_user);
        TRY(stage(r, FTHMS_STAGE_SYNTH_FWD, st, &nl, [&] { return launch_fwd_after_sum(J, st, &nl); }));
      } else {
        TRY(stage(r, FTHMS_STAGE_SYNTH_FWD, st, &nl, [&] { return launch_synth_fwd(J, st, &nl); }));
      }
      TRY(stage(r, FTHMS_STAGE_RESTRICT, st, &nl, [&] { return launch_restrict(J, st, &nl); }));
    }
  }
  TRY(stage(r, FTHMS_STAGE_TRACES, st, &nl, [&] { return launch_traces(J, st, &nl); }));
  if (r->plan.ranks > 1 && J.n_obs * J.n_tout > 0)
    r->allreduce(J.traces, (size_t)J.n_obs * J.n_tout, st, r->allreduce_user);
  if (bracket) {
    CK(cudaEventRecord(r->ev1, st));
    r->ran = true;
  }
  r->launches = nl;
  return FTHMS_OK;
}

// Time `reps` back-to-back launches of one stage (milliseconds per launch).
template <class F>
fthms_status time_stage(fthms_req* r, int reps, float* ms, F&& launch) {
  cudaStream_t st = r->stream;
  cudaEvent_t a = nullptr, b = nullptr;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  cudaError_t e = launch();            // warm-up (attributes, caches)
  if (e == cudaSuccess) e = cudaEventRecord(a, st);
  for (int k = 0; k < reps && e == cudaSuccess; ++k) e = launch();
  if (e == cudaSuccess) e = cudaEventRecord(b, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return cuda_fail(e, "fthms_autotune");
  *ms /= reps;
  return FTHMS_OK;
}

}  // namespace

extern "C" {

fthms_status fthms_create(fthms_ctx** out, int device, size_t hbm_budget_bytes, void* cuda_stream) {
  if (!out) return fail(FTHMS_EINVAL, "fthms_create: out is NULL");
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= n) return fail(FTHMS_EINVAL, "fthms_create: no such device");
  TRY(ensure_device(device));
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  bool own = false;
  if (!st) {
    // A stream of its own (the legacy default stream cannot be captured into a CUDA graph).
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreateWithFlags");
    own = true;
  }
  fthms_ctx* c = new fthms_ctx;
  c->device = device;
  c->budget = hbm_budget_bytes;
  c->stream = st;
  c->own_stream = own;
  *out = c;
  return FTHMS_OK;
}

fthms_status fthms_destroy(fthms_ctx* ctx) {
  if (!ctx) return fail(FTHMS_EINVAL, "fthms_destroy: NULL context");
  ensure_device(ctx->device);
  {
    // Jobs still alive: wait for their work, free their device memory and detach them, so that
    // their handles stay valid for fthms_release alone.
    std::lock_guard<std::mutex> lk(ctx->mu);
    for (fthms_req* r : ctx->live) {
      if (r->ran) cudaEventSynchronize(r->ev1);
      free_req(r);
      cudaStreamSynchronize(r->stream);
      r->ctx = nullptr;
    }
    ctx->live.clear();
  }
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return FTHMS_OK;
}

fthms_status fthms_plan_info(const fthms_curve* curves, int ncurves, const fthms_arc* arcs, int narcs,
                             const fthms_signal* signal, const fthms_options* options, size_t* device_bytes,
                             int* n_systems) {
  fthms::Plan plan;
  std::string err;
  const int st = build_plan(curves, ncurves, arcs, narcs, signal, options, plan, err);
  if (st != FTHMS_OK) return fail((fthms_status)st, "fthms_prepare: " + err);
  if (device_bytes) *device_bytes = plan.device_bytes;
  if (n_systems) *n_systems = (int)plan.sys_order.size();   // this rank's systems
  return FTHMS_OK;
}

fthms_status fthms_prepare(fthms_ctx* ctx, const fthms_curve* curves, int ncurves, const fthms_arc* arcs,
                           int narcs, const fthms_signal* signal, const fthms_options* options,
                           fthms_req** out) {
  if (!ctx || !out) return fail(FTHMS_EINVAL, "fthms_prepare: NULL context or output");
  *out = nullptr;
  auto t0 = std::chrono::steady_clock::now();
  fthms_req* r = new fthms_req;
  r->ctx = ctx;
  r->stream = ctx->stream;
  std::string err;
  int st = build_plan(curves, ncurves, arcs, narcs, signal, options, r->plan, err);
  if (st != FTHMS_OK) {
    delete r;
    return fail((fthms_status)st, "fthms_prepare: " + err);
  }
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->budget && ctx->in_use + r->plan.device_bytes > ctx->budget) {
      char buf[160];
      snprintf(buf, sizeof buf, "fthms_prepare: job needs %.3f GB, budget leaves %.3f GB",
               r->plan.device_bytes / 1e9, (ctx->budget - ctx->in_use) / 1e9);
      delete r;
      return fail(FTHMS_ENOMEM, buf);
    }
    ctx->in_use += r->plan.device_bytes;
  }
  fthms_status s = ensure_device(ctx->device);
  if (s == FTHMS_OK) {
    cudaError_t e1 = cudaEventCreate(&r->ev0), e2 = cudaEventCreate(&r->ev1);
    if (e1 != cudaSuccess || e2 != cudaSuccess) s = cuda_fail(e1 != cudaSuccess ? e1 : e2, "cudaEventCreate");
  }
  if (s == FTHMS_OK) s = upload_job(r);
  if (s != FTHMS_OK) {
    bool oom = g_last_error.find("out of memory") != std::string::npos;
    std::string msg = g_last_error;
    free_req(r);
    {
      std::lock_guard<std::mutex> lk(ctx->mu);
      ctx->in_use -= r->plan.device_bytes;
    }
    delete r;
    cudaGetLastError();
    return fail(oom ? FTHMS_ENOMEM : s, msg);
  }
  r->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->live.insert(r);
  }
  *out = r;
  return FTHMS_OK;
}

fthms_status fthms_run(fthms_req* req) {
  if (!req) return fail(FTHMS_EINVAL, "fthms_run: NULL job");
  if (!req->ctx) return fail(FTHMS_EINVAL, "fthms_run: the job's context was destroyed");
  TRY(ensure_device(req->ctx->device));
  return enqueue(req);
}

fthms_status fthms_submit(fthms_ctx* ctx, const fthms_curve* curves, int ncurves, const fthms_arc* arcs,
                          int narcs, const fthms_signal* signal, const fthms_options* options,
                          fthms_req** out) {
  TRY(fthms_prepare(ctx, curves, ncurves, arcs, narcs, signal, options, out));
  fthms_status s = fthms_run(*out);
  if (s != FTHMS_OK) {
    std::string msg = g_last_error;
    fthms_release(*out);
    *out = nullptr;
    return fail(s, msg);
  }
  return FTHMS_OK;
}

fthms_status fthms_poll(fthms_req* req, int* done) {
  if (!req || !done) return fail(FTHMS_EINVAL, "fthms_poll: NULL argument");
  if (!req->ctx) return fail(FTHMS_EINVAL, "fthms_poll: the job's context was destroyed");
  if (!req->ran) { *done = 0; return FTHMS_OK; }
  cudaError_t e = cudaEventQuery(req->ev1);
  if (e == cudaSuccess) { *done = 1; return FTHMS_OK; }
  if (e == cudaErrorNotReady) { *done = 0; return FTHMS_OK; }
  return cuda_fail(e, "fthms_poll");
}

// Wait for the last run's completion event (no convergence check).
static fthms_status wait_run(fthms_req* req, int timeout_ms) {
  auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t e = cudaEventQuery(req->ev1);
    if (e == cudaSuccess) return FTHMS_OK;
    if (e != cudaErrorNotReady) return cuda_fail(e, "fthms_wait");
    if (timeout_ms >= 0) {
      double el = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      if (el > timeout_ms) return fail(FTHMS_ETIMEOUT, "fthms_wait: timed out");
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

// After a finished run of a mixed-form job: read how many (system, step) refinements stayed above
// refine_tol; with refine_fallback the whole job runs again in FP64 (every stage, on the job's stream).
static fthms_status check_convergence(fthms_req* req) {
  if (req->conv_checked) {
    if (req->conv_status != FTHMS_OK) g_last_error = req->conv_msg;
    return req->conv_status;
  }
  req->conv_checked = true;
  req->conv_status = FTHMS_OK;
  int derr = 0;
  CK(cudaMemcpyAsync(&derr, req->J.dev_err, sizeof derr, cudaMemcpyDeviceToHost, req->stream));
  CK(cudaStreamSynchronize(req->stream));
  if (derr) {
    req->conv_status = FTHMS_ECUDA;
    req->conv_msg = "fthms_wait: a tensor-core LU update did not complete within its bounded wait";
    g_last_error = req->conv_msg;
    return FTHMS_ECUDA;
  }
  if (!req->J.mixed) return FTHMS_OK;
  unsigned long long bad = 0;
  CK(cudaMemcpyAsync(&bad, reinterpret_cast<const unsigned long long*>(req->J.refine_resid) + 2, sizeof bad,
                     cudaMemcpyDeviceToHost, req->stream));
  CK(cudaStreamSynchronize(req->stream));
  if (bad == 0) return FTHMS_OK;
  // (a frequency-partitioned job never falls back alone: its ranks would stop meeting in the all-reduce)
  if (req->plan.opt.refine_fallback && req->plain_apply_fits && req->plan.ranks <= 1) {
    req->J.mixed = 0;
    req->J.fp64keep = 0;
    if (req->graph) {                  // the captured graph holds the mixed-form kernels
      cudaGraphExecDestroy(req->graph);
      req->graph = nullptr;
    }
    ++req->fallback_runs;
    TRY(enqueue_stages(req));
    TRY(wait_run(req, -1));
    req->conv_checked = true;
    return FTHMS_OK;
  }
  char buf[200];
  snprintf(buf, sizeof buf, "fthms_wait: %llu (system, step) refinements stayed above refine_tol = %.3g after %d "
           "passes%s", bad, req->plan.opt.refine_tol, req->plan.opt.refine_max,
           req->plan.opt.refine_fallback ? " (no FP64 fallback: the stored cross rows exceed its apply)" : "");
  req->conv_status = FTHMS_ENOCONV;
  req->conv_msg = buf;
  g_last_error = buf;
  return FTHMS_ENOCONV;
}

fthms_status fthms_wait(fthms_req* req, int timeout_ms) {
  if (!req) return fail(FTHMS_EINVAL, "fthms_wait: NULL job");
  if (!req->ctx) return fail(FTHMS_EINVAL, "fthms_wait: the job's context was destroyed");
  if (!req->ran) return fail(FTHMS_EINVAL, "fthms_wait: job was never run");
  TRY(ensure_device(req->ctx->device));
  TRY(wait_run(req, timeout_ms));
  return check_convergence(req);
}

// Wait before reading results: a run whose refinement did not converge still has readable results.
static fthms_status wait_results(fthms_req* req) {
  fthms_status s = fthms_wait(req, -1);
  return s == FTHMS_ENOCONV ? FTHMS_OK : s;
}

fthms_status fthms_traces(fthms_req* req, double* out, size_t cap) {
  if (!req || (!out && cap)) return fail(FTHMS_EINVAL, "fthms_traces: NULL argument");
  if (!req->ctx) return fail(FTHMS_EINVAL, "fthms_traces: the job's context was destroyed");
  size_t n = (size_t)req->plan.n_obs * req->plan.n_tout;
  if (cap < n) return fail(FTHMS_EINVAL, "fthms_traces: output buffer too small");
  TRY(wait_results(req));
  if (n) {
    CK(cudaMemcpyAsync(out, req->J.traces, n * sizeof(double), cudaMemcpyDeviceToHost, req->stream));
    CK(cudaStreamSynchronize(req->stream));
  }
  return FTHMS_OK;
}

static fthms_status density_range(fthms_req* req, int arc, int m, int q, const double2** base,
                                  long long* first, long long* last, size_t* needed) {
  const Plan& p = req->plan;
  if (arc < 0 || arc >= p.P || q < 0 || q >= p.Q || m < 0 || m > p.M)
    return fail(FTHMS_EINVAL, "fthms_densities: arc, m or q out of range");
  if (m > 0 && !p.opt.keep_densities)
    return fail(FTHMS_EINVAL, "fthms_densities: per-step densities need keep_densities = 1");
  size_t n = 0;
  for (int l = p.lb; l < p.le; ++l) n += 2 * (size_t)p.Ntab[(size_t)arc * p.L + l];
  if (needed) *needed = n;
  const SysDesc& s0 = p.sys[(size_t)arc * (p.L - 1) + p.lb - 1];      // this rank's first and last frequency
  const SysDesc& s1 = p.sys[(size_t)arc * (p.L - 1) + p.le - 2];
  *first = s0.vec_off;
  *last = s1.vec_off + (long long)p.Q * s1.N;
  *base = m == 0 ? req->J.phi_sum : req->J.phi_all + (long long)(m - 1) * p.vec_total;
  return FTHMS_OK;
}

fthms_status fthms_densities(fthms_req* req, int arc, int m, int q, double* out, size_t cap, size_t* needed) {
  if (!req) return fail(FTHMS_EINVAL, "fthms_densities: NULL job");
  if (!req->ctx) return fail(FTHMS_EINVAL, "fthms_densities: the job's context was destroyed");
  const double2* base;
  long long first, last;
  size_t n;
  TRY(density_range(req, arc, m, q, &base, &first, &last, &n));
  if (needed) *needed = n;
  if (!out || cap < n) return fail(FTHMS_EINVAL, "fthms_densities: output buffer too small");
  TRY(wait_results(req));
  const Plan& p = req->plan;
  std::vector<double2> h((size_t)(last - first));
  CK(cudaMemcpyAsync(h.data(), base + first, h.size() * sizeof(double2), cudaMemcpyDeviceToHost, req->stream));
  CK(cudaStreamSynchronize(req->stream));
  size_t o = 0;
  for (int l = p.lb; l < p.le; ++l) {
    const SysDesc& s = p.sys[(size_t)arc * (p.L - 1) + l - 1];
    const double2* src = h.data() + (s.vec_off - first) + (long long)q * s.N;
    for (int i = 0; i < s.N; ++i) {
      out[o++] = src[i].x;
      out[o++] = src[i].y;
    }
  }
  return FTHMS_OK;
}

fthms_status fthms_densities_dev(fthms_req* req, int arc, int m, int q, double* out_dev, size_t cap) {
  if (!req || !out_dev) return fail(FTHMS_EINVAL, "fthms_densities_dev: NULL argument");
  if (!req->ctx) return fail(FTHMS_EINVAL, "fthms_densities_dev: the job's context was destroyed");
  const double2* base;
  long long first, last;
  size_t n;
  TRY(density_range(req, arc, m, q, &base, &first, &last, &n));
  if (cap < n) return fail(FTHMS_EINVAL, "fthms_densities_dev: output buffer too small");
  TRY(ensure_device(req->ctx->device));
  const Plan& p = req->plan;
  size_t o = 0;
  for (int l = p.lb; l < p.le; ++l) {
    const SysDesc& s = p.sys[(size_t)arc * (p.L - 1) + l - 1];
    CK(cudaMemcpyAsync(out_dev + o, base + s.vec_off + (long long)q * s.N, (size_t)s.N * sizeof(double2),
                       cudaMemcpyDeviceToDevice, req->stream));
    o += 2 * (size_t)s.N;
  }
  return FTHMS_OK;
}

fthms_status fthms_node_counts(fthms_req* req, int* out, size_t cap) {
  if (!req || !out) return fail(FTHMS_EINVAL, "fthms_node_counts: NULL argument");
  if (!req->ctx) return fail(FTHMS_EINVAL, "fthms_node_counts: the job's context was destroyed");
  const Plan& p = req->plan;
  if (cap < (size_t)p.P * (p.L - 1)) return fail(FTHMS_EINVAL, "fthms_node_counts: buffer too small");
  for (int j = 0; j < p.P; ++j)
    for (int l = 1; l < p.L; ++l) out[(size_t)j * (p.L - 1) + l - 1] = p.Ntab[(size_t)j * p.L + l];
  return FTHMS_OK;
}

fthms_status fthms_stats(fthms_req* req, fthms_stats_t* out) {
  if (!req || !out) return fail(FTHMS_EINVAL, "fthms_stats: NULL argument");
  if (!req->ctx) return fail(FTHMS_EINVAL, "fthms_stats: the job's context was destroyed");
  const Plan& p = req->plan;
  std::memset(out, 0, sizeof *out);
  out->setup_ms = req->setup_ms;
  out->systems = (long long)p.P * (p.le - p.lb);           // this rank's frequencies
  out->solves = (long long)p.P * (p.le - p.lb) * p.M * p.Q;
  out->kernel_launches = req->launches;
  out->device_bytes = req->bytes;
  out->cross_entries = (double)p.e_total;
  out->hankel_evals = p.hankel_self + p.hankel_cross;
  out->h2d_bytes = req->h2d;
  double lu = 0.0, sv = 0.0;
  for (const SysDesc& s : p.sys) {
    if (!p.own(s.l)) continue;
    lu += (8.0 / 3.0) * (double)s.N * s.N * s.N;
    sv += 8.0 * (double)s.N * s.N * p.Q * p.M;
  }
  out->lu_flops = lu;
  out->solve_flops = sv;
  out->apply_flops = 8.0 * p.Q * p.M * (double)p.e_total;
  out->precision = p.opt.precision;
  out->fallback_runs = req->fallback_runs;
  out->lu_tensor_systems = req->J.mixed ? req->J.n_lu_big : 0;
  if (req->ran) {
    TRY(wait_results(req));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, req->ev0, req->ev1));
    out->gpu_ms = ms;
    if (req->J.mixed) {
      double buf[3] = {0.0, 0.0, 0.0};
      CK(cudaMemcpyAsync(buf, req->J.refine_resid, 3 * sizeof(double), cudaMemcpyDeviceToHost, req->stream));
      CK(cudaStreamSynchronize(req->stream));
      unsigned long long passes = 0, bad = 0;
      std::memcpy(&passes, &buf[1], sizeof passes);
      std::memcpy(&bad, &buf[2], sizeof bad);
      out->max_refine_resid = buf[0];
      out->refine_passes = (double)passes / ((double)req->J.nsys * p.M);
      out->n_unconverged = (long long)bad;
    }
  }
  return FTHMS_OK;
}

fthms_status fthms_result_errors(fthms_req* req, double* out, size_t cap) {
  if (!req || !out) return fail(FTHMS_EINVAL, "fthms_result_errors: NULL argument");
  if (!req->ctx) return fail(FTHMS_EINVAL, "fthms_result_errors: the job's context was destroyed");
  const Plan& p = req->plan;
  const size_t n = (size_t)p.P * (p.L - 1);
  if (cap < n) return fail(FTHMS_EINVAL, "fthms_result_errors: buffer too small");
  if (!req->ran || !req->J.mixed) {
    for (size_t i = 0; i < n; ++i) out[i] = 0.0;
    return req->ran ? FTHMS_OK : fail(FTHMS_EINVAL, "fthms_result_errors: job was never run");
  }
  TRY(wait_results(req));
  if (!req->J.mixed) {                 // replaced by the FP64 fallback
    for (size_t i = 0; i < n; ++i) out[i] = 0.0;
    return FTHMS_OK;
  }
  std::vector<float> e(n);
  CK(cudaMemcpyAsync(e.data(), req->J.sys_err, n * sizeof(float), cudaMemcpyDeviceToHost, req->stream));
  CK(cudaStreamSynchronize(req->stream));
  for (size_t i = 0; i < n; ++i) out[i] = e[i];     // systems are numbered j*(L-1) + l-1
  return FTHMS_OK;
}

fthms_status fthms_set_allreduce(fthms_req* req, fthms_allreduce_fn fn, void* user) {
  if (!req || !fn) return fail(FTHMS_EINVAL, "fthms_set_allreduce: NULL argument");
  if (!req->ctx) return fail(FTHMS_EINVAL, "fthms_set_allreduce: the job's context was destroyed");
  req->allreduce = fn;
  req->allreduce_user = user;
  return FTHMS_OK;
}

fthms_status fthms_release(fthms_req* req) {
  if (!req) return fail(FTHMS_EINVAL, "fthms_release: NULL job");
  if (!req->ctx) {            // detached by fthms_destroy: device memory already freed
    delete req;
    return FTHMS_OK;
  }
  if (req->ran) cudaEventSynchronize(req->ev1);
  free_req(req);
  cudaStreamSynchronize(req->stream);   // the stream-ordered frees have run before the budget is returned
  {
    std::lock_guard<std::mutex> lk(req->ctx->mu);
    req->ctx->in_use -= req->plan.device_bytes;
    req->ctx->live.erase(req);
  }
  delete req;
  return FTHMS_OK;
}

const char* fthms_last_error(void) { return g_last_error.c_str(); }

fthms_status fthms_autotune(fthms_req* req, int reps, int* shapes) {
  if (!req) return fail(FTHMS_EINVAL, "fthms_autotune: NULL job");
  if (!req->ctx) return fail(FTHMS_EINVAL, "fthms_autotune: the job's context was destroyed");
  if (reps < 1) return fail(FTHMS_EINVAL, "fthms_autotune: reps must be >= 1");
  TRY(ensure_device(req->ctx->device));
  if (req->graph) {                    // a captured graph holds the old launch shapes
    cudaGraphExecDestroy(req->graph);
    req->graph = nullptr;
  }
  const bool prof = req->profiling;
  req->profiling = false;
  fthms_status s = enqueue_stages(req);   // valid factors, densities and spectra for every stage
  req->profiling = prof;
  TRY(s);
  CK(cudaStreamSynchronize(req->stream));
  DevJob& J = req->J;
  cudaStream_t st = req->stream;
  int nl = 0;
  struct Knob {
    int* field;
    std::vector<int> cand;
    std::function<cudaError_t()> launch;
  };
  std::vector<Knob> knobs;
  knobs.push_back({&J.shape_solve, {4, 2, 1}, [&] { return launch_solve(J, 1, st, &nl); }});
  if (!J.otf) knobs.push_back({&J.shape_asm, {128, 64, 256}, [&] { return launch_cross_assemble(J, st, &nl); }});
  knobs.push_back({&J.shape_time, {256, 128, 512}, [&] { return launch_synth_fwd(J, st, &nl); }});
  knobs.push_back({&J.shape_restr, {128, 64, 256}, [&] { return launch_restrict(J, st, &nl); }});
  // Mixed forms: the smallest N factored with tensor-core updates (candidates above 800 keep the default,
  // the one-CTA LU cannot hold more); every candidate factors the same matrices, its time is compared.
  int lu_min = kLuBigMin;
  // the number of systems (a prefix of sys_order, decreasing N) with at least nmin nodes; lives as long as
  // the knobs that call it
  const Plan& plan = req->plan;
  auto split_for = [&plan](int nmin) {
    int nb = 0;
    while (nb < (int)plan.sys_order.size() && plan.sys[plan.sys_order[nb]].N >= nmin) ++nb;
    return nb;
  };
  if (J.mixed) {
    std::vector<int> cand{kLuBigMin};
    for (int c : {512, 384, 256})
      if (!plan.sys_order.empty() && plan.sys[plan.sys_order[0]].N >= c) cand.push_back(c);
    if (cand.size() > 1) {
      knobs.push_back({&lu_min, cand, [&] {
                         set_lu_split(req, split_for(lu_min));
                         // the LU works in place: re-assemble the matrices before every factorisation
                         cudaError_t e = launch_assemble_self(J, st, &nl);
                         return e == cudaSuccess ? launch_lu(J, st, &nl) : e;
                       }});
    }
  }
  for (Knob& k : knobs) {
    float best = 0.f;
    int pick = k.cand[0];
    for (int c : k.cand) {
      *k.field = c;
      float ms = 0.f;
      TRY(time_stage(req, reps, &ms, k.launch));
      if (c == k.cand[0] || ms < best) {
        best = ms;
        pick = c;
      }
    }
    *k.field = pick;
  }
  set_lu_split(req, J.mixed ? split_for(lu_min) : 0);
  req->lu_min = lu_min;
  if (shapes) {
    shapes[0] = J.shape_solve;
    shapes[1] = J.shape_asm;
    shapes[2] = J.shape_time;
    shapes[3] = J.shape_restr;
    shapes[4] = J.mixed ? req->lu_min : 0;
  }
  return FTHMS_OK;
}

fthms_status fthms_set_shapes(fthms_req* req, const int* shapes) {
  if (!req || !shapes) return fail(FTHMS_EINVAL, "fthms_set_shapes: NULL argument");
  if (!req->ctx) return fail(FTHMS_EINVAL, "fthms_set_shapes: the job's context was destroyed");
  if (!shapes_valid(shapes, req->plan.opt.precision >= 1))
    return fail(FTHMS_EINVAL, "fthms_set_shapes: a choice outside its candidates");
  if (req->graph) {                    // a captured graph holds the old launch shapes
    cudaGraphExecDestroy(req->graph);
    req->graph = nullptr;
  }
  apply_shapes(req, shapes);
  return FTHMS_OK;
}

fthms_status fthms_use_fused(fthms_req* req, int enable) {
  if (!req) return fail(FTHMS_EINVAL, "fthms_use_fused: NULL job");
  if (!req->ctx) return fail(FTHMS_EINVAL, "fthms_use_fused: the job's context was destroyed");
  if (enable && req->plan.opt.precision != 0)
    return fail(FTHMS_EINVAL, "fthms_use_fused: the fused kernel is the FP64 form's (precision 0)");
  if (req->graph) {                    // a captured graph holds the other stage sequence
    cudaGraphExecDestroy(req->graph);
    req->graph = nullptr;
  }
  req->use_fused = enable != 0;
  return FTHMS_OK;
}

fthms_status fthms_use_graph(fthms_req* req, int enable) {
  if (!req) return fail(FTHMS_EINVAL, "fthms_use_graph: NULL job");
  if (!req->ctx) return fail(FTHMS_EINVAL, "fthms_use_graph: the job's context was destroyed");
  req->use_graph = enable != 0;
  return FTHMS_OK;
}

fthms_status fthms_profile(fthms_req* req, int enable) {
  if (!req) return fail(FTHMS_EINVAL, "fthms_profile: NULL job");
  if (!req->ctx) return fail(FTHMS_EINVAL, "fthms_profile: the job's context was destroyed");
  TRY(flush_marks(req));
  if (enable) {
    for (int k = 0; k < FTHMS_NSTAGES; ++k) {
      req->stage_ms[k] = 0.0;
      req->stage_launches[k] = 0;
    }
  }
  req->profiling = enable != 0;
  return FTHMS_OK;
}

fthms_status fthms_stage_times(fthms_req* req, double* ms, long long* launches) {
  if (!req || !ms || !launches) return fail(FTHMS_EINVAL, "fthms_stage_times: NULL argument");
  if (!req->ctx) return fail(FTHMS_EINVAL, "fthms_stage_times: the job's context was destroyed");
  TRY(flush_marks(req));
  for (int k = 0; k < FTHMS_NSTAGES; ++k) {
    ms[k] = req->stage_ms[k];
    launches[k] = req->stage_launches[k];
  }
  return FTHMS_OK;
}

fthms_status fthms_bessel0(const double* z_dev, double* j0_dev, double* y0_dev, double* yhat0_dev, int n,
                           void* cuda_stream) {
  if (n < 0 || (n > 0 && !z_dev)) return fail(FTHMS_EINVAL, "fthms_bessel0: bad arguments");
  int dev = 0;
  CK(cudaGetDevice(&dev));
  TRY(ensure_device(dev));
  CK(launch_bessel0(z_dev, j0_dev, y0_dev, yhat0_dev, n, static_cast<cudaStream_t>(cuda_stream)));
  return FTHMS_OK;
}

fthms_status fthms_assemble_self(const fthms_curve* curve, const fthms_arc* arc, int N, double kappa,
                                 double* A_dev, void* cuda_stream) {
  if (!curve || !arc || !A_dev || !curve->ax || !curve->bx || !curve->ay || !curve->by || curve->degree < 1 ||
      N < 2 || N > 1024 || !(kappa > 0) || !(arc->theta_b > arc->theta_a))
    return fail(FTHMS_EINVAL, "fthms_assemble_self: bad arguments");
  int dev = 0;
  CK(cudaGetDevice(&dev));
  TRY(ensure_device(dev));
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  Curve c;
  c.ax.assign(curve->ax, curve->ax + curve->degree + 1);
  c.bx.assign(curve->bx, curve->bx + curve->degree + 1);
  c.ay.assign(curve->ay, curve->ay + curve->degree + 1);
  c.by.assign(curve->by, curve->by + curve->degree + 1);
  std::vector<double> t, x, y, sp;
  arc_nodes(c, arc->theta_a, arc->theta_b, N, t, x, y, sp);
  fthms_req tmp;
  tmp.stream = st;
  DevJob& J = tmp.J;
  std::vector<SysDesc> sys(1);
  // One system in a band of length 1 at frequency index 1 with step h = kappa: the band kernel's
  // kappa = l h, ln l = 0 and the recurrence step h R all refer to this kappa.
  sys[0].arc = 0; sys[0].l = 1; sys[0].N = N; sys[0].panel = 0; sys[0].mat_off = 0; sys[0].vec_off = 0;
  sys[0].piv_off = 0; sys[0].rlog_off = 0; sys[0].kappa = kappa;
  std::vector<Panel> panels(1, Panel{0, N, 0});
  std::vector<int> rlogN(1, N);
  std::vector<long long> rlog_off(1, 0);
  std::vector<SelfTile> tiles;
  int nt = (N + kSelfTile - 1) / kSelfTile;
  for (int a = 0; a < nt; ++a)
    for (int b = a; b < nt; ++b) tiles.push_back(SelfTile{0, 1, a, b});
  fthms_status s = FTHMS_OK;
  if (s == FTHMS_OK) s = dev_upload(&tmp, sys, &J.sys);
  if (s == FTHMS_OK) s = dev_upload(&tmp, panels, &J.panels);
  if (s == FTHMS_OK) s = dev_upload(&tmp, t, &J.node_t);
  if (s == FTHMS_OK) s = dev_upload(&tmp, x, &J.node_x);
  if (s == FTHMS_OK) s = dev_upload(&tmp, y, &J.node_y);
  if (s == FTHMS_OK) s = dev_upload(&tmp, sp, &J.node_sp);
  if (s == FTHMS_OK) s = dev_upload(&tmp, rlogN, &J.rlogN);
  if (s == FTHMS_OK) s = dev_upload(&tmp, rlog_off, &J.rlog_off_N);
  if (s == FTHMS_OK) s = dev_upload(&tmp, tiles, &J.tiles);
  if (s == FTHMS_OK) s = dev_alloc(&tmp, (size_t)N * N, &J.rlog);
  if (s == FTHMS_OK) {
    J.A = reinterpret_cast<double2*>(A_dev);
    J.h = kappa;
    J.n_rlogN = 1;
    J.n_tiles = (int)tiles.size();
    J.max_n = N;
    J.K = 16;  // unused FFT tables are not launched below
    int nl = 0;
    cudaError_t e = launch_tables_rlog_only(J, st, &nl);
    if (e == cudaSuccess) e = launch_assemble_self(J, st, &nl);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_fail(e, "fthms_assemble_self");
  }
  free_req(&tmp);
  return s;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Request server: continuous admission of jobs onto per-slot streams under the HBM budget.

namespace {

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct ServerReq {
  long long id = 0;
  // owned copies of the inputs (the caller may free its buffers after submit)
  std::vector<std::vector<double>> coef;
  std::vector<fthms_curve> curves;
  std::vector<fthms_arc> arcs;
  fthms_signal sig{};
  std::vector<double> sig_f;    // samples of a sampled signal
  fthms_options opt{};
  std::vector<double> obs;
  fthms_req* req = nullptr;
  int state = 0;            // 0 queued, 1 running, 2 done, 3 failed
  int slot = -1;
  fthms_status err = FTHMS_OK;
  std::string msg;
  double t_submit = 0, t_start = 0, t_done = 0;
};

}  // namespace

struct fthms_server {
  fthms_ctx* ctx = nullptr;
  int max_inflight = 1;
  std::vector<cudaStream_t> streams;
  std::vector<int> slot_used;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<long long> queue;
  std::map<long long, ServerReq*> reqs;
  long long next_id = 1;
  bool stop = false;
  bool retry = true;          // admission worth retrying (a job finished, was released or arrived)
  cudaStream_t upload = nullptr;
  std::thread worker;
};

namespace {

// One scheduling pass (called with the server lock held): retire finished jobs, then admit queued
// jobs in arrival order while a slot is free and the context's HBM budget has room.
void server_pass(fthms_server* s) {
  for (auto& kv : s->reqs) {
    ServerReq* q = kv.second;
    if (q->state != 1) continue;
    cudaError_t e = cudaEventQuery(q->req->ev1);
    if (e == cudaErrorNotReady) continue;
    q->t_done = now_ms();
    q->state = e == cudaSuccess ? 2 : 3;
    if (e != cudaSuccess) {
      q->err = FTHMS_ECUDA;
      q->msg = cudaGetErrorString(e);
    }
    s->slot_used[q->slot] = 0;
    s->retry = true;
    s->cv.notify_all();
  }
  while (!s->queue.empty() && s->retry) {
    int slot = -1;
    for (int i = 0; i < s->max_inflight; ++i)
      if (!s->slot_used[i]) { slot = i; break; }
    if (slot < 0) return;
    ServerReq* q = s->reqs[s->queue.front()];
    fthms_req* r = nullptr;
    // plan first: a job that cannot fit even an empty budget fails; one that does not fit now waits
    fthms_status st = fthms_prepare(s->ctx, q->curves.data(), (int)q->curves.size(), q->arcs.data(),
                                    (int)q->arcs.size(), &q->sig, &q->opt, &r);
    if (st == FTHMS_ENOMEM) {
      bool alone_fits = s->ctx->budget == 0 || s->ctx->in_use == 0;
      if (!alone_fits) {       // wait until a running or resident job finishes or is released
        s->retry = false;
        return;
      }
    }
    s->queue.pop_front();
    if (st != FTHMS_OK) {
      q->state = 3;
      q->err = st;
      q->msg = g_last_error;
      q->t_done = now_ms();
      s->cv.notify_all();
      continue;
    }
    // move the job to the slot's stream: its uploads were issued on the context stream
    cudaStreamSynchronize(r->stream);
    r->stream = s->streams[slot];
    st = fthms_run(r);
    if (st != FTHMS_OK) {
      q->state = 3;
      q->err = st;
      q->msg = g_last_error;
      q->t_done = now_ms();
      fthms_release(r);
      s->cv.notify_all();
      continue;
    }
    q->req = r;
    q->slot = slot;
    q->state = 1;
    q->t_start = now_ms();
    s->slot_used[slot] = 1;
  }
}

void server_loop(fthms_server* s) {
  cudaSetDevice(s->ctx->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    server_pass(s);
    s->cv.wait_for(lk, std::chrono::microseconds(100));
  }
}

ServerReq* find_req(fthms_server* s, long long id) {
  auto it = s->reqs.find(id);
  return it == s->reqs.end() ? nullptr : it->second;
}

}  // namespace

extern "C" {

fthms_status fthms_server_create(fthms_server** out, int device, size_t hbm_budget_bytes, int max_inflight) {
  if (!out || max_inflight < 1 || max_inflight > 64) return fail(FTHMS_EINVAL, "fthms_server_create: bad arguments");
  *out = nullptr;
  fthms_server* s = new fthms_server;
  fthms_status st = fthms_create(&s->ctx, device, hbm_budget_bytes, nullptr);
  if (st != FTHMS_OK) {
    delete s;
    return st;
  }
  s->max_inflight = max_inflight;
  s->upload = s->ctx->stream;     // the context's own stream carries the uploads of admitted jobs
  s->streams.resize(max_inflight);
  s->slot_used.assign(max_inflight, 0);
  for (int i = 0; i < max_inflight; ++i) {
    cudaError_t e = cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      for (int k = 0; k < i; ++k) cudaStreamDestroy(s->streams[k]);
      fthms_destroy(s->ctx);
      delete s;
      return cuda_fail(e, "cudaStreamCreate");
    }
  }
  s->worker = std::thread(server_loop, s);
  *out = s;
  return FTHMS_OK;
}

fthms_status fthms_server_submit(fthms_server* s, const fthms_curve* curves, int ncurves, const fthms_arc* arcs,
                                 int narcs, const fthms_signal* signal, const fthms_options* options,
                                 long long* ticket) {
  if (!s || !ticket || !curves || ncurves <= 0 || !arcs || narcs <= 0 || !signal || !options)
    return fail(FTHMS_EINVAL, "fthms_server_submit: NULL or empty argument");
  ServerReq* q = new ServerReq;
  for (int c = 0; c < ncurves; ++c) {
    if (curves[c].degree < 1) {
      delete q;
      return fail(FTHMS_EINVAL, "fthms_server_submit: curve degree < 1");
    }
    const int n = curves[c].degree + 1;
    for (const double* src : {curves[c].ax, curves[c].bx, curves[c].ay, curves[c].by}) {
      if (!src) {
        delete q;
        return fail(FTHMS_EINVAL, "fthms_server_submit: NULL curve coefficients");
      }
      q->coef.emplace_back(src, src + n);
    }
  }
  for (int c = 0; c < ncurves; ++c) {
    fthms_curve cv;
    cv.degree = curves[c].degree;
    cv.ax = q->coef[4 * c].data();
    cv.bx = q->coef[4 * c + 1].data();
    cv.ay = q->coef[4 * c + 2].data();
    cv.by = q->coef[4 * c + 3].data();
    q->curves.push_back(cv);
  }
  q->arcs.assign(arcs, arcs + narcs);
  q->sig = *signal;
  if (signal->n_t > 0 && signal->f) {
    q->sig_f.assign(signal->f, signal->f + signal->n_t);
    q->sig.f = q->sig_f.data();
  }
  q->opt = *options;
  if (options->n_obs > 0 && options->obs_xy) q->obs.assign(options->obs_xy, options->obs_xy + 2 * options->n_obs);
  q->opt.obs_xy = q->obs.empty() ? nullptr : q->obs.data();
  q->t_submit = now_ms();
  std::lock_guard<std::mutex> lk(s->mu);
  q->id = s->next_id++;
  s->reqs[q->id] = q;
  s->queue.push_back(q->id);
  *ticket = q->id;
  s->retry = true;
  s->cv.notify_all();
  return FTHMS_OK;
}

fthms_status fthms_server_poll(fthms_server* s, long long ticket, int* state) {
  if (!s || !state) return fail(FTHMS_EINVAL, "fthms_server_poll: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  ServerReq* q = find_req(s, ticket);
  if (!q) return fail(FTHMS_EINVAL, "fthms_server_poll: unknown ticket");
  *state = q->state;
  return FTHMS_OK;
}

fthms_status fthms_server_wait(fthms_server* s, long long ticket, int timeout_ms) {
  if (!s) return fail(FTHMS_EINVAL, "fthms_server_wait: NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    ServerReq* q = find_req(s, ticket);
    if (!q) return fail(FTHMS_EINVAL, "fthms_server_wait: unknown ticket");
    if (q->state == 2) return FTHMS_OK;
    if (q->state == 3) return fail(q->err, "fthms_server_wait: request failed: " + q->msg);
    if (timeout_ms >= 0 &&
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count() > timeout_ms)
      return fail(FTHMS_ETIMEOUT, "fthms_server_wait: timed out");
    s->cv.wait_for(lk, std::chrono::microseconds(200));
  }
}

fthms_status fthms_server_result(fthms_server* s, long long ticket, fthms_req** req) {
  if (!s || !req) return fail(FTHMS_EINVAL, "fthms_server_result: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  ServerReq* q = find_req(s, ticket);
  if (!q) return fail(FTHMS_EINVAL, "fthms_server_result: unknown ticket");
  if (q->state != 2) return fail(q->state == 3 ? q->err : FTHMS_EBUSY, "fthms_server_result: request not done");
  *req = q->req;
  return FTHMS_OK;
}

fthms_status fthms_server_latency(fthms_server* s, long long ticket, double* queue_ms, double* total_ms) {
  if (!s || !queue_ms || !total_ms) return fail(FTHMS_EINVAL, "fthms_server_latency: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  ServerReq* q = find_req(s, ticket);
  if (!q) return fail(FTHMS_EINVAL, "fthms_server_latency: unknown ticket");
  if (q->state < 2) return fail(FTHMS_EBUSY, "fthms_server_latency: request not finished");
  *queue_ms = (q->state == 2 ? q->t_start : q->t_done) - q->t_submit;
  *total_ms = q->t_done - q->t_submit;
  return FTHMS_OK;
}

fthms_status fthms_server_release(fthms_server* s, long long ticket) {
  if (!s) return fail(FTHMS_EINVAL, "fthms_server_release: NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  ServerReq* q = find_req(s, ticket);
  if (!q) return fail(FTHMS_EINVAL, "fthms_server_release: unknown ticket");
  if (q->state < 2) return fail(FTHMS_EBUSY, "fthms_server_release: request still queued or running");
  if (q->req) fthms_release(q->req);
  s->reqs.erase(ticket);
  delete q;
  s->retry = true;
  s->cv.notify_all();
  return FTHMS_OK;
}

fthms_status fthms_server_destroy(fthms_server* s) {
  if (!s) return fail(FTHMS_EINVAL, "fthms_server_destroy: NULL server");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  s->worker.join();
  for (auto& kv : s->reqs) {
    ServerReq* q = kv.second;
    if (q->req) {
      cudaEventSynchronize(q->req->ev1);
      fthms_release(q->req);
    }
    delete q;
  }
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  fthms_destroy(s->ctx);
  delete s;
  return FTHMS_OK;
}

}  // extern "C"
