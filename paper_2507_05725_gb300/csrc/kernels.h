// Launch wrappers of the FTH-MS CUDA kernels (host-callable, C++ linkage, device pointers).
#pragma once
#include <cuda_runtime.h>

#include "common.h"

namespace fthms {

// Device-side view of one job: every pointer is device memory owned by the job.
struct DevJob {
  int P, L, Q, K, NT, M, n_obs, n_tout, nsys, n_act, n_grp, n_asm, n_tiles, n_rlogN, n_restr;
  int logK, max_nmax, max_n, acc_cap;
  int row_cap, ph_cap;           // max rows and max sum of source N over the cross groups
  int mixed;                     // 1: mixed-precision form (FP32 LU + double-float refinement/apply)
  int fp64keep;                  // mixed form with FP64 kept for the small-argument Hankel series, the
                                 // refinement residuals and the FFT butterflies (precision 2)
  double refine_tol;             // stop refining once the estimated relative error left is below this
  int refine_max;                // at most this many refinement passes per system and step
  long long mat_total;
  double h, dt, sign;
  // signal
  int sig_kind;
  double z0x, z0y, dirx, diry, amp, carrier, centre, width;
  int sig_nt;                    // > 0: sampled signal f[0..sig_nt) at sig_t0 + i sig_dt
  double sig_t0, sig_dt, sig_band;
  const double* sig_f;
  // tables
  const SysDesc* sys;
  const int* sys_order;       // systems by decreasing N (launch order of the solves and restriction)
  const int* lu_small;        // systems factored by one CTA each (k_lu), decreasing N
  const int* lu_big;          // mixed forms: systems above kLuBigMin, factored with tensor-core updates
  int n_lu_small, n_lu_big, big_max_n;
  int* dev_err;               // set by a kernel whose bounded wait ran out (reported by fthms_wait)
  int* work_counter;          // the fused kernel's next-system counter
  const Panel* panels;
  const double *node_t, *node_x, *node_y, *node_sp;
  const int* rlogN;
  const long long* rlog_off_N;
  double* rlog;
  const int* restr_N;        // [n_restr][2] (N, Nmax)
  const long long* restr_off;
  double* restr;             // transposed tables RT[x][i]
  float2* restr_df;          // the same as double-float pairs (mixed form)
  const long long* restr_of_sys;
  const SelfTile* tiles;
  const CrossTgt* tgts;
  const PairDesc* pairs;
  const long long* e_off;
  const CrossAsm* asms;
  const CrossGrp* grps;
  const CrossBlk* blks;
  const ApplySlice* slices;  // mixed-form apply: row slices of the groups
  const long long* grp_res_off;
  double2* apply_res;        // [group rows][Q] per-row cross sums (mixed form)
  int n_slices, slice_ph_cap;
  // cross_mode 1: cross rows evaluated every step (nothing stored)
  int otf, n_otf;
  // launch shapes chosen by fthms_autotune (0 = built-in default): warps per solve block, threads per
  // cross-assembly block, per time-transform block and per restriction block
  int shape_solve, shape_asm, shape_time, shape_restr;
  const CrossOtf* otf_tasks;
  const long long* wn_off;   // per assembly task: near weights offset or -1
  double* wn;                // near weights, nrows x N per assembly task with near rows
  const long long* otf_res_off;
  const int* tpanel;
  const long long* tr_off;
  const double* chi;
  const int *act_off, *act_idx, *act_arc;
  const double* win;         // [Q][NT]
  const double* wl;          // [L]
  const double* c_q;         // [Q]
  const int* nlo;            // [Q]
  const double* tout;        // [n_tout]
  const double* s_q;         // [Q]
  double H, period;
  // work arrays
  double2* A;                // LU factors (mixed form: the matrix itself, as double-float)
  float2* LU32;              // FP32 factors (mixed form)
  float2* dinv32;            // FP32 1 / U_kk (mixed form)
  double* refine_resid;      // [0] max estimated error left, [1] refinement passes, [2] unconverged
                             // (system, step) pairs (64-bit integers in [1], [2]; mixed form)
  float* sys_err;            // per system: max over steps of the estimated relative error left (mixed form)
  float2* rres;              // FP32-rounded refinement residuals, laid out like G (mixed form)
  double2* rres64;           // FP64-kept systems: the residual the next pass updates, laid out like G
  float2* dcorr;             // FP64-kept systems: the last FP32 correction, laid out like G
  int* mdone;                // per system: 1 once its refinement has finished this step (mixed form)
  float* mrel;               // per system: relative size of its last correction (mixed form)
  float* mrho;               // per system: largest contraction factor measured in earlier steps (0: none yet)
  double* mscale;            // per system and step: power of two near max |G|; refinement runs in G / mscale
  float2* arow;              // FP64-kept systems, per row (once per job): upper bounds of the 1-norm and the 2-norm
                             // of the row's 2N real components (|Re a_ij|, |Im a_ij|)
  float2* phistat;           // FP64-kept systems, per system and window (4 slots a system, every step): max |component|
                             // and an upper bound of the 2-norm of the pass-0 FP32 solution
  int f64_min_n;             // mixed forms: systems of at least this N keep FP64 matrices and residuals
  const ResidChunk* rchunks; // 32-row chunks of the systems, largest first (mixed form)
  int n_rchunks;
  int* piv;
  double2* dinv;             // 1 / U_kk
  double2* G;                // data on solve nodes [s][q][i]
  double2* phi;              // current densities
  float4* phi_df;            // the same as double-float pairs, written by the mixed solve for the apply
  double2* phi_sum;
  double2* phi_all;          // [m][...] or null
  double2* W;                // cross fields at transfer nodes [(tr_off+x)*Q+q]*L+l
  double2* Gt;               // transfer-node spectra (same layout)
  double* ginc;              // m = 1 time samples sign chi_k u^i at the active transfer nodes [a][NT]
  double2* E;                // cross matrices
  double2* Vobs;             // [z][q][l]
  double* traces;            // [z][tout]
  double2* fft_tw;           // K/2 twiddles e^{-2 pi i r/K}
  float4* fft_tw_df;         // the same as double-float pairs (mixed form)
  double2* syn_tw;           // [Q][L]
  double2* fwd_tw;           // [Q][L]
  long long vec_total;
};

cudaError_t init_constants();

// Sets the calling thread's message returned by fthms_last_error() (defined with the C ABI).
void set_last_error(const char* msg);

cudaError_t launch_bessel0(const double* z, double* j0, double* y0, double* yh, int n, cudaStream_t st);

// Individual pipeline stages (all asynchronous on `st`).
cudaError_t launch_tables(const DevJob& J, cudaStream_t st, int* launches);
cudaError_t launch_tables_rlog_only(const DevJob& J, cudaStream_t st, int* launches);
cudaError_t launch_assemble_self(const DevJob& J, cudaStream_t st, int* launches);
cudaError_t launch_lu(const DevJob& J, cudaStream_t st, int* launches);
// The one-CTA LU of the systems below the tensor-core split (all systems in the FP64 form).
cudaError_t launch_lu_small(const DevJob& J, cudaStream_t st, int* launches);
// Mixed forms, systems above the split: blocked LU with tcgen05 trailing updates (lu_large.cu), as one
// sequence or panel by panel (panel k: columns 32k .. 32k+31, then the trailing update; then the finish).
cudaError_t launch_lu_large(const DevJob& J, cudaStream_t st, int* launches);
int lu_big_panels(const DevJob& J);
cudaError_t launch_lu_big_panel(const DevJob& J, int panel, cudaStream_t st, int* launches);
cudaError_t launch_lu_big_update(const DevJob& J, int panel, cudaStream_t st, int* launches);
cudaError_t launch_lu_big_finish(const DevJob& J, cudaStream_t st, int* launches);
size_t lu_big_panel_smem(int maxN);
// Plain FP64 form, batching: self assembly, LU and the step-1 solve of every system in one persistent launch
// (counter: one device int, reset on the stream before the launch).
cudaError_t launch_fused_asf(const DevJob& J, int* counter, cudaStream_t st, int* launches);
cudaError_t launch_cross_assemble(const DevJob& J, cudaStream_t st, int* launches);
cudaError_t launch_incident(const DevJob& J, cudaStream_t st, int* launches);
cudaError_t launch_restrict(const DevJob& J, cudaStream_t st, int* launches);
cudaError_t launch_solve(const DevJob& J, int m, cudaStream_t st, int* launches);
// Mixed forms, the same step piece by piece: launch_msolve(pass 0), then for pass = 1 .. refine_passes(J)
// launch_resid(pass) and launch_msolve(pass).
int refine_passes(const DevJob& J);
cudaError_t launch_msolve(const DevJob& J, int m, int pass, cudaStream_t st, int* launches);
cudaError_t launch_resid(const DevJob& J, int pass, cudaStream_t st, int* launches);
cudaError_t launch_cross_apply(const DevJob& J, cudaStream_t st, int* launches);
cudaError_t launch_near_weights(const DevJob& J, cudaStream_t st, int* launches);
cudaError_t launch_cross_otf(const DevJob& J, cudaStream_t st, int* launches);
cudaError_t launch_synth_fwd(const DevJob& J, cudaStream_t st, int* launches);
// Frequency-partitioned jobs: the partial synthesis into J.ginc, then (after the ranks' sum) the rest.
cudaError_t launch_synth_partial(const DevJob& J, cudaStream_t st, int* launches);
cudaError_t launch_fwd_after_sum(const DevJob& J, cudaStream_t st, int* launches);
cudaError_t launch_traces(const DevJob& J, cudaStream_t st, int* launches);

}  // namespace fthms
