/*
 * fthms.h -- C ABI of the GB300 (sm_103a) FTH-MS open-arc hot path.
 *
 * The library runs the data-parallel core of the frequency-time hybrid multiple-scattering
 * method of arxiv 2507.05725 (FTH-MS, Algorithm 1 and Sections 3.1-4.3): for every open arc
 * Gamma_j and every frequency omega_l it assembles the log-split Chebyshev Nystrom matrix of the
 * single-layer operator V_Gamma_j (eq. FDBIEk-interior), factors it once, and then for each
 * multiple-scattering step m and time window q solves for the density, evaluates the arc's
 * potential S_Gamma_j (eq. FDsolk-interior) on the other arcs and at observation points,
 * synthesises it back to time with recentring (eq. TDsol), applies the partition-of-unity and
 * overlap masks of eqs. criterion_int2 / vtilde and takes the windowed slow transform
 * (eq. Fourierk) that is the next step's data.
 *
 * Conventions shared by every call:
 *  - Plain C types only; every pointer argument is a HOST pointer unless its name ends in _dev.
 *  - All inputs are copied before the call returns; the caller may free them immediately.
 *  - Outputs go into caller-owned buffers whose capacity (in doubles) is passed; when it is too
 *    small the call returns FTHMS_EINVAL and writes the required size to *needed if given.
 *  - Errors are status codes only; fthms_last_error() returns a message for the calling thread.
 *  - Complex values are interleaved (re, im) doubles.
 *  - Wave speed c = 1, so kappa = omega.  Time convention of eqs. forwardFT/backwardFT:
 *    G(omega) = int g(t) e^{i omega t} dt; the kernel is (i/4) H0^(1)(kappa |x - y|).
 */
#ifndef FTHMS_H
#define FTHMS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FTHMS_OK = 0,
  FTHMS_EINVAL = 1,   /* invalid argument, geometry or option (nothing was enqueued) */
  FTHMS_ENOMEM = 2,   /* the job does not fit the context's HBM budget or device memory */
  FTHMS_ENOCONV = 3,  /* fthms_wait: the job finished, but the iterative refinement of some (arc, omega)
                         systems (mixed forms) did not reach refine_tol within refine_max passes */
  FTHMS_ETIMEOUT = 4, /* fthms_wait: the job did not finish within the timeout */
  FTHMS_ECUDA = 5,    /* a CUDA runtime call failed; the message names it */
  FTHMS_EBUSY = 6,    /* results requested before the job finished */
  FTHMS_ENOTIMPL = 7  /* option value not implemented in this build */
} fthms_status;

typedef struct fthms_ctx fthms_ctx; /* device, stream, memory budget */
typedef struct fthms_req fthms_req; /* one FTH-MS job and its device-resident state */

/* Closed or open curve X(theta) = sum_{k=0}^{degree} (ax[k] cos k theta + bx[k] sin k theta,
 * ay[k] cos k theta + by[k] sin k theta); each array has degree+1 entries (b[0] is ignored).
 * Covers circles, ellipses, the kite and r = 1 + a cos(n theta + p) stars exactly. */
typedef struct {
  int degree;
  const double* ax;
  const double* bx;
  const double* ay;
  const double* by;
} fthms_curve;

/* Overlapping patch Gamma_j = X([theta_a, theta_b]) of curve `curve` (Section 3.1): theta_b >
 * theta_a, theta may exceed 2 pi.  Arcs of one curve must each overlap exactly their cyclic
 * neighbours; an arc alone on its curve is an open-arc obstacle (chi = 1). */
typedef struct {
  int curve;
  double theta_a, theta_b;
} fthms_arc;

/* Incident field u^i(x, t) of a real time signal f (Section 2's boundary data; Section 5's incident-field
 * families): kind 0 = point source at z0: u = (1/(2 pi)) int_0^inf f(t - |x - z0| cosh v) dv (the 2-D
 * retarded field, evaluated by the trapezoid rule in v), kind 1 = plane wave along unit vector dir:
 * u = f(t - x.dir).  Boundary data g_{j,1} = sign chi_j u^i (eq. criterion_int1 has sign = -1).
 * The signal is either
 *  - analytic (n_t = 0): f(t) = amp sin(carrier t) exp(-((t - centre)/width)^2), width > 0; or
 *  - sampled (n_t >= 8): f[i] = f(t0 + i dt), i = 0..n_t-1 (host array, copied at prepare), dt > 0.
 *    Between the samples f is the degree-7 Lagrange interpolant through the 8 samples whose indices
 *    are floor(s) - 3 .. floor(s) + 4, s = (t - t0)/dt (indices outside 0..n_t-1 count as zero
 *    samples), and f = 0 outside [t0, t0 + (n_t - 1) dt].  band > 0 is the highest angular frequency
 *    that the signal carries (it sets the point-source rule's step, as carrier + 8/width does for the
 *    analytic signal); amp, carrier, centre and width are ignored.
 * The point-source rule integrates over the v-range where f(t - |x - z0| cosh v) can be nonzero (the
 * analytic signal: |tau - (t - centre)| <= 8 width; the sampled one: its sample range) with
 * n = ceil((v_hi - v_lo)(1.25 rate + 24)/pi) + 16 intervals, rate = B |x - z0| sinh(v_hi) + 1,
 * B = |carrier| + 8/width or band. */
typedef struct {
  int kind;
  double z0[2];
  double dir[2];
  double sign;
  double amp, carrier, centre, width;
  int n_t;            /* 0: analytic signal; >= 8: sampled signal */
  double t0, dt;
  const double* f;
  double band;
} fthms_signal;

/* Discretisation and output options.
 *  W, L      : frequencies omega_l = l*(W/(L-1)), l = 0..L-1; l = 1..L-1 are solved.
 *  N rule    : nodes per arc N_j(omega) = N_fixed if > 0, else max(N_min, ceil(N_ppw*omega*len_j)
 *              + N_off), len_j the arc length; every N_j(omega) must lie in [2, 800] (precision 0) or
 *              [2, 2048] (precisions 1 and 2; stored cross rows, cross_mode 0, need N <= 1427).  The transfer
 *              mesh of arc j is its first-kind Chebyshev grid of size N_j(omega_{L-1}).
 *  M         : multiple-scattering steps (Algorithm 1's outer loop).
 *  Q, H      : 1 <= Q <= 4 time windows sqcap_q(t) = sqcap(t - s_q), s_q = 1.5 (q-1) H (Section 5).
 *  n_period  : internal time samples per period 2 pi/h of the frequency grid (power of two,
 *              16..16384); dt = 2 pi/(h n_period), t_n = -H + n dt covering [-H, s_Q + H].  The time
 *              kernels keep one period and these N_T samples of a node in shared memory:
 *              16 n_period + 8 N_T <= 232448 bytes, else EINVAL.
 *  obs_xy    : n_obs observation points (x, y), host array of 2*n_obs doubles.
 *  n_tout, tout0, dtout : output times tout0 + k dtout of the traces u_M(z, t) (eq. mult-scatt-int).
 *  precision : 0 = FP64 throughout.  1 = mixed form: FP32 LU factors; solutions refined against the
 *              matrix kept as double-float (two floats, ~48 bits) until the relative error estimated
 *              to remain (last correction x estimated contraction factor) is below refine_tol, at most
 *              refine_max steps; self and cross entries (Taylor range and far-field recurrence), the
 *              refinement residuals, the FFT butterflies of the time transforms, the restriction and the
 *              cross apply in double-float on the FP32 pipe; diagonal self entries, per-pair setup,
 *              phase-seed reduction, log-singular corrections, transform folds and phase factors stay
 *              FP64.  The refinement solves the double-float matrix exactly; its rounding (~2^-44 of an
 *              entry) still reaches the densities through the matrix's conditioning, so the systems with
 *              N > 800 (factored with tensor-core updates, conditioning growing with N) keep FP64 matrices
 *              and FP64 residuals as in form 2.  N > 800 (up to 2048): FP32 LU with tcgen05 (3xTF32)
 *              trailing updates, precisions 1 and 2 only.  2 = the mixed form
 *              with FP64 kept where accuracy is decided: the self matrices assembled and kept in FP64 (the
 *              FP32 factor is their rounding) with FP64 refinement residuals, the small-argument (z < 20)
 *              Hankel series of the stored cross entries, and the FFT butterflies of the time transforms
 *              (everything else as in 1).  Others -> ENOTIMPL.
 *  keep_densities : 1 keeps phi_{j,m,q}(omega_l) of every step for fthms_densities; 0 keeps only
 *              the sum over m.
 *  cross_mode: 0 = the cross-arc and observation rows of eq. FDsolk-interior are assembled once per job,
 *              stored in device memory and applied every step (fast while they fit: 16 bytes per
 *              entry).  1 = they are evaluated again in every step and summed at once, nothing stored
 *              (for jobs whose cross rows do not fit, e.g. many arcs on one curve at high frequency).
 *              Both modes give the same densities to rounding.  Others -> EINVAL.
 *  refine_tol, refine_max : mixed forms: a system stops refining once the estimated relative error left
 *              is below refine_tol (0 = 1e-12), after at most refine_max passes (0 = 3; at most 16).  The
 *              estimate is the last correction's relative size times the contraction factor: the ratio
 *              of the last two corrections; after the first correction, twice the largest ratio measured
 *              for the system in an earlier step of the run, or (first step) 10 x the correction's size.
 *  refine_fallback : mixed forms: 0 = a job in which some system did not meet refine_tol within
 *              refine_max passes finishes with those results and fthms_wait returns FTHMS_ENOCONV;
 *              1 = fthms_wait then runs the whole job again in FP64 (precision 0) and returns its
 *              status (the FP64 results replace the mixed ones; fthms_stats reports the fallback).
 *  omega_rank, omega_ranks : frequency partition of one job over omega_ranks ranks (one GPU each; 0 or 1
 *              = no partition).  The per-frequency sub-problems of a step are independent (Section 3), so
 *              rank r assembles, factors and solves only the solved frequencies l in
 *              [1 + r (L-1)/R, 1 + (r+1)(L-1)/R) (R = omega_ranks), and holds only their device memory; the
 *              one coupling, the omega -> t synthesis of every step (eq. TDsol), is a sum over all
 *              frequencies, so the ranks add their partial time samples with the all-reduce given to
 *              fthms_set_allreduce before the windowed forward transforms (eq. Fourierk) of their own
 *              frequencies.  fthms_densities then covers the rank's frequencies only; the traces are
 *              summed across ranks the same way.
 *  shapes    : launch shapes and LU path, the five choices fthms_autotune returns and fthms_set_shapes
 *              takes (same candidates; all 0 = built-in defaults), applied from the job's first run: a job
 *              submitted with fthms_submit runs tuned without an autotuning pass.  Others -> EINVAL. */
typedef struct {
  double W;
  int L;
  int N_fixed, N_min, N_off;
  double N_ppw;
  int M, Q;
  double H;
  int n_period;
  int interior;
  int n_obs;
  const double* obs_xy;
  int n_tout;
  double tout0, dtout;
  int precision;
  int keep_densities;
  int cross_mode;
  double refine_tol;
  int refine_max;
  int refine_fallback;
  int omega_rank, omega_ranks;
  int shapes[5];
} fthms_options;

typedef struct {
  double gpu_ms;          /* device time of the last run of the job (CUDA events on the ctx stream) */
  double setup_ms;        /* host planning time of fthms_prepare */
  long long systems;      /* P (L-1): (arc, omega) systems assembled and factored */
  long long solves;       /* P (L-1) M Q: executions of Algorithm 1's BIE solve */
  long long kernel_launches; /* kernels launched by one run */
  size_t device_bytes;    /* device memory held by the job */
  double cross_entries;   /* stored cross-evaluation matrix entries */
  double hankel_evals;    /* kernel evaluations in assembly (self + cross) */
  size_t h2d_bytes;       /* host -> device bytes uploaded by fthms_prepare */
  double lu_flops;        /* (8/3) sum N^3: complex LU of every system */
  double solve_flops;     /* 8 sum N^2 Q M: triangular solves of one run */
  double apply_flops;     /* 8 Q M (cross + observation entries): cross matvecs of one run */
  int precision;          /* the job's precision option */
  double max_refine_resid; /* mixed forms: max over systems and steps of the relative error estimated to
                              remain after the last correction (its size x the estimated contraction) */
  double refine_passes;   /* mixed forms: mean refinement passes (residual + correction) per system and step */
  long long n_unconverged; /* mixed forms: (system, step) pairs whose estimate stayed above refine_tol */
  int fallback_runs;      /* runs of the job repeated in FP64 by refine_fallback = 1 */
  int lu_tensor_systems;  /* systems factored with tensor-core (tcgen05) trailing updates (mixed forms) */
} fthms_stats_t;

/* Create a context on CUDA device `device` that enqueues all work on `cuda_stream` (a
 * cudaStream_t; NULL = a non-blocking stream that the context creates, owns and destroys).
 * hbm_budget_bytes caps the device memory of all live jobs (0 = no cap).  Returns FTHMS_ECUDA if
 * the device cannot be used.  Job memory comes from the device's default stream-ordered memory
 * pool (cudaMallocAsync); the first use of a device in the process raises that pool's release
 * threshold, so memory freed by released jobs stays in the pool for later jobs of the process
 * (cudaMemPoolTrimTo on the default pool returns it to the driver). */
fthms_status fthms_create(fthms_ctx** out, int device, size_t hbm_budget_bytes, void* cuda_stream);
/* Destroy a context.  Jobs of the context that were not released are waited for and their device
 * memory is freed; their handles then accept fthms_release only (every other call returns
 * FTHMS_EINVAL). */
fthms_status fthms_destroy(fthms_ctx* ctx);

/* Plan a job (Section 3.1 geometry, Section 5 grids) on the host, allocate its device memory and
 * upload its tables; enqueues no compute.  Validation failures return FTHMS_EINVAL (overlapping
 * rules of Section 3.1 violated, window wider than one period 2 pi/h, n_period not a power of
 * two, ...); a job above the budget returns FTHMS_ENOMEM.  *out receives the job handle. */
fthms_status fthms_prepare(fthms_ctx* ctx, const fthms_curve* curves, int ncurves,
                           const fthms_arc* arcs, int narcs, const fthms_signal* signal,
                           const fthms_options* options, fthms_req** out);

/* Plan a job on the host only: the same validation as fthms_prepare (same status codes and
 * messages), without a device, allocation or upload.  *device_bytes receives the device memory the job
 * would hold (what fthms_prepare charges against a context budget) and *n_systems its number of
 * (arc, omega) systems (of this rank's frequencies for a partitioned job); either pointer may be NULL.
 * For capacity planning (no counterpart in the paper). */
fthms_status fthms_plan_info(const fthms_curve* curves, int ncurves, const fthms_arc* arcs, int narcs,
                             const fthms_signal* signal, const fthms_options* options,
                             size_t* device_bytes, int* n_systems);

/* Enqueue the whole hot path of a prepared job on the context stream (asynchronous): assembly,
 * factorisation, m = 1 data, M multiple-scattering steps, output traces.  May be called again
 * (recomputes everything from the uploaded tables). */
fthms_status fthms_run(fthms_req* req);

/* fthms_prepare followed by fthms_run. */
fthms_status fthms_submit(fthms_ctx* ctx, const fthms_curve* curves, int ncurves,
                          const fthms_arc* arcs, int narcs, const fthms_signal* signal,
                          const fthms_options* options, fthms_req** out);

/* *done = 1 when the last run finished (0 otherwise); never blocks. */
fthms_status fthms_poll(fthms_req* req, int* done);
/* Block until the last run finished or timeout_ms elapsed (negative = no limit):
 * FTHMS_ETIMEOUT on timeout, FTHMS_ECUDA if the device reported an error, FTHMS_ENOCONV if the run
 * finished but some system of a mixed-form job did not meet refine_tol within refine_max passes (its
 * results stay readable; with refine_fallback = 1 the job is first run again in FP64, see
 * fthms_options). */
fthms_status fthms_wait(fthms_req* req, int timeout_ms);

/* Output traces u_M(z_k, t_i) (eq. mult-scatt-int, evaluated directly at the output times),
 * row-major [n_obs][n_tout] doubles into out (cap >= n_obs*n_tout).  Waits for the job. */
fthms_status fthms_traces(fthms_req* req, double* out, size_t cap);

/* Densities phi_{j,m,q}(omega_l)[i] of arc j: m in 1..M (requires keep_densities) or m = 0 for
 * the sum over m; q in 0..Q-1.  Layout: for l = 1..L-1 (a frequency-partitioned job: the rank's own l,
 * in increasing order), N_j(omega_l) complex values at the
 * first-kind nodes t_i = cos((2i+1) pi/(2N)), i = 0..N-1, where phi(t) = Psi(x(t)) |x'(t)|
 * sqrt(1 - t^2) is the smooth factor of eq. singularity.  Needs 2 sum_l N_j(omega_l) doubles;
 * the size is written to *needed (may be NULL).  Waits for the job. */
fthms_status fthms_densities(fthms_req* req, int arc, int m, int q, double* out, size_t cap,
                             size_t* needed);

/* Same layout, written to a device buffer on the context stream (no host copy). */
fthms_status fthms_densities_dev(fthms_req* req, int arc, int m, int q, double* out_dev,
                                 size_t cap);

/* Node counts N_j(omega_l) for l = 1..L-1, row-major [narcs][L-1] ints (cap >= narcs*(L-1)). */
fthms_status fthms_node_counts(fthms_req* req, int* out, size_t cap);

fthms_status fthms_stats(fthms_req* req, fthms_stats_t* out);

/* Per-result error statement of the mixed forms: out[j*(L-1) + l-1] = the relative error estimated to
 * remain in the densities phi_{j,m,q}(omega_l) after refinement, maximised over the steps m and windows
 * q (the estimate of refine_tol's stopping rule; the smooth densities of Algorithm 1's BIE solve).  0 for
 * every system of an FP64 job (direct solve, no estimate) and of a job replaced by the FP64 fallback.
 * cap >= narcs*(L-1).  Waits for the job. */
fthms_status fthms_result_errors(fthms_req* req, double* out, size_t cap);

/* Pipeline stages, in enqueue order, for the per-stage timers below. */
enum {
  FTHMS_STAGE_TABLES = 0,      /* FFT twiddles, recentring phases, log and restriction tables */
  FTHMS_STAGE_ASSEMBLE = 1,    /* self matrices (eq. FDBIEk-interior, log-split rule) */
  FTHMS_STAGE_LU = 2,          /* LU factorisation of every (arc, omega) matrix (large systems: the panels) */
  FTHMS_STAGE_CROSS_ASM = 3,   /* stored cross-arc single-layer rows (eq. FDsolk-interior) */
  FTHMS_STAGE_INCIDENT = 4,    /* g_{k,1} and its slow transform (eqs. criterion_int1, Fourierk) */
  FTHMS_STAGE_RESTRICT = 5,    /* transfer mesh -> solve nodes */
  FTHMS_STAGE_SOLVE = 6,       /* triangular solves (Algorithm 1, BIE solve; mixed forms: every pass's) */
  FTHMS_STAGE_CROSS_APPLY = 7, /* cross-arc and observation potentials */
  FTHMS_STAGE_SYNTH_FWD = 8,   /* eq. TDsol, eq. criterion_int2, eq. Fourierk */
  FTHMS_STAGE_TRACES = 9,      /* eq. mult-scatt-int at the output times */
  FTHMS_STAGE_RESID = 10,      /* mixed forms: refinement residuals G - A phi of the first pass */
  FTHMS_STAGE_RESID_UPD = 11,  /* mixed forms: residuals of later passes (updated with the last correction) */
  FTHMS_STAGE_LU_UPDATE = 12,  /* mixed forms: tensor-core trailing updates of the large-system LU */
  FTHMS_STAGE_FUSED = 13,      /* FP64 form with fthms_use_fused: assembly + LU + step-1 solve in one launch */
  FTHMS_NSTAGES = 14
};

/* Pick launch shapes and the LU path for this job's hardware and sizes: runs the job once, then times
 * each tunable stage `reps` times per candidate -- warps (systems) per solve block {4, 2, 1}, threads per
 * cross-assembly block {128, 64, 256} (stored rows only), per time-transform block {256, 128, 512}, per
 * restriction block {128, 64, 256} and, in the mixed forms, the smallest N factored with tensor-core
 * updates {801, 512, 384, 256} (below it the one-CTA LU) -- and keeps the fastest for later fthms_run
 * calls (a captured graph is dropped and re-captured).  The launch shapes change no number; the LU path
 * changes the FP32 factor's rounding only, which the refinement removes.  shapes (NULL allowed) receives
 * the five choices (the last 0 for an FP64 job).  The job's earlier results are overwritten: call
 * fthms_run afterwards.  Not in the paper (a batching aid of this library). */
fthms_status fthms_autotune(fthms_req* req, int reps, int* shapes);

/* Apply five choices as fthms_autotune returns them (e.g. tuned once on a job of the same sizes) without
 * timing anything: shapes[0] warps per solve block {1, 2, 4}, [1] threads per cross-assembly block
 * {64, 128, 256}, [2] per time-transform block {128, 256, 512}, [3] per restriction block {64, 128, 256},
 * [4] the smallest N factored with tensor-core updates {256, 384, 512, 801} (mixed forms; must be 0 for an
 * FP64 job); 0 anywhere keeps the built-in default.  FTHMS_EINVAL for any other value (nothing changes
 * then).  A captured graph is dropped.  Later fthms_run calls use them. */
fthms_status fthms_set_shapes(fthms_req* req, const int* shapes);

/* Sum across the ranks of a frequency-partitioned job (options omega_ranks > 1): called on the host from
 * fthms_run, M times per run (after each step's partial synthesis, with buf_dev = the n_act x N_T time
 * samples of the active transfer nodes, and for the traces, n_obs x n_tout), it must replace buf_dev
 * (count doubles, device memory of the job) by its elementwise sum over all ranks, in order on
 * cuda_stream (e.g. an in-place NCCL all-reduce enqueued on that stream) or before it returns.  user is
 * passed through.  Every rank must call fthms_run the same number of times.  fthms_run returns
 * FTHMS_EINVAL for a partitioned job without an all-reduce; a partitioned job is never captured into a
 * CUDA graph (fthms_use_graph is ignored). */
typedef void (*fthms_allreduce_fn)(double* buf_dev, size_t count, void* cuda_stream, void* user);
fthms_status fthms_set_allreduce(fthms_req* req, fthms_allreduce_fn fn, void* user);

/* enable != 0 (FP64 form only; FTHMS_EINVAL for a mixed form): later runs assemble, factor and solve (step 1)
 * every (arc, omega) system in one persistent launch -- each CTA takes the next system (largest N first) from a
 * work counter and carries it through its self matrix (the same rule as the staged assembly, evaluated per
 * system), its LU and its step-1 solve -- instead of three launches over all systems; the incident field and
 * the restriction to the solve nodes run first.  Densities agree with the staged path to rounding (the
 * assembly's operation order differs).  Algorithm 1 lines 7-9 per (arc, omega); not a paper form (batching). */
fthms_status fthms_use_fused(fthms_req* req, int enable);

/* enable != 0: fthms_run captures the job's whole pipeline (all stages and steps) into a CUDA graph on
 * its first run and replays it afterwards as one launch; the graph is rebuilt never (the job's inputs
 * are fixed at prepare).  Runs with per-stage profiling enabled launch stage by stage. */
fthms_status fthms_use_graph(fthms_req* req, int enable);

/* enable != 0: later runs record CUDA events around every stage launch on the context stream
 * (small overhead); 0 stops recording.  Accumulated totals are kept until reset by enabling again. */
fthms_status fthms_profile(fthms_req* req, int enable);

/* Accumulated device milliseconds and kernel launches per stage over the profiled runs; both
 * arrays need FTHMS_NSTAGES entries.  Waits for the last run. */
fthms_status fthms_stage_times(fthms_req* req, double* ms, long long* launches);
fthms_status fthms_release(fthms_req* req);

/* Message of the last failed call on this thread (never NULL). */
const char* fthms_last_error(void);

/* ---- request server (continuous batching of jobs) --------------------------------------------
 * A server owns a context on `device` with an HBM budget and `max_inflight` slots, each with its own
 * CUDA stream.  Submitted jobs (same inputs as fthms_submit, copied at submit) wait in arrival order;
 * a worker thread admits the oldest one whenever a slot is free and the budget has room for its
 * device memory (fthms_prepare's estimate), so jobs that arrive while others run start as soon as
 * slots and memory free up and their kernels overlap on the device.  Finished jobs stay resident
 * (factors, densities, traces) until fthms_server_release; a job larger than the whole budget fails
 * with FTHMS_ENOMEM.  This is a serving form of the solver; the paper has no counterpart (it notes only that the
 * sub-problems are independent of one another, Section 3). */
typedef struct fthms_server fthms_server;

fthms_status fthms_server_create(fthms_server** out, int device, size_t hbm_budget_bytes, int max_inflight);
fthms_status fthms_server_submit(fthms_server* s, const fthms_curve* curves, int ncurves,
                                 const fthms_arc* arcs, int narcs, const fthms_signal* signal,
                                 const fthms_options* options, long long* ticket);
/* *state: 0 queued, 1 running, 2 done, 3 failed. */
fthms_status fthms_server_poll(fthms_server* s, long long ticket, int* state);
/* Block until done (FTHMS_OK), failed (the job's status) or timeout_ms (FTHMS_ETIMEOUT; <0 = none). */
fthms_status fthms_server_wait(fthms_server* s, long long ticket, int timeout_ms);
/* Borrow the finished job (valid until fthms_server_release) for fthms_traces / fthms_densities /
 * fthms_stats; do not release it directly. */
fthms_status fthms_server_result(fthms_server* s, long long ticket, fthms_req** req);
/* Host wall-clock milliseconds from submit to admission (queue) and to completion (total). */
fthms_status fthms_server_latency(fthms_server* s, long long ticket, double* queue_ms, double* total_ms);
fthms_status fthms_server_release(fthms_server* s, long long ticket);
fthms_status fthms_server_destroy(fthms_server* s);

/* ---- kernel-level entry points (device buffers, enqueued on `cuda_stream`) -------------------- */

/* Bessel functions of order 0 for z_dev[i] > 0 (the kernel of Section 2.1): J0, Y0 and the
 * regular part Yhat0 = Y0 - (2/pi)(ln(z/2) + gamma) J0.  Any output pointer may be NULL.
 * Returns FTHMS_EINVAL for n < 0. */
fthms_status fthms_bessel0(const double* z_dev, double* j0_dev, double* y0_dev,
                           double* yhat0_dev, int n, void* cuda_stream);

/* Nystrom matrix of V_Gamma on one arc (eq. FDBIEk-interior with the log-split Chebyshev rule):
 * A[i + l*N] (column-major, interleaved complex, 2*N*N doubles in A_dev) for N first-kind nodes
 * at wavenumber kappa > 0.  Allocates and frees its own temporary tables and returns after the matrix
 * is written (it synchronizes cuda_stream).  FTHMS_EINVAL for a NULL argument or coefficient array,
 * curve degree < 1, N outside [2, 1024], kappa <= 0 or theta_b <= theta_a. */
fthms_status fthms_assemble_self(const fthms_curve* curve, const fthms_arc* arc, int N,
                                 double kappa, double* A_dev, void* cuda_stream);

/* Allocation-free variant of fthms_assemble_self (the paper has no counterpart; this is a library
 * convenience).  It is for callers that must not allocate device memory: a host application whose
 * own allocator owns all device memory and forbids cudaMalloc/cudaFree from third-party code, a
 * process running under a fixed memory cap, or a latency-bound pipeline that cannot accept the
 * device-wide synchronisation that cudaFree implies.  It computes the same matrix (same kernels, same
 * layout: A[i + l*N], interleaved complex, 2*N*N doubles in A_dev) but keeps its temporary device
 * data in a fixed ~534 KB static device array of the library instead of allocating: every GPU that
 * loads the library holds that array until the process exits.  The caller still provides A_dev.
 *  - Arguments are checked as in fthms_assemble_self, except that N must lie in [2, 256] (the
 *    array's capacity); N outside that range returns FTHMS_EINVAL.
 *  - The first call on each device (with that device current) looks up the array's device address
 *    and uploads the Bessel coefficient tables; make that first call before any stream capture.
 *  - The call is asynchronous on cuda_stream: it returns with its copies and kernels queued.  A_dev
 *    holds the matrix, and the static array is free for the next caller, only once that stream's
 *    work has completed (synchronize the stream or order later work after it).
 *  - All calls share the one array and leave their data in it.  Calls whose work overlaps on the
 *    GPU (different streams or threads without ordering) race on it; calls on one stream are
 *    ordered.  Every call rewrites all of the array that it reads, so nothing needs clearing.
 *  - No cudaMalloc/cudaFree or other allocating routine is called; the per-call tables go up with
 *    cudaMemcpyAsync on cuda_stream. */
fthms_status fthms_assemble_self_noalloc(const fthms_curve* curve, const fthms_arc* arc, int N,
                                         double kappa, double* A_dev, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* FTHMS_H */
