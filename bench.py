"""Benchmark of the FTH-MS hot path on GB300: arc-omega BIE solves per second.

Headline workload (one step = one whole job, every hot-path stage): the mixed-precision configuration -- 6
arcs of a seeded exterior configuration of 5 ellipses (one closed ellipse in 2 overlapping arcs, four open
270-degree elliptic arcs), N = 512 nodes on every arc, 1023 solved frequencies on (0, 400], 8
multiple-scattering steps, 2 time windows, plane-wave pulse; cross rows stored in HBM -- in the fastest mixed
variant (default launch shapes, autotuned shapes and LU path, replayed as one CUDA graph, or the FP64-kept
form) whose densities agree with the FP64 form of the same job within 1e-10 in the same run.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload c4|c2|c3]

`value` is device-timed with the job's tables resident in HBM (CUDA events on the library's stream around K
back-to-back runs); `e2e` times the public C ABI call with host buffers (prepare + run + wait + traces +
densities to host + release) per step.  Under "forms": the same workload in FP64 and in each mixed variant,
N = 1024 on every arc (tensor-core LU, cross rows every step), the 4-obstacle configuration, the 12-arc star
cavity (one job), and a served request mix against the plain form on the same mix.  With --gpus N (torchrun)
every rank runs its own replica of the job (weak scaling, no collective on the data path) and rank 0 prints
the job-wide line; --partition splits one job's frequencies over the ranks instead (one all-reduce of the
time samples per step, NCCL; strong scaling).  `--impl reference` times the CPU oracle on a bounded sample
of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "arc-ω BIE solves/s at ≤1e-10 rel err, served+batched vs plain FP64; p50/p99 ms"
MIXED_BAR = 1e-10      # the metric's error bar: mixed densities against the FP64 form of the same job


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


PEAKS = _peaks()


def _hbm_peak_gbs():
    """Measured copy bandwidth of this GPU type (MEASURED_PEAKS.json), else the 6.8 TB/s fallback."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


HBM_PEAK_GBS = _hbm_peak_gbs()
FP64_PEAK_GFLOPS = 152 * 4 * 2.07  # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz max SM clock
# Algorithmic FP64 flops of one stored kernel entry: one far-field Hankel step at four asymptotic terms, the
# most common count at this workload (4 + 4 Horner FMAs, 1/z and 1/z^2, the amplitude, the two components,
# the phase rotation).
FLOPS_PER_KERNEL_ENTRY = 34


def kernels_hash():
    """sha256 of kernels.cu's code: comments, trailing blanks and empty lines removed, so that a change of
    wording leaves the recorded counters valid and any change of code invalidates them."""
    import hashlib
    import re
    with open(os.path.join(ROOT, "paper_2507_05725_gb300", "csrc", "kernels.cu")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    code = "\n".join(line.rstrip() for line in src.splitlines() if line.strip())
    return hashlib.sha256(code.encode()).hexdigest()[:16]


def measured_traffic_per_unit():
    """DRAM bytes per unit of work and kernel, from the committed ncu summary, if it was taken on the
    current kernels.cu (else {})."""
    try:
        txt = open(TRAFFIC_FILE).read()
    except OSError:
        return {}
    h = None
    out = {}
    for line in txt.splitlines():
        if line.startswith("kernels.cu code sha256:"):
            h = line.split("`")[1] if line.count("`") >= 2 else None
        cells = [c.strip().strip("`") for c in line.strip().strip("|").split("|")]
        if len(cells) >= 6 and cells[0].startswith("k_"):
            try:
                out[cells[0]] = float(cells[5])
            except ValueError:
                pass
    return out if h == kernels_hash() else {}


def max_over_ranks(ms, device="cuda"):
    """Largest per-rank time (replicas run concurrently; the job-wide step ends with the slowest)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world_size, solves_per_rank, ms):
    """Whole-job throughput: the solves of every rank's replica over the slowest rank's time."""
    return world_size * solves_per_rank / (ms / 1000.0)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    lrank = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, lrank


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# TF32 dense tensor rate: the measured bf16 rate x the nominal TF32 / BF16 ratio (1.1 / 2.25 PFLOP/s), sustained
# (the LU runs inside a long job).
TF32_PEAK_TFLOPS = PEAKS.get("bf16_tflops_sustained", 1700.0) * (1.1 / 2.25)
PEAK_NOTE = "of measured" if PEAKS else "of fallback"
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic_config4_small.md")


def workload(name, N=512):
    import workloads
    return {"c4": lambda: workloads.config4(N), "c2": workloads.config2, "c3": workloads.config3}[name]()


WORKLOAD_NAMES = {
    "c4": "5ellipses6arcs-N{N}: 6 arcs (1 closed ellipse in 2 + 4 open 270-degree arcs), N={N} on every arc, "
          "L=1024 on [0,400], M=8, Q=2 (one whole job per step)",
    "c2": "4obstacles-planewave: 8 arcs, N 48..259, L=1025 on [0,60], M=12, Q=1 (one whole job per step)",
    "c3": "star12-cavity: 12 arcs, N 32..760, L=2049 on [0,200], M=8, Q=4, cross rows every step (one job per step)",
}


def solves_of(problem):
    o = problem["options"]
    return len(problem["arcs"]) * (o["L"] - 1) * o["M"] * o["Q"]


def cpu_sample_problem(name="c4", n_freq=16):
    """Bounded sample of the headline workload for the CPU oracle: the same 6 arcs, N = 512, signal and
    8 steps x 2 windows on n_freq solved frequencies (spacing h = 0.75, so that the windows fit one period):
    about 14 s of CPU time at 16 frequencies (the cpu_baseline), 7 s at 8 (one step of the reference arm)."""
    import workloads
    if name == "c4":
        return workloads.config4(512, L=n_freq + 1, W=0.75 * n_freq, n_period=256)
    return workloads.config2(L=65, W=30.0, H=6.0, M=12, n_period=512, T=6.0)


def run_oracle_sample(name="c4", n_freq=16):
    from oracle import run_oracle
    p = cpu_sample_problem(name, n_freq)
    t0 = time.perf_counter()
    run_oracle(p, arcs_phi=[])
    return solves_of(p), time.perf_counter() - t0


def cpu_cores_used():
    try:
        from threadpoolctl import threadpool_info
        n = max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
        return int(n)
    except Exception:
        return os.cpu_count() or 1


def reference_arm(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        run_oracle_sample(args.workload, 8)
    times, solves = [], 0
    for _ in range(args.steps):
        s, dt = run_oracle_sample(args.workload, 8)
        solves, times = s, times + [dt]
    ms = 1000.0 * statistics.mean(times)
    value = solves / (ms / 1000.0)
    p = cpu_sample_problem(args.workload, 8)
    o = p["options"]
    sample = (f"oracle (numpy/scipy FP64) on {len(p['arcs'])} arcs x {o['L'] - 1} frequencies x {o['M']} steps x "
              f"{o['Q']} windows ({solves} solves) per step, same geometry, N, signal and steps as the bench workload")
    cores = cpu_cores_used()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{p['name']} sample on host cores", "sample": sample},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def rel_l2(a, b):
    """Relative L2 distance of two lists (per arc) of {l: densities}, against the first."""
    num = den = 0.0
    for x, y in zip(a, b):
        for l in x:
            num += float(np.sum(np.abs(x[l] - y[l]) ** 2))
            den += float(np.sum(np.abs(x[l]) ** 2))
    return math.sqrt(num / den) if den > 0 else 0.0


def _wait(F, job):
    try:
        job.wait()
        return "ok"
    except F.FthmsError as e:
        return str(e)


class _NoClock:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        pass

    def summary(self):
        return None


def time_job(F, ctx, stream, problem, precision, steps, warmup, autotune=False, graph=False, clocks=None,
             dens=False, allreduce=None, ws=1, fused=False):
    """Device time of `steps` back-to-back runs of one prepared job after `warmup` runs (CUDA events on the
    library's stream, synchronised on both sides, max over ranks), with its stage times (direct launches)."""
    import torch
    P = len(problem["arcs"])
    job = F.Job(ctx, problem, keep_densities=False, precision=precision)
    if allreduce is not None:
        job.set_allreduce(allreduce)
    tune = F.fthms_autotune(job.req, 2) if autotune else None
    if fused:
        F.fthms_use_fused(job.req)
    if graph:
        F.fthms_use_graph(job.req, True)
    for _ in range(warmup):
        job.run()
    status = _wait(F, job)
    if not graph:
        F.fthms_profile(job.req, True)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with (ClockSampler(clocks) if clocks is not None else _NoClock()) as clk:
        e0.record(stream)
        for _ in range(steps):
            job.run()
        e1.record(stream)
        torch.cuda.synchronize()
    s = _wait(F, job)
    status = s if s != "ok" else status
    ms = max_over_ranks(e0.elapsed_time(e1) / steps)
    stages = None if graph else {k: (v[0] / steps, v[1] / steps) for k, v in F.fthms_stage_times(job.req).items()}
    st = job.stats()
    d = [job.densities(j, 0, 0) for j in range(P)] if dens else None
    ok = bool(np.all(np.isfinite(job.traces())))
    job.release()
    return {"ms": ms, "stages": stages, "stats": st, "dens": d, "ok": ok, "status": status, "shapes": tune,
            "precision": precision, "autotune": autotune, "graph": graph, "clocks": clk.summary()}


def lu_update_flops(problem, n_tensor):
    """Algorithmic tensor flops of the tcgen05 trailing updates of one job: per system and 32-column panel,
    8 x 32 x T^2 real flops (T = trailing size), times 3 for the three-term TF32 split (N fixed per batch)."""
    N = int(problem["options"].get("N_fixed") or 0)
    per = sum(8.0 * 32 * (N - 32 * (k + 1)) ** 2 for k in range(N // 32 + 1) if N - 32 * (k + 1) > 0)
    return 3.0 * per * n_tensor


def stage_rooflines(r, problem, stored_rows):
    """Per stage with a model (stage CUDA-event timers over the timed region; each stage below is one kernel,
    or one kernel and a small companion named in its note): algorithmic bytes or flops per job over the
    stage's device time per job."""
    stages, st = r["stages"], r["stats"]
    o = problem["options"]
    M, Q = o["M"], o["Q"]
    prec = r["precision"]
    sum_n2 = st["solve_flops"] / (8.0 * Q * M)
    passes = st["refine_passes"]
    tpu = measured_traffic_per_unit()
    out = {}

    def add(stage, kernel, bound, amount, peak, unit, note, traffic=None, launches=None):
        ms, stage_launches = stages.get(stage, (0.0, 0))
        launches = stage_launches if launches is None else launches
        if ms <= 0 or amount <= 0:
            return
        ach = amount / (ms * 1e-3) / (1e12 if unit == "TFLOP/s" else 1e9)
        out[stage] = {"kernel": kernel, "bound": bound, "achieved": ach, "peak": peak, "unit": unit,
                      "frac": ach / peak, "traffic": traffic, "ms_per_job": ms, "launches_per_job": launches,
                      "ms_per_launch": ms / max(launches, 1),
                      ("algorithmic_flops_per_launch" if unit.endswith("FLOP/s") else "algorithmic_bytes_per_launch"):
                          amount / max(launches, 1),
                      "note": note}

    hbm = f"peak: measured copy bandwidth ({PEAK_NOTE})"
    fp64 = "peak: FP64 pipe derived from the unit counts and clock: 152 SMs x 4 flop/clk x 2.07 GHz"
    if stored_rows:
        name = "k_cross_rows_df" if prec >= 1 else "k_cross_apply"
        by = 16.0 * st["cross_entries"] * M
        tr = tpu[name] * st["cross_entries"] * M if name in tpu else None
        add("cross_apply", name, "hbm", by, HBM_PEAK_GBS, "GB/s",
            f"every stored cross entry (16 B) read once per step{', then an ordered per-group reduce (~1% of the stage)' if prec else ''}; {hbm}",
            traffic=tr, launches=M)
    if prec >= 1:
        solve_units = sum_n2 * M * (1.0 + passes)
        add("solve", "k_msolve", "hbm", 8.0 * solve_units, HBM_PEAK_GBS, "GB/s",
            f"the FP32 factor (8 B per entry) read once per solve pass, 1 + {passes:.3f} passes per system and step; {hbm}",
            traffic=tpu["k_msolve"] * solve_units if "k_msolve" in tpu else None)
        if prec == 2:
            add("resid", "k_mresid64", "hbm", 16.0 * sum_n2 * M, HBM_PEAK_GBS, "GB/s",
                f"first-pass residual to FP64 accuracy: the FP64 matrix (16 B per entry) read once per step; a "
                f"sixth of the rows on the FP64 pipe (8 DFMA per entry, two windows), the rest in anchored sums of "
                f"exact products on the FP32 pipe; {hbm}", traffic=tpu["k_mresid64"] * sum_n2 * M if "k_mresid64" in tpu else None)
            upd_units = sum_n2 * M * max(passes - 1.0, 0.0)
            add("resid_upd", "k_mresid_upd", "hbm", 16.0 * upd_units, HBM_PEAK_GBS,
                "GB/s", f"later-pass residual updates: the FP64 matrix (16 B per entry) read once per pass, "
                        f"{max(passes - 1.0, 0.0):.3f} passes per system and step; {hbm}",
                traffic=tpu["k_mresid_upd"] * upd_units if "k_mresid_upd" in tpu else None)
        else:
            add("resid", "k_mresid", "hbm", 16.0 * sum_n2 * M, HBM_PEAK_GBS, "GB/s",
                f"first-pass double-float residual: the kept matrix (16 B per entry) read once; {hbm}")
            add("resid_upd", "k_mresid", "hbm", 16.0 * sum_n2 * M * max(passes - 1.0, 0.0), HBM_PEAK_GBS, "GB/s",
                f"later-pass residuals: the kept matrix read once per pass; {hbm}")
        if st.get("lu_tensor_systems", 0) > 0:
            add("lu_update", "k_lu_big_update", "tensor", lu_update_flops(problem, st["lu_tensor_systems"]),
                TF32_PEAK_TFLOPS, "TFLOP/s",
                f"tcgen05 kind::tf32 trailing updates, 3 TF32 products per FP32 product (8 x 32 x T^2 real flops "
                f"per panel); peak: TF32 dense = measured bf16 sustained x 1.1/2.25 ({PEAK_NOTE})")
    else:
        add("solve", "k_solve", "alu", st["solve_flops"], FP64_PEAK_GFLOPS, "GFLOP/s", fp64)
        add("lu", "k_lu<double2>", "alu", st["lu_flops"], FP64_PEAK_GFLOPS, "GFLOP/s", "(8/3) sum N^3; " + fp64)
        if stored_rows:
            add("cross_assemble", "k_cross_assemble", "alu", FLOPS_PER_KERNEL_ENTRY * st["cross_entries"],
                FP64_PEAK_GFLOPS, "GFLOP/s", "34-flop model of one far-field Hankel step per entry; " + fp64)
    return out


def roofline_of(r, problem, stored_rows):
    """The dominant stage's roofline (largest device time per job among the stage timers)."""
    stages = r["stages"]
    dom = max(stages, key=lambda k: stages[k][0])
    rl = stage_rooflines(r, problem, stored_rows)
    if dom in rl:
        return dict(rl[dom], stage=dom)
    return {"stage": dom, "kernel": None, "bound": "alu", "achieved": None, "peak": FP64_PEAK_GFLOPS,
            "unit": "GFLOP/s", "frac": None, "traffic": None, "note": "no roofline model for this stage"}


# The fifth configuration's bands (omega_max to 300, up to 2049 frequencies) make single requests as large as
# the 12-arc cavity's jobs (about a minute each in FP64); the bench samples the lower part of its range.
SERVED_WMAX = (20.0, 150.0)
SERVED_LS = (257, 513, 1025)


def served_vs_plain(F, ctx, n=48, seed=11, max_inflight=4, precision=1, wmax=None, Ls=None):
    """Served stream on a bounded seeded sample of the fifth configuration (disk / star cavity / ellipse
    obstacles, 2-12 arcs, omega_max in [20, 150], 257 / 513 / 1025 frequencies, M 3-6), admitted by an HBM
    budget of 3/4 of the free device memory: a saturated pass (every request at t = 0) measures capacity;
    Poisson arrivals at 0.7 x that rate give per-request latency; the plain FP64 form runs the same requests
    back to back through fthms_submit for comparison."""
    import torch
    import workloads
    wmax, Ls = wmax or SERVED_WMAX, Ls or SERVED_LS
    problems = workloads.served_requests(seed, n, wmax=wmax, Ls=Ls, arcs=(2, 12))
    solves = sum(solves_of(p) for p in problems)
    budget = int(0.75 * torch.cuda.mem_get_info()[0])
    srv = F.Server(0, budget, max_inflight=max_inflight)
    for p in problems[:2]:
        t = srv.submit(p, precision=precision)
        srv.wait(t)
        srv.release(t)
    t0 = time.perf_counter()
    tickets = [srv.submit(p, precision=precision) for p in problems]
    for t in tickets:
        srv.wait(t)
    makespan = time.perf_counter() - t0
    for t in tickets:
        srv.release(t)
    rate = 0.7 * n / makespan
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n))
    t_start = time.perf_counter()
    tickets = []
    for p, a in zip(problems, arrivals):
        dt = t_start + a - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        tickets.append(srv.submit(p, precision=precision))
    for t in tickets:
        srv.wait(t)
    t_end = time.perf_counter()
    lat = []
    for t in tickets:
        lat.append(srv.latency(t)[1])
        srv.release(t)
    srv.close()
    # the same requests in the plain FP64 form, one after another through the public call
    for p in problems[:2]:
        req = F.fthms_submit(ctx, F.Marshalled(p, keep_densities=False, precision=0))
        F.fthms_wait(req)
        F.fthms_release(req)
    t0 = time.perf_counter()
    for p in problems:
        m = F.Marshalled(p, keep_densities=False, precision=0)
        req = F.fthms_submit(ctx, m)
        F.fthms_wait(req)
        F.fthms_traces(req, m.options.n_obs, p["options"]["n_tout"])
        F.fthms_release(req)
    plain_s = time.perf_counter() - t0
    lat = np.array(lat)
    return {"value": float(solves / (t_end - t_start)), "unit": "solves/s",
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "saturated_solves_per_s": float(solves / makespan),
            "plain_fp64_same_mix_solves_per_s": float(solves / plain_s),
            "vs_plain_same_mix": float(plain_s / makespan), "arrival_rate_per_s": rate, "requests": n,
            "max_inflight": max_inflight, "precision": precision, "hbm_budget_gb": budget / 1e9,
            "sample": f"{n} seeded requests (disk / star cavity / 1-5 ellipses, 2-12 arcs, omega_max in "
                      f"[{wmax[0]:g}, {wmax[1]:g}], {' / '.join(map(str, Ls))} frequencies, "
                      f"M 3-6), Poisson arrivals at 0.7 x saturated capacity; vs_plain_same_mix = the same "
                      f"requests in FP64 back to back through fthms_submit"}


def ours(args):
    import torch

    from paper_2507_05725_gb300 import fthms as F

    ws, rank, lrank = _dist()
    torch.cuda.set_device(lrank)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.Stream()
    problem = workload(args.workload, args.N)
    o = problem["options"]
    P, M, Q = len(problem["arcs"]), o["M"], o["Q"]
    solves = solves_of(problem)
    stored_rows = o.get("cross_mode", 0) == 0
    ctx = F.fthms_create(lrank, 0, stream.cuda_stream)
    wname = WORKLOAD_NAMES[args.workload].format(N=args.N)

    if args.partition and ws > 1:
        # one job split over the ranks by frequency (strong scaling): one all-reduce of the time samples per step
        import copy
        part = copy.deepcopy(problem)
        part["options"].update(omega_rank=rank, omega_ranks=ws)
        r = time_job(F, ctx, stream, part, args.precision, args.steps, args.warmup, clocks=lrank,
                     allreduce=F.TorchAllreduce(torch.device("cuda", lrank)), ws=ws)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": solves / (r["ms"] / 1e3), "unit": "solves/s", "n_gpus": ws,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms"],
                              "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
                              "dtype": "mixed" if args.precision else "f64", "data": "synthetic",
                              "config": {"workload": wname, "parallelism": f"omega-partition x{ws}"},
                              "clocks": r["clocks"], "status": r["status"]}))
        torch.distributed.destroy_process_group()
        return 0

    # FP64 form of the same job: the densities every mixed variant is checked against, and the plain number
    plain = time_job(F, ctx, stream, problem, 0, 1 if args.workload == "c4" else min(args.steps, 3), 1, dens=True,
                     ws=ws) if not args.no_plain else None
    variants = []
    if not args.plain_only:
        for prec, tune, graph in ((1, False, False), (1, True, False), (1, True, True), (2, True, False)):
            v = time_job(F, ctx, stream, problem, prec, 3, 2, autotune=tune, graph=graph, dens=plain is not None, ws=ws)
            v["err"] = rel_l2(plain["dens"], v["dens"]) if plain is not None else None
            variants.append(v)
    eligible = [v for v in variants if v["status"] == "ok" and v["ok"] and v["err"] is not None and v["err"] <= MIXED_BAR]
    best = min(eligible, key=lambda v: v["ms"]) if eligible else None
    # the headline run: the chosen form over the requested steps, clocks sampled
    if best is not None:
        head = time_job(F, ctx, stream, problem, best["precision"], args.steps, args.warmup, autotune=best["autotune"],
                        graph=best["graph"], clocks=lrank, dens=plain is not None, ws=ws)
        head["err"] = rel_l2(plain["dens"], head["dens"]) if plain is not None else None
        if best["graph"]:                        # stage timers need direct launches: the same form, 2 runs
            d = time_job(F, ctx, stream, problem, best["precision"], 2, 1, autotune=best["autotune"], ws=ws)
            head["stages"], head["stages_from"] = d["stages"], "the same form launched stage by stage (2 runs)"
    else:
        head = time_job(F, ctx, stream, problem, 0, args.steps, args.warmup, clocks=lrank, ws=ws)
        head["err"] = 0.0
    value = job_value(ws, solves, head["ms"])

    # end to end through the C ABI with host buffers, the headline form's tuned shapes given in the options
    e2e_problem = dict(problem, options=dict(problem["options"]))
    if head.get("shapes"):
        e2e_problem["options"]["shapes"] = [int(v) for v in head["shapes"]]
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    d2h = h2d = 0
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        m = F.Marshalled(e2e_problem, keep_densities=False, precision=head["precision"])
        req = F.fthms_submit(ctx, m)
        try:
            F.fthms_wait(req)
        except F.FthmsError:
            pass
        tr = F.fthms_traces(req, m.options.n_obs, o["n_tout"])
        d2h = tr.nbytes
        for j in range(P):
            d2h += F.fthms_densities(req, j, 0, 0).nbytes
        h2d = F.fthms_stats(req)["h2d_bytes"]
        F.fthms_release(req)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(1000.0 * (time.perf_counter() - t0) / e2e_steps)

    roof = roofline_of(head, problem, stored_rows) if head.get("stages") else None
    stage_roofs = stage_rooflines(head, problem, stored_rows) if head.get("stages") else None

    def summary(r, with_stages=True):
        if r is None:
            return None
        st = r["stats"]
        out = {"value": job_value(ws, solves, r["ms"]), "ms_per_step": r["ms"], "precision": r["precision"],
               "autotuned": r["autotune"], "graph": r["graph"], "status": r["status"],
               "rel_l2_vs_fp64_densities": r.get("err"), "max_refine_resid": st["max_refine_resid"],
               "refine_passes": st["refine_passes"], "n_unconverged": st["n_unconverged"],
               "lu_tensor_systems": st.get("lu_tensor_systems"), "shapes": r["shapes"],
               "gpu_launches_per_step": st["kernel_launches"], "device_gb": st["device_bytes"] / 1e9}
        if with_stages and r["stages"]:
            out["stages_ms_per_step"] = {k: v[0] for k, v in r["stages"].items()}
        return out

    forms = {"plain_fp64": summary(plain)}
    for v in variants:
        key = "mixed" if v["precision"] == 1 else "fp64_kept"
        key += ("_autotuned" if v["autotune"] else "") + ("_graph" if v["graph"] else "")
        forms[key] = summary(v)
    if rank == 0 and ws == 1 and not args.no_forms:
        import workloads
        if args.workload == "c4":
            big = time_job(F, ctx, stream, workloads.config4(1024), 1, 1, 1, autotune=True)
            forms["c4_N1024"] = dict(summary(big), workload=WORKLOAD_NAMES["c4"].format(N=1024) +
                                     "; cross rows every step", solves_per_step=solves_of(workloads.config4(1024)))
            c2 = workloads.config2()
            p2 = time_job(F, ctx, stream, c2, 0, 3, 2)
            m2 = time_job(F, ctx, stream, c2, 1, 3, 2, autotune=True, graph=True)
            forms["c2_plain_fp64"] = dict(summary(p2), value=solves_of(c2) / (p2["ms"] / 1e3),
                                          workload=WORKLOAD_NAMES["c2"])
            f2 = time_job(F, ctx, stream, c2, 0, 3, 2, fused=True)
            forms["c2_plain_fp64_fused"] = dict(
                summary(f2), value=solves_of(c2) / (f2["ms"] / 1e3), workload=WORKLOAD_NAMES["c2"],
                note="batching form: assembly, LU and step-1 solve of every system in one persistent launch "
                     "(fthms_use_fused), against c2_plain_fp64's staged launches of the same FP64 kernels",
                fused_ms_per_job=f2["stages"].get("fused", (0.0, 0))[0] if f2["stages"] else None,
                staged_ms_per_job=sum(p2["stages"][k][0] for k in ("assemble_self", "lu")) + p2["stages"]["solve"][0]
                / c2["options"]["M"] if p2["stages"] else None)
            forms["c2_mixed_autotuned_graph"] = dict(summary(m2), value=solves_of(c2) / (m2["ms"] / 1e3),
                                                     workload=WORKLOAD_NAMES["c2"])
        if not args.no_c3 and args.workload != "c3":
            c3 = workloads.config3()
            r3 = time_job(F, ctx, stream, c3, 1, 1, 1)
            forms["c3_mixed"] = dict(summary(r3), value=solves_of(c3) / (r3["ms"] / 1e3), workload=WORKLOAD_NAMES["c3"])
        if not args.no_served:
            forms["served"] = served_vs_plain(F, ctx)
    F.fthms_destroy(ctx)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        s, dt = run_oracle_sample(args.workload)
        p = cpu_sample_problem(args.workload)
        cpu = {"value": s / dt, "unit": "solves/s", "cores": cpu_cores_used(), "kind": "oracle",
               "sample": f"{s} solves: {p['name']} on {p['options']['L'] - 1} frequencies, {p['options']['M']} steps, "
                         f"{p['options']['Q']} windows ({dt:.1f} s of CPU time)"}
    if rank == 0:
        mixed = head["precision"] >= 1
        line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": head["ms"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None,
                "dtype": ({1: "f32 factors (tensor-core 3xTF32 updates above N = 800) + double-float (2 x f32) "
                              "assembly, refinement, FFT butterflies, restriction and cross apply; f64 set-up, "
                              "folds and outputs",
                           2: "f32 factors + f64 self matrices and refinement residuals, f64 small-argument Hankel "
                              "series and FFT butterflies; double-float far-field recurrence, restriction and cross "
                              "apply"}[head["precision"]] if mixed else "f64"),
                "data": "synthetic",
                "config": {"workload": wname, "solves_per_step": solves, "systems_per_step": P * (o["L"] - 1),
                           "form": (("mixed" if head["precision"] == 1 else "fp64-kept mixed") +
                                    (", autotuned" if head["autotune"] else "") +
                                    (", CUDA-graph replay" if head["graph"] else "") +
                                    f" (densities {head['err']:.2e} from the FP64 form in-run, bar 1e-10)")
                           if mixed else "plain FP64",
                           "l2": "working set > L2 (stored cross rows "
                                 f"{head['stats']['cross_entries'] * 16 / 1e9:.0f} GB, matrices and factors)",
                           "parallelism": f"replicas x{ws}"},
                "e2e": {"value": job_value(ws, solves, e2e_ms), "unit": "solves/s", "ms_per_step": e2e_ms,
                        "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                        "note": "fthms_submit + wait + traces and summed densities to host + release, the headline "
                                "form's shapes passed in fthms_options.shapes"},
                "gpu_launches": int(head["stats"]["kernel_launches"] * args.steps),
                "roofline": roof,
                "stage_rooflines": stage_roofs,
                "stages_ms_per_step": {k: v[0] for k, v in head["stages"].items()} if head.get("stages") else None,
                "clocks": head["clocks"],
                "cpu_baseline": cpu,
                "traces_finite": head["ok"],
                "forms": forms}
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c4", choices=["c4", "c2", "c3"],
                    help="c4: the mixed-precision configuration (N per --N); c2: 4 obstacles; c3: 12-arc star cavity")
    ap.add_argument("--N", type=int, default=512, help="nodes per arc of the c4 workload (512 or 1024 on one GPU)")
    ap.add_argument("--partition", action="store_true", help="split one job's frequencies over the ranks")
    ap.add_argument("--precision", type=int, default=1, help="precision of the partitioned job")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the secondary workloads")
    ap.add_argument("--no-c3", action="store_true", help="skip the 12-arc cavity form")
    ap.add_argument("--no-plain", action="store_true", help="skip the FP64 reference job (no in-run error check)")
    ap.add_argument("--plain-only", action="store_true", help="time the plain FP64 form only (profiling runs)")
    ap.add_argument("--served-only", action="store_true",
                    help="only the served stream against the plain FP64 form on the same requests, one JSON line")
    ap.add_argument("--served-n", type=int, default=48, help="requests of --served-only")
    ap.add_argument("--served-wmax", type=float, default=SERVED_WMAX[1],
                    help="largest omega_max of --served-only (the fifth configuration's range ends at 300)")
    ap.add_argument("--served-ls", default=",".join(map(str, SERVED_LS)),
                    help="frequency counts of --served-only (the fifth configuration's: 257,513,1025,2049)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    if args.served_only:
        return served_only(args)
    return ours(args)


def served_only(args):
    """The served stream on a chosen sample of the fifth configuration's ranges (bounded by the time a GPU run
    may take: its plain FP64 pass runs the requests one after another)."""
    import torch
    from paper_2507_05725_gb300 import fthms as F
    torch.cuda.set_device(0)
    ctx = F.fthms_create(0, 0, None)
    r = served_vs_plain(F, ctx, n=args.served_n, wmax=(SERVED_WMAX[0], args.served_wmax),
                        Ls=tuple(int(v) for v in args.served_ls.split(",")))
    F.fthms_destroy(ctx)
    print(json.dumps({"metric": METRIC, "served": r}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
