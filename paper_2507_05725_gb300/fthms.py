"""Thin Python binding of the FTH-MS C ABI (include/fthms.h).

Argument marshalling only: every step of the hot path runs in the CUDA library libfthms.so.  The
functions carry the C names; ``Job`` is a small convenience wrapper over the same calls.  Importing
this module loads the library and raises if it has not been built (there is no fallback).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libfthms.so")

FTHMS_OK, FTHMS_EINVAL, FTHMS_ENOMEM, FTHMS_ENOCONV, FTHMS_ETIMEOUT, FTHMS_ECUDA, FTHMS_EBUSY, FTHMS_ENOTIMPL = range(8)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ENOCONV", "ETIMEOUT", "ECUDA", "EBUSY", "ENOTIMPL"]


class FthmsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


class fthms_curve(C.Structure):
    _fields_ = [("degree", C.c_int), ("ax", C.POINTER(C.c_double)), ("bx", C.POINTER(C.c_double)),
                ("ay", C.POINTER(C.c_double)), ("by", C.POINTER(C.c_double))]


class fthms_arc(C.Structure):
    _fields_ = [("curve", C.c_int), ("theta_a", C.c_double), ("theta_b", C.c_double)]


class fthms_signal(C.Structure):
    _fields_ = [("kind", C.c_int), ("z0", C.c_double * 2), ("dir", C.c_double * 2), ("sign", C.c_double),
                ("amp", C.c_double), ("carrier", C.c_double), ("centre", C.c_double), ("width", C.c_double),
                ("n_t", C.c_int), ("t0", C.c_double), ("dt", C.c_double), ("f", C.POINTER(C.c_double)),
                ("band", C.c_double)]


class fthms_options(C.Structure):
    _fields_ = [("W", C.c_double), ("L", C.c_int), ("N_fixed", C.c_int), ("N_min", C.c_int), ("N_off", C.c_int),
                ("N_ppw", C.c_double), ("M", C.c_int), ("Q", C.c_int), ("H", C.c_double), ("n_period", C.c_int),
                ("interior", C.c_int), ("n_obs", C.c_int), ("obs_xy", C.POINTER(C.c_double)),
                ("n_tout", C.c_int), ("tout0", C.c_double), ("dtout", C.c_double), ("precision", C.c_int),
                ("keep_densities", C.c_int), ("cross_mode", C.c_int), ("refine_tol", C.c_double),
                ("refine_max", C.c_int), ("refine_fallback", C.c_int), ("omega_rank", C.c_int),
                ("omega_ranks", C.c_int), ("shapes", C.c_int * 5)]


class fthms_stats_t(C.Structure):
    _fields_ = [("gpu_ms", C.c_double), ("setup_ms", C.c_double), ("systems", C.c_longlong),
                ("solves", C.c_longlong), ("kernel_launches", C.c_longlong), ("device_bytes", C.c_size_t),
                ("cross_entries", C.c_double), ("hankel_evals", C.c_double), ("h2d_bytes", C.c_size_t),
                ("lu_flops", C.c_double), ("solve_flops", C.c_double), ("apply_flops", C.c_double),
                ("precision", C.c_int), ("max_refine_resid", C.c_double),
                ("refine_passes", C.c_double), ("n_unconverged", C.c_longlong), ("fallback_runs", C.c_int),
                ("lu_tensor_systems", C.c_int)]


# void (*)(double* buf_dev, size_t count, void* cuda_stream, void* user)
ALLREDUCE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)

STAGES = ["tables", "assemble_self", "lu", "cross_assemble", "incident", "restrict", "solve", "cross_apply",
          "synth_fwd", "traces", "resid", "resid_upd", "lu_update", "fused"]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libfthms.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    vp, st = C.c_void_p, C.c_int
    pp = C.POINTER(C.c_void_p)
    sigs = {
        "fthms_create": (st, [pp, C.c_int, C.c_size_t, vp]),
        "fthms_destroy": (st, [vp]),
        "fthms_prepare": (st, [vp, C.POINTER(fthms_curve), C.c_int, C.POINTER(fthms_arc), C.c_int,
                               C.POINTER(fthms_signal), C.POINTER(fthms_options), pp]),
        "fthms_run": (st, [vp]),
        "fthms_submit": (st, [vp, C.POINTER(fthms_curve), C.c_int, C.POINTER(fthms_arc), C.c_int,
                              C.POINTER(fthms_signal), C.POINTER(fthms_options), pp]),
        "fthms_poll": (st, [vp, C.POINTER(C.c_int)]),
        "fthms_wait": (st, [vp, C.c_int]),
        "fthms_traces": (st, [vp, C.POINTER(C.c_double), C.c_size_t]),
        "fthms_densities": (st, [vp, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double), C.c_size_t,
                                 C.POINTER(C.c_size_t)]),
        "fthms_densities_dev": (st, [vp, C.c_int, C.c_int, C.c_int, vp, C.c_size_t]),
        "fthms_node_counts": (st, [vp, C.POINTER(C.c_int), C.c_size_t]),
        "fthms_stats": (st, [vp, C.POINTER(fthms_stats_t)]),
        "fthms_result_errors": (st, [vp, C.POINTER(C.c_double), C.c_size_t]),
        "fthms_set_allreduce": (st, [vp, ALLREDUCE_FN, vp]),
        "fthms_release": (st, [vp]),
        "fthms_last_error": (C.c_char_p, []),
        "fthms_bessel0": (st, [vp, vp, vp, vp, C.c_int, vp]),
        "fthms_assemble_self": (st, [C.POINTER(fthms_curve), C.POINTER(fthms_arc), C.c_int, C.c_double, vp, vp]),
        "fthms_assemble_self_noalloc": (st, [C.POINTER(fthms_curve), C.POINTER(fthms_arc), C.c_int, C.c_double,
                                             vp, vp]),
        "fthms_server_create": (st, [pp, C.c_int, C.c_size_t, C.c_int]),
        "fthms_server_submit": (st, [vp, C.POINTER(fthms_curve), C.c_int, C.POINTER(fthms_arc), C.c_int,
                                     C.POINTER(fthms_signal), C.POINTER(fthms_options), C.POINTER(C.c_longlong)]),
        "fthms_server_poll": (st, [vp, C.c_longlong, C.POINTER(C.c_int)]),
        "fthms_server_wait": (st, [vp, C.c_longlong, C.c_int]),
        "fthms_server_result": (st, [vp, C.c_longlong, pp]),
        "fthms_server_latency": (st, [vp, C.c_longlong, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "fthms_server_release": (st, [vp, C.c_longlong]),
        "fthms_server_destroy": (st, [vp]),
        "fthms_use_graph": (st, [vp, C.c_int]),
        "fthms_autotune": (st, [vp, C.c_int, C.POINTER(C.c_int)]),
        "fthms_set_shapes": (st, [vp, C.POINTER(C.c_int)]),
        "fthms_use_fused": (st, [vp, C.c_int]),
        "fthms_profile": (st, [vp, C.c_int]),
        "fthms_stage_times": (st, [vp, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


LIB = _load()

EXPORTED = ["fthms_create", "fthms_destroy", "fthms_prepare", "fthms_run", "fthms_submit", "fthms_poll",
            "fthms_wait", "fthms_traces", "fthms_densities", "fthms_densities_dev", "fthms_node_counts",
            "fthms_stats", "fthms_release", "fthms_last_error", "fthms_bessel0", "fthms_assemble_self",
            "fthms_profile", "fthms_stage_times", "fthms_assemble_self_noalloc", "fthms_server_create",
            "fthms_server_submit", "fthms_server_poll", "fthms_server_wait", "fthms_server_result",
            "fthms_server_latency", "fthms_server_release", "fthms_server_destroy", "fthms_use_graph",
            "fthms_autotune", "fthms_plan_info", "fthms_result_errors", "fthms_set_allreduce", "fthms_set_shapes",
            "fthms_use_fused"]


def _check(status):
    if status != FTHMS_OK:
        raise FthmsError(status, LIB.fthms_last_error().decode())


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class Marshalled:
    """ctypes views of a problem dict (see workloads); keeps the numpy buffers alive."""

    def __init__(self, problem, keep_densities=True, precision=0):
        self._keep = []
        curves = problem["curves"]
        self.curves = (fthms_curve * len(curves))()
        for i, c in enumerate(curves):
            arrs = [np.ascontiguousarray(np.asarray(c[k], dtype=np.float64)) for k in ("ax", "bx", "ay", "by")]
            self._keep += arrs
            self.curves[i] = fthms_curve(len(arrs[0]) - 1, *[_dptr(a) for a in arrs])
        arcs = problem["arcs"]
        self.arcs = (fthms_arc * len(arcs))(*[fthms_arc(int(c), float(a), float(b)) for c, a, b in arcs])
        s = problem["signal"]
        smp = s.get("samples")
        if smp is not None:
            fs = np.ascontiguousarray(np.asarray(smp["f"], dtype=np.float64))
            self._keep.append(fs)
            sampled = (fs.size, float(smp["t0"]), float(smp["dt"]), _dptr(fs), float(smp["band"]))
        else:
            sampled = (0, 0.0, 0.0, None, 0.0)
        self.signal = fthms_signal(int(s["kind"]), (C.c_double * 2)(*s["z0"]), (C.c_double * 2)(*s["dir"]),
                                   s["sign"], s["amp"], s["carrier"], s["centre"], s["width"], *sampled)
        o = problem["options"]
        obs = np.ascontiguousarray(np.asarray(o["obs"], dtype=np.float64).reshape(-1))
        self._keep.append(obs)
        self.options = fthms_options(o["W"], o["L"], o["N_fixed"], o["N_min"], o["N_off"], o["N_ppw"], o["M"],
                                     o["Q"], o["H"], o["n_period"], o["interior"], obs.size // 2,
                                     _dptr(obs) if obs.size else None, o["n_tout"], o["tout0"], o["dtout"],
                                     int(precision), int(keep_densities), int(o.get("cross_mode", 0)),
                                     float(o.get("refine_tol", 0.0)), int(o.get("refine_max", 0)),
                                     int(o.get("refine_fallback", 0)), int(o.get("omega_rank", 0)),
                                     int(o.get("omega_ranks", 0)),
                                     (C.c_int * 5)(*[int(v) for v in o.get("shapes", (0, 0, 0, 0, 0))]))
        self.ncurves, self.narcs = len(curves), len(arcs)


def fthms_create(device=0, hbm_budget_bytes=0, cuda_stream=None):
    ctx = C.c_void_p()
    _check(LIB.fthms_create(C.byref(ctx), int(device), int(hbm_budget_bytes), cuda_stream))
    return ctx


def fthms_destroy(ctx):
    _check(LIB.fthms_destroy(ctx))


def fthms_prepare(ctx, m: Marshalled):
    req = C.c_void_p()
    _check(LIB.fthms_prepare(ctx, m.curves, m.ncurves, m.arcs, m.narcs, C.byref(m.signal), C.byref(m.options),
                             C.byref(req)))
    return req


def fthms_plan_info(m: Marshalled):
    """(device bytes, number of systems) of a job, planned on the host only (no GPU needed)."""
    nbytes, nsys = C.c_size_t(), C.c_int()
    _check(LIB.fthms_plan_info(m.curves, m.ncurves, m.arcs, m.narcs, C.byref(m.signal), C.byref(m.options),
                               C.byref(nbytes), C.byref(nsys)))
    return nbytes.value, nsys.value


def fthms_run(req):
    _check(LIB.fthms_run(req))


def fthms_submit(ctx, m: Marshalled):
    req = C.c_void_p()
    _check(LIB.fthms_submit(ctx, m.curves, m.ncurves, m.arcs, m.narcs, C.byref(m.signal), C.byref(m.options),
                            C.byref(req)))
    return req


def fthms_poll(req):
    d = C.c_int()
    _check(LIB.fthms_poll(req, C.byref(d)))
    return bool(d.value)


def fthms_wait(req, timeout_ms=-1):
    _check(LIB.fthms_wait(req, int(timeout_ms)))


def fthms_traces(req, n_obs, n_tout, out=None):
    if out is None:
        out = np.empty((n_obs, n_tout), dtype=np.float64)
    _check(LIB.fthms_traces(req, _dptr(out), out.size))
    return out


def fthms_densities(req, arc, m, q, out=None):
    need = C.c_size_t()
    LIB.fthms_densities(req, int(arc), int(m), int(q), None, 0, C.byref(need))
    if out is None:
        out = np.empty(need.value, dtype=np.float64)
    _check(LIB.fthms_densities(req, int(arc), int(m), int(q), _dptr(out), out.size, C.byref(need)))
    return out


def fthms_densities_dev(req, arc, m, q, out_ptr, cap):
    _check(LIB.fthms_densities_dev(req, int(arc), int(m), int(q), C.c_void_p(out_ptr), int(cap)))


def fthms_node_counts(req, narcs, L):
    out = np.empty((narcs, L - 1), dtype=np.int32)
    _check(LIB.fthms_node_counts(req, out.ctypes.data_as(C.POINTER(C.c_int)), out.size))
    return out


def fthms_stats(req):
    s = fthms_stats_t()
    _check(LIB.fthms_stats(req, C.byref(s)))
    return {k: getattr(s, k) for k, _ in fthms_stats_t._fields_}


def fthms_result_errors(req, narcs, L):
    """[narcs, L-1] estimated relative error left in each (arc, omega) result (mixed forms; 0 in FP64)."""
    out = np.empty((narcs, L - 1), dtype=np.float64)
    _check(LIB.fthms_result_errors(req, _dptr(out), out.size))
    return out


def fthms_set_allreduce(req, fn):
    """Install fn(buf_dev, count, cuda_stream) as the cross-rank sum of a frequency-partitioned job; returns
    the ctypes callback object, which the caller must keep alive while the job runs."""
    cb = ALLREDUCE_FN(lambda buf, n, stream, user: fn(buf, n, stream))
    _check(LIB.fthms_set_allreduce(req, cb, None))
    return cb


_CUDART = None


def _cudart():
    """The CUDA runtime (for the device <-> host copies of the all-reduce helpers below)."""
    global _CUDART
    if _CUDART is None:
        home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
        for name in (os.path.join(home, "lib64", "libcudart.so"), "libcudart.so", "libcudart.so.13"):
            try:
                _CUDART = C.CDLL(name)
                break
            except OSError:
                continue
        if _CUDART is None:
            raise OSError("libcudart not found")
        _CUDART.cudaMemcpyAsync.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int, C.c_void_p]
        _CUDART.cudaStreamSynchronize.argtypes = [C.c_void_p]
    return _CUDART


def _copy(dst, src, nbytes, kind, stream):
    rt = _cudart()
    if rt.cudaMemcpyAsync(dst, src, nbytes, kind, stream) != 0 or rt.cudaStreamSynchronize(stream) != 0:
        raise RuntimeError("cudaMemcpyAsync failed")


class HostAllreduce:
    """All-reduce through host memory: the partial samples go to a host array, `reduce(array)` sums it
    across ranks in place (e.g. torch.distributed.all_reduce on a CPU tensor with gloo), and the sum goes
    back to the device."""

    def __init__(self, reduce):
        self.reduce = reduce

    def __call__(self, buf, count, stream):
        h = np.empty(count, dtype=np.float64)
        _copy(h.ctypes.data, buf, count * 8, 2, stream)        # device -> host
        self.reduce(h)
        _copy(buf, h.ctypes.data, count * 8, 1, stream)        # host -> device


class TorchAllreduce:
    """All-reduce with torch.distributed on the device (NCCL): the partial samples are copied into a torch
    tensor on the job's stream, summed across ranks there, and copied back."""

    def __init__(self, device):
        self.device = device
        self.buf = None

    def __call__(self, buf, count, stream):
        import torch
        import torch.distributed as dist
        if self.buf is None or self.buf.numel() < count:
            self.buf = torch.empty(count, dtype=torch.float64, device=self.device)
        rt = _cudart()
        t = self.buf[:count]
        if rt.cudaMemcpyAsync(t.data_ptr(), buf, count * 8, 3, stream) != 0:
            raise RuntimeError("cudaMemcpyAsync failed")
        with torch.cuda.stream(torch.cuda.ExternalStream(stream, device=self.device)):
            dist.all_reduce(t)
        if rt.cudaMemcpyAsync(buf, t.data_ptr(), count * 8, 3, stream) != 0:
            raise RuntimeError("cudaMemcpyAsync failed")


def fthms_autotune(req, reps=3):
    """Choices for the job: solve warps, assembly threads, time threads, restriction threads and (mixed
    forms) the smallest N factored with tensor-core updates (0 for FP64)."""
    out = (C.c_int * 5)()
    _check(LIB.fthms_autotune(req, int(reps), out))
    return list(out)


def fthms_set_shapes(req, shapes):
    """Apply five choices as fthms_autotune returns them, without timing."""
    arr = (C.c_int * 5)(*[int(v) for v in shapes])
    _check(LIB.fthms_set_shapes(req, arr))


def fthms_use_fused(req, enable=True):
    _check(LIB.fthms_use_fused(req, int(bool(enable))))


def fthms_use_graph(req, enable=True):
    _check(LIB.fthms_use_graph(req, int(bool(enable))))


def fthms_profile(req, enable=True):
    _check(LIB.fthms_profile(req, int(bool(enable))))


def fthms_stage_times(req):
    ms = (C.c_double * len(STAGES))()
    n = (C.c_longlong * len(STAGES))()
    _check(LIB.fthms_stage_times(req, ms, n))
    return {s: (ms[i], n[i]) for i, s in enumerate(STAGES)}


def fthms_release(req):
    _check(LIB.fthms_release(req))


def fthms_last_error():
    return LIB.fthms_last_error().decode()


def fthms_bessel0(z_ptr, j0_ptr, y0_ptr, yh_ptr, n, stream=None):
    _check(LIB.fthms_bessel0(z_ptr, j0_ptr, y0_ptr, yh_ptr, int(n), stream))


def fthms_assemble_self(curve: dict, arc, N, kappa, A_ptr, stream=None):
    arrs = [np.ascontiguousarray(np.asarray(curve[k], dtype=np.float64)) for k in ("ax", "bx", "ay", "by")]
    c = fthms_curve(len(arrs[0]) - 1, *[_dptr(a) for a in arrs])
    a = fthms_arc(0, float(arc[0]), float(arc[1]))
    _check(LIB.fthms_assemble_self(C.byref(c), C.byref(a), int(N), float(kappa), C.c_void_p(A_ptr), stream))


def fthms_assemble_self_noalloc(curve: dict, arc, N, kappa, A_ptr, stream=None):
    """Same matrix as fthms_assemble_self, without device allocation (static scratch, N <= 256)."""
    arrs = [np.ascontiguousarray(np.asarray(curve[k], dtype=np.float64)) for k in ("ax", "bx", "ay", "by")]
    c = fthms_curve(len(arrs[0]) - 1, *[_dptr(a) for a in arrs])
    a = fthms_arc(0, float(arc[0]), float(arc[1]))
    _check(LIB.fthms_assemble_self_noalloc(C.byref(c), C.byref(a), int(N), float(kappa), C.c_void_p(A_ptr),
                                           stream))


class Job:
    """One FTH-MS job through the C ABI: ``Job(ctx, problem).run().wait()``."""

    def __init__(self, ctx, problem, keep_densities=True, precision=0):
        self.problem = problem
        self.m = Marshalled(problem, keep_densities=keep_densities, precision=precision)
        self.req = fthms_prepare(ctx, self.m)
        o = problem["options"]
        self.P, self.L, self.M, self.Q = len(problem["arcs"]), o["L"], o["M"], o["Q"]
        self.n_obs, self.n_tout = self.m.options.n_obs, o["n_tout"]

    def run(self):
        fthms_run(self.req)
        return self

    def wait(self, timeout_ms=-1):
        fthms_wait(self.req, timeout_ms)
        return self

    def node_counts(self):
        return fthms_node_counts(self.req, self.P, self.L)

    def traces(self):
        return fthms_traces(self.req, self.n_obs, self.n_tout)

    def densities(self, arc, m, q=0):
        """{l: complex array (N_arc(omega_l),)} for l = 1..L-1 (the rank's own l for a partitioned job)."""
        flat = fthms_densities(self.req, arc, m, q)
        z = flat[0::2] + 1j * flat[1::2]
        Ns = self.node_counts()[arc]
        out, o = {}, 0
        for l in self.own_frequencies():
            n = int(Ns[l - 1])
            out[l] = z[o:o + n]
            o += n
        return out

    def stats(self):
        return fthms_stats(self.req)

    def result_errors(self):
        return fthms_result_errors(self.req, self.P, self.L)

    def set_allreduce(self, fn):
        self._allreduce = fthms_set_allreduce(self.req, fn)
        return self

    def own_frequencies(self):
        """The solved frequency indices l of this job's rank (all of 1..L-1 without a partition)."""
        o = self.problem["options"]
        R, r, n = max(1, int(o.get("omega_ranks", 0))), int(o.get("omega_rank", 0)), self.L - 1
        return range(1 + r * n // R, 1 + (r + 1) * n // R)

    def release(self):
        if self.req is not None:
            fthms_release(self.req)
            self.req = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


def fthms_server_create(device=0, hbm_budget_bytes=0, max_inflight=4):
    s = C.c_void_p()
    _check(LIB.fthms_server_create(C.byref(s), int(device), int(hbm_budget_bytes), int(max_inflight)))
    return s


def fthms_server_submit(server, m: Marshalled):
    t = C.c_longlong()
    _check(LIB.fthms_server_submit(server, m.curves, m.ncurves, m.arcs, m.narcs, C.byref(m.signal),
                                   C.byref(m.options), C.byref(t)))
    return t.value


def fthms_server_poll(server, ticket):
    st = C.c_int()
    _check(LIB.fthms_server_poll(server, C.c_longlong(ticket), C.byref(st)))
    return st.value


def fthms_server_wait(server, ticket, timeout_ms=-1):
    _check(LIB.fthms_server_wait(server, C.c_longlong(ticket), int(timeout_ms)))


def fthms_server_result(server, ticket):
    r = C.c_void_p()
    _check(LIB.fthms_server_result(server, C.c_longlong(ticket), C.byref(r)))
    return r


def fthms_server_latency(server, ticket):
    q, t = C.c_double(), C.c_double()
    _check(LIB.fthms_server_latency(server, C.c_longlong(ticket), C.byref(q), C.byref(t)))
    return q.value, t.value


def fthms_server_release(server, ticket):
    _check(LIB.fthms_server_release(server, C.c_longlong(ticket)))


def fthms_server_destroy(server):
    _check(LIB.fthms_server_destroy(server))


class Server:
    """Request server over the C ABI: submit problem dicts, wait, read results by ticket."""

    def __init__(self, device=0, hbm_budget_bytes=0, max_inflight=4):
        self.s = fthms_server_create(device, hbm_budget_bytes, max_inflight)
        self.meta = {}

    def submit(self, problem, precision=0, keep_densities=False):
        m = Marshalled(problem, keep_densities=keep_densities, precision=precision)
        t = fthms_server_submit(self.s, m)
        o = problem["options"]
        self.meta[t] = (len(problem["arcs"]), o["L"], m.options.n_obs, o["n_tout"])
        return t

    def wait(self, ticket, timeout_ms=-1):
        fthms_server_wait(self.s, ticket, timeout_ms)

    def traces(self, ticket):
        P, L, n_obs, n_tout = self.meta[ticket]
        return fthms_traces(fthms_server_result(self.s, ticket), n_obs, n_tout)

    def densities(self, ticket, arc, m=0, q=0):
        P, L, _, _ = self.meta[ticket]
        req = fthms_server_result(self.s, ticket)
        flat = fthms_densities(req, arc, m, q)
        return flat[0::2] + 1j * flat[1::2]

    def stats(self, ticket):
        return fthms_stats(fthms_server_result(self.s, ticket))

    def latency(self, ticket):
        return fthms_server_latency(self.s, ticket)

    def release(self, ticket):
        fthms_server_release(self.s, ticket)
        self.meta.pop(ticket, None)

    def close(self):
        if self.s is not None:
            fthms_server_destroy(self.s)
            self.s = None
