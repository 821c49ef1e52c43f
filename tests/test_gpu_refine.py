"""Refinement control of the mixed forms through the C ABI: the FP64-kept form (precision 2), the per-result
error statement, refinement that does not converge (FTHMS_ENOCONV) and the FP64 fallback, and sampled
signals (the boundary time signal given as data) against the oracle."""
import copy
import math

import numpy as np
import pytest
import torch

import workloads as wl
from oracle import run_oracle

pytestmark = pytest.mark.gpu

DENSITY_TOL = 1e-11
MIXED_TOL = 1e-10


@pytest.fixture(scope="module")
def F():
    from paper_2507_05725_gb300 import fthms
    return fthms


@pytest.fixture(scope="module")
def ctx(F):
    torch.cuda.set_device(0)
    c = F.fthms_create(0, 0, None)
    yield c
    F.fthms_destroy(c)


def _rel_vs_oracle(job, ref, problem):
    o = problem["options"]
    P, L, M, Q = len(problem["arcs"]), o["L"], o["M"], o["Q"]
    num = den = 0.0
    for m in range(1, M + 1):
        for j in range(P):
            for q in range(Q):
                d = job.densities(j, m, q)
                for l in range(1, L):
                    r = ref.phi[(m, j, l)][q]
                    num += float(np.sum(np.abs(d[l] - r) ** 2))
                    den += float(np.sum(np.abs(r) ** 2))
    return math.sqrt(num / den)


@pytest.mark.parametrize("name", ["point", "two-curves-Q2", "config2-reduced"])
def test_fp64_kept_form_parity(F, ctx, name):
    """precision 2 (FP64 small-argument Hankel series, residuals and FFT butterflies) meets the mixed bar,
    and every per-result error estimate is below refine_tol."""
    problem = {"point": lambda: wl.random_small(2, n_arcs_per_curve=3, kind=0, M=3),
               "two-curves-Q2": lambda: wl.random_small(5, n_curves=2, n_arcs_per_curve=2, Q=2, L=65, M=2),
               "config2-reduced": lambda: wl.config2_reduced(M=2)}[name]()
    job = F.Job(ctx, problem, precision=2).run().wait()
    ref = run_oracle(problem)
    assert _rel_vs_oracle(job, ref, problem) < MIXED_TOL
    tr = job.traces()
    assert np.max(np.abs(tr - ref.traces)) < MIXED_TOL * max(1e-300, np.max(np.abs(ref.traces)))
    st = job.stats()
    err = job.result_errors()
    job.release()
    assert st["precision"] == 2 and st["n_unconverged"] == 0
    assert err.shape == (len(problem["arcs"]), problem["options"]["L"] - 1)
    assert np.all(err >= 0.0) and np.all(err < 1e-12) and np.max(err) == pytest.approx(st["max_refine_resid"],
                                                                                         rel=1e-6)


def test_per_result_errors_are_zero_in_fp64(F, ctx):
    job = F.Job(ctx, wl.random_small(0, n_arcs_per_curve=3, kind=1), precision=0).run().wait()
    err = job.result_errors()
    job.release()
    assert np.all(err == 0.0)


def test_refinement_that_cannot_converge_reports_enoconv(F, ctx):
    """A tolerance no refinement can meet (1e-30 in one pass): fthms_wait returns FTHMS_ENOCONV, every
    (system, step) is counted, the results stay readable and carry their error estimates."""
    problem = wl.random_small(7, n_arcs_per_curve=4, M=2)
    problem["options"].update(refine_tol=1e-30, refine_max=1)
    job = F.Job(ctx, problem, precision=1).run()
    with pytest.raises(F.FthmsError) as e:
        job.wait()
    assert e.value.status == F.FTHMS_ENOCONV and "refine_tol" in str(e.value)
    st = job.stats()
    nsys = len(problem["arcs"]) * (problem["options"]["L"] - 1)
    assert st["n_unconverged"] == nsys * problem["options"]["M"] and st["fallback_runs"] == 0
    ref = run_oracle(problem)
    assert _rel_vs_oracle(job, ref, problem) < MIXED_TOL          # one pass already gets close
    err = job.result_errors()
    assert np.all(err > 0.0)
    job.release()


def test_fp64_fallback_replaces_unconverged_results(F, ctx):
    """refine_fallback = 1: the job that did not converge runs again in FP64; its results are bitwise those of
    an FP64 job and fthms_stats reports the fallback."""
    problem = wl.random_small(5, n_curves=2, n_arcs_per_curve=2, Q=2, L=65, M=2)
    plain = F.Job(ctx, problem, precision=0).run().wait()
    bad = copy.deepcopy(problem)
    bad["options"].update(refine_tol=1e-30, refine_max=1, refine_fallback=1)
    job = F.Job(ctx, bad, precision=1).run().wait()               # no error: the fallback met the bar
    st = job.stats()
    assert st["fallback_runs"] == 1
    assert np.array_equal(job.traces(), plain.traces())
    for j in range(len(problem["arcs"])):
        for q in range(2):
            a, b = plain.densities(j, 2, q), job.densities(j, 2, q)
            for l in a:
                assert np.array_equal(a[l], b[l])
    assert np.all(job.result_errors() == 0.0)
    plain.release()
    job.release()


def test_tighter_refinement_tolerance_is_met(F, ctx):
    """refine_tol = 1e-14 with up to 6 passes: more passes per system, every estimate below the target and
    the densities closer to the FP64 oracle than the default form's bar."""
    problem = wl.random_small(2, n_arcs_per_curve=3, kind=0, M=3)
    problem["options"].update(refine_tol=1e-14, refine_max=6)
    job = F.Job(ctx, problem, precision=1).run().wait()
    st = job.stats()
    assert st["n_unconverged"] == 0 and st["max_refine_resid"] < 1e-14 and st["refine_passes"] > 1.0
    rel = _rel_vs_oracle(job, run_oracle(problem), problem)
    job.release()
    assert rel < DENSITY_TOL


def test_fp64_kept_residual_updates_meet_a_tighter_tolerance(F, ctx):
    """FP64-kept form with refine_tol = 1e-14 and up to 6 passes: the first residual in FP64, every later
    one (at least the second pass's) updated with the last correction (r <- r - A d on the FP32 pipe); the
    updated residual must stay accurate, so the densities land on the FP64 oracle well inside the mixed
    form's bar."""
    problem = wl.random_small(2, n_arcs_per_curve=3, kind=0, M=3)
    problem["options"].update(refine_tol=1e-14, refine_max=6)
    job = F.Job(ctx, problem, precision=2).run().wait()
    st = job.stats()
    assert st["n_unconverged"] == 0 and st["max_refine_resid"] < 1e-14 and st["refine_passes"] >= 2.0
    rel = _rel_vs_oracle(job, run_oracle(problem), problem)
    job.release()
    assert rel < DENSITY_TOL


# ---- sampled signals ---------------------------------------------------------------------------------

def _sampled_problem(kind):
    p = wl.random_small(3 if kind == 1 else 2, n_arcs_per_curve=3, kind=kind, L=33, W=12.0, Q=2, H=8.0,
                        n_period=256, M=2)
    return wl.with_samples(p, wl.multipulse_samples(t0=0.0, dt=0.02, t_end=22.0))


@pytest.mark.parametrize("kind", [1, 0])
@pytest.mark.parametrize("precision", [0, 1])
def test_sampled_multipulse_signal_parity(F, ctx, kind, precision):
    """The multi-pulse signal of eq. multi given as samples (plane wave and point source) through the C ABI:
    densities and traces against the oracle reading the same samples."""
    problem = _sampled_problem(kind)
    job = F.Job(ctx, problem, precision=precision).run().wait()
    ref = run_oracle(problem)
    rel = _rel_vs_oracle(job, ref, problem)
    tr = job.traces()
    job.release()
    tol = DENSITY_TOL if precision == 0 else MIXED_TOL
    assert rel < tol
    assert np.max(np.abs(tr - ref.traces)) < 10 * tol * max(1e-300, np.max(np.abs(ref.traces)))
