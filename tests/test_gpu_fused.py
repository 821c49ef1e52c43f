"""The batching form's persistent fused kernel (fthms_use_fused, FP64 form): every (arc, omega) system
assembled, factored and solved for step 1 in one launch, each CTA taking the next system (largest N first)
from a work counter.  Its densities and traces against the staged FP64 path and the FP64 oracle, uneven node
counts (N growing with omega), several windows, graph replay; refused for the mixed forms."""
import math

import numpy as np
import pytest
import torch

import workloads as wl
from oracle import run_oracle

pytestmark = pytest.mark.gpu

DENSITY_TOL = 1e-11


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


def _all_densities(job, problem):
    o = problem["options"]
    out = {}
    for m in range(1, o["M"] + 1):
        for j in range(len(problem["arcs"])):
            for q in range(o["Q"]):
                for l, v in job.densities(j, m, q).items():
                    out[(m, j, q, l)] = v
    return out


def _rel(a, b):
    num = sum(float(np.sum(np.abs(a[k] - b[k]) ** 2)) for k in a)
    den = sum(float(np.sum(np.abs(b[k]) ** 2)) for k in a)
    return math.sqrt(num / den)


CASES = {
    "point-uneven": lambda: wl.random_small(2, n_arcs_per_curve=3, kind=0, L=65, W=20.0, M=3),
    "two-curves-Q2": lambda: wl.random_small(5, n_curves=2, n_arcs_per_curve=2, Q=2, L=65, M=2),
    "Q4": lambda: wl.random_small(4, Q=4, L=129, H=5.0, M=2),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_fused_matches_staged_and_oracle(F, ctx, name):
    problem = CASES[name]()
    staged = F.Job(ctx, problem, precision=0).run().wait()
    fused = F.Job(ctx, problem, precision=0)
    F.fthms_use_fused(fused.req)
    fused.run().wait()
    st = fused.stats()
    a, b = _all_densities(fused, problem), _all_densities(staged, problem)
    ref = run_oracle(problem)
    o = problem["options"]
    oracle = {(m, j, q, l): ref.phi[(m, j, l)][q] for (m, j, q, l) in a}
    tr_f, tr_s = fused.traces(), staged.traces()
    fused.release()
    staged.release()
    assert _rel(a, b) < 1e-12, _rel(a, b)
    assert _rel(a, oracle) < DENSITY_TOL, _rel(a, oracle)
    assert np.max(np.abs(tr_f - tr_s)) < 1e-12 * max(1e-300, np.max(np.abs(tr_s)))
    assert st["systems"] == len(problem["arcs"]) * (o["L"] - 1)


def test_fused_with_graph_replay_and_profile(F, ctx):
    """Graph replay reproduces the direct fused run bitwise; the stage timers count one fused launch per run."""
    problem = CASES["point-uneven"]()
    job = F.Job(ctx, problem, precision=0)
    F.fthms_use_fused(job.req)
    F.fthms_profile(job.req, True)
    job.run().wait()
    times = F.fthms_stage_times(job.req)
    direct = _all_densities(job, problem)
    F.fthms_profile(job.req, False)
    F.fthms_use_graph(job.req, True)
    job.run().wait()
    job.run().wait()
    replay = _all_densities(job, problem)
    job.release()
    assert times["fused"][1] == 1 and times["assemble_self"][1] == 0 and times["lu"][1] == 0
    for k in direct:
        assert np.array_equal(direct[k], replay[k])


def test_fused_is_refused_in_the_mixed_forms(F, ctx):
    job = F.Job(ctx, CASES["point-uneven"](), precision=1)
    with pytest.raises(F.FthmsError) as e:
        F.fthms_use_fused(job.req)
    assert e.value.status == F.FTHMS_EINVAL
    F.fthms_use_fused(job.req, False)
    job.release()
