"""Served form: continuous admission of jobs onto per-slot streams under an HBM budget.  Each result is
the same alone and in the mix (the jobs share no device data; the tolerance is the plain form's)."""
import math

import numpy as np
import pytest
import torch

import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-11


@pytest.fixture(scope="module")
def F():
    from paper_2507_05725_gb300 import fthms
    torch.cuda.set_device(0)
    return fthms


def _alone(F, problems, precision=0):
    ctx = F.fthms_create(0, 0, None)
    res = []
    for p in problems:
        job = F.Job(ctx, p, keep_densities=False, precision=precision).run().wait()
        dens = [job.densities(j, 0, 0) for j in range(len(p["arcs"]))]
        res.append((job.traces(), [np.concatenate([d[l] for l in sorted(d)]) for d in dens], job.stats()))
        job.release()
    F.fthms_destroy(ctx)
    return res


def _close(a, b):
    return np.linalg.norm(a - b) <= TOL * max(1e-300, np.linalg.norm(b))


@pytest.mark.parametrize("precision", [0, 1])
def test_served_results_same_alone_and_in_mix(F, precision):
    problems = wl.served_requests(7, 6)
    ref = _alone(F, problems, precision)
    srv = F.Server(0, 0, max_inflight=4)
    tickets = [srv.submit(p, precision=precision) for p in problems]     # arrive together: overlap
    for t in tickets:
        srv.wait(t)
    for (tr, dens, st), t, p in zip(ref, tickets, problems):
        assert _close(srv.traces(t), tr)
        for j in range(len(p["arcs"])):
            assert _close(srv.densities(t, j), dens[j])
        q_ms, tot_ms = srv.latency(t)
        assert 0.0 <= q_ms <= tot_ms
        srv.release(t)
    srv.close()


def test_budget_admission_and_oversized_job(F):
    problems = wl.served_requests(3, 4)
    ctx = F.fthms_create(0, 0, None)
    sizes = []
    for p in problems:
        job = F.Job(ctx, p, keep_densities=False)
        sizes.append(job.stats()["device_bytes"])
        job.release()
    F.fthms_destroy(ctx)
    budget = int(1.5 * max(sizes))        # about one job resident at a time
    srv = F.Server(0, budget, max_inflight=4)
    tickets = [srv.submit(p) for p in problems]
    for t in tickets:
        srv.wait(t)
        srv.release(t)                    # frees the budget for the next admission
    big = wl.config2(L=513, W=60.0, H=20.0, n_period=2048, M=2)
    tb = srv.submit(big)                  # larger than the whole budget: fails, does not hang
    with pytest.raises(F.FthmsError) as e:
        srv.wait(tb, 60000)
    assert e.value.status == F.FTHMS_ENOMEM
    srv.release(tb)
    srv.close()
