"""Frequency-partitioned jobs on the GPU through the C ABI: two ranks of one job, emulated on this one GPU by
two host threads (each rank on its own stream; the all-reduce of the partial time samples goes through host
memory with a thread barrier, so no kernel ever waits for another), give the densities and traces of the
unpartitioned job."""
import copy
import math
import threading

import numpy as np
import pytest
import torch

import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_2507_05725_gb300 import fthms
    return fthms


def _two_rank_run(F, problem, precision):
    barrier = threading.Barrier(2)
    parts = [None, None]
    calls = [0, 0]

    def reducer(rank):
        def red(h):
            parts[rank] = h.copy()
            calls[rank] += 1
            barrier.wait()
            h[:] = parts[0] + parts[1]
            barrier.wait()
        return red

    ctxs = [F.fthms_create(0, 0, None) for _ in range(2)]
    jobs = []
    for rank in range(2):
        q = copy.deepcopy(problem)
        q["options"].update(omega_rank=rank, omega_ranks=2)
        jobs.append(F.Job(ctxs[rank], q, precision=precision).set_allreduce(F.HostAllreduce(reducer(rank))))
    errors = []

    def run(job):
        try:
            job.run().wait()
        except Exception as e:          # surfaced below
            errors.append(e)
            barrier.abort()

    th = [threading.Thread(target=run, args=(j,)) for j in jobs]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors, errors
    return ctxs, jobs, calls


@pytest.mark.parametrize("precision", [0, 1])
def test_two_rank_frequency_partition_matches_one_job(F, precision):
    torch.cuda.set_device(0)
    problem = wl.random_small(5, n_curves=2, n_arcs_per_curve=2, Q=2, L=65, M=3)
    ctx = F.fthms_create(0, 0, None)
    whole = F.Job(ctx, problem, precision=precision).run().wait()
    ctxs, jobs, calls = _two_rank_run(F, problem, precision)
    try:
        assert calls == [problem["options"]["M"]] * 2          # M - 1 steps + the traces
        tw = whole.traces()
        for job in jobs:
            assert np.max(np.abs(job.traces() - tw)) < 1e-12 * np.max(np.abs(tw))
        seen = set()
        num = den = 0.0
        for job in jobs:
            st = job.stats()
            assert st["systems"] == len(problem["arcs"]) * len(job.own_frequencies())
            for j in range(len(problem["arcs"])):
                for m in range(1, problem["options"]["M"] + 1):
                    for q in range(2):
                        d, w = job.densities(j, m, q), whole.densities(j, m, q)
                        for l, v in d.items():
                            seen.add(l)
                            num += float(np.sum(np.abs(v - w[l]) ** 2))
                            den += float(np.sum(np.abs(w[l]) ** 2))
        assert seen == set(range(1, problem["options"]["L"]))
        assert math.sqrt(num / den) < 1e-12
    finally:
        whole.release()
        for job in jobs:
            job.release()
        for c in ctxs + [ctx]:
            F.fthms_destroy(c)


def test_partitioned_job_needs_an_allreduce(F):
    torch.cuda.set_device(0)
    ctx = F.fthms_create(0, 0, None)
    q = wl.random_small(1)
    q["options"].update(omega_rank=1, omega_ranks=2)
    job = F.Job(ctx, q)
    with pytest.raises(F.FthmsError) as e:
        job.run()
    assert e.value.status == F.FTHMS_EINVAL and "allreduce" in str(e.value)
    job.release()
    F.fthms_destroy(ctx)
