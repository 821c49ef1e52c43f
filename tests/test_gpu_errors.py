"""Error behaviour of the C ABI (status codes and messages, no device faults)."""
import copy
import math

import pytest
import torch

import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_2507_05725_gb300 import fthms
    torch.cuda.set_device(0)
    return fthms


def _status(F, fn):
    with pytest.raises(F.FthmsError) as e:
        fn()
    return e.value.status, str(e.value)


def test_budget_rejects_job_with_enomem(F):
    ctx = F.fthms_create(0, 1 << 10, None)          # 1 KiB budget
    st, msg = _status(F, lambda: F.fthms_prepare(ctx, F.Marshalled(wl.random_small(0))))
    assert st == F.FTHMS_ENOMEM and "budget" in msg
    F.fthms_destroy(ctx)


def test_invalid_geometry_and_options(F):
    ctx = F.fthms_create(0, 0, None)
    p = wl.random_small(0)
    bad = copy.deepcopy(p)                          # arcs that do not overlap their neighbours
    bad["arcs"] = [(0, 2 * math.pi * k / 3, 2 * math.pi * k / 3 + 1.0) for k in range(3)]
    assert _status(F, lambda: F.fthms_prepare(ctx, F.Marshalled(bad)))[0] == F.FTHMS_EINVAL
    bad = copy.deepcopy(p)                          # window wider than the frequency grid's period
    bad["options"]["H"] = 1e3
    st, msg = _status(F, lambda: F.fthms_prepare(ctx, F.Marshalled(bad)))
    assert st == F.FTHMS_EINVAL and "period" in msg
    bad = copy.deepcopy(p)
    bad["options"]["n_period"] = 1000               # not a power of two
    assert _status(F, lambda: F.fthms_prepare(ctx, F.Marshalled(bad)))[0] == F.FTHMS_EINVAL
    bad = copy.deepcopy(p)                          # a period and time grid too long for the time kernels
    bad["options"]["n_period"] = 16384
    bad["options"]["Q"] = 4
    st, msg = _status(F, lambda: F.fthms_prepare(ctx, F.Marshalled(bad)))
    assert st == F.FTHMS_EINVAL and "shared memory" in msg
    bad = copy.deepcopy(p)                          # unknown cross mode
    bad["options"]["cross_mode"] = 2
    assert _status(F, lambda: F.fthms_prepare(ctx, F.Marshalled(bad)))[0] == F.FTHMS_EINVAL
    st, _ = _status(F, lambda: F.fthms_prepare(ctx, F.Marshalled(p, precision=3)))
    assert st == F.FTHMS_ENOTIMPL
    F.fthms_destroy(ctx)


def test_wait_poll_and_results_after_completion(F):
    ctx = F.fthms_create(0, 0, None)
    job = F.Job(ctx, wl.random_small(1)).run()
    try:
        F.fthms_wait(job.req, 0)                    # either finished already or ETIMEOUT
    except F.FthmsError as e:
        assert e.status == F.FTHMS_ETIMEOUT
    job.wait()
    assert F.fthms_poll(job.req)
    st = job.stats()
    assert st["solves"] == st["systems"] * job.M * job.Q and st["kernel_launches"] > 0
    with pytest.raises(F.FthmsError) as e:           # arc out of range
        F.fthms_densities(job.req, 99, 0, 0)
    assert e.value.status == F.FTHMS_EINVAL
    job.release()
    F.fthms_destroy(ctx)


def test_destroying_a_context_detaches_its_live_jobs(F):
    """A job that outlives its context: destroy waits for it and frees its device memory; the
    handle then accepts release only."""
    ctx = F.fthms_create(0, 0, None)
    m = F.Marshalled(wl.random_small(3))
    req = F.fthms_prepare(ctx, m)
    F.fthms_run(req)
    F.fthms_destroy(ctx)
    st, msg = _status(F, lambda: F.fthms_run(req))
    assert st == F.FTHMS_EINVAL and "context was destroyed" in msg
    st, _ = _status(F, lambda: F.fthms_wait(req, 0))
    assert st == F.FTHMS_EINVAL
    F.fthms_release(req)
