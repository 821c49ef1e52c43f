"""Host-only planning through the C ABI (fthms_plan_info): the validation of fthms_prepare and the job's
device-memory accounting, without a GPU."""
import copy
import math

import numpy as np

import pytest

import workloads as wl


@pytest.fixture(scope="module")
def F():
    from paper_2507_05725_gb300 import fthms
    return fthms


def _status(F, problem, **kw):
    with pytest.raises(F.FthmsError) as e:
        F.fthms_plan_info(F.Marshalled(problem, **kw))
    return e.value.status, str(e.value)


def test_config_sizes_and_determinism(F):
    """Config 2 has 8 arcs x 1024 solved frequencies; the same input plans to the same footprint."""
    m = F.Marshalled(wl.config2(), keep_densities=False, precision=1)
    b1, n1 = F.fthms_plan_info(m)
    b2, n2 = F.fthms_plan_info(m)
    assert n1 == n2 == 8 * 1024
    assert b1 == b2 and 5e9 < b1 < 2e10


def test_memory_accounting_follows_the_options(F):
    """Mixed precision adds the FP32 factors; every-step cross rows drop the stored cross matrices;
    keeping every step's densities adds M copies of them."""
    p = wl.config2_reduced()
    base, nsys = F.fthms_plan_info(F.Marshalled(p, keep_densities=False, precision=0))
    mixed, _ = F.fthms_plan_info(F.Marshalled(p, keep_densities=False, precision=1))
    kept, _ = F.fthms_plan_info(F.Marshalled(p, keep_densities=True, precision=0))
    q = copy.deepcopy(p)
    q["options"]["cross_mode"] = 1
    otf, _ = F.fthms_plan_info(F.Marshalled(q, keep_densities=False, precision=0))
    assert nsys == len(p["arcs"]) * (p["options"]["L"] - 1)
    assert mixed > base and kept > base and otf < base


def test_validation_without_a_gpu(F):
    p = wl.random_small(0)
    bad = copy.deepcopy(p)                          # arcs that do not overlap their neighbours
    bad["arcs"] = [(0, 2 * math.pi * k / 3, 2 * math.pi * k / 3 + 1.0) for k in range(3)]
    assert _status(F, bad)[0] == F.FTHMS_EINVAL
    bad = copy.deepcopy(p)                          # window wider than the frequency grid's period
    bad["options"]["H"] = 1e3
    st, msg = _status(F, bad)
    assert st == F.FTHMS_EINVAL and "period" in msg
    bad = copy.deepcopy(p)
    bad["options"]["n_period"] = 1000               # not a power of two
    assert _status(F, bad)[0] == F.FTHMS_EINVAL
    bad = copy.deepcopy(p)                          # period and time grid too long for the time kernels
    bad["options"]["n_period"] = 16384
    bad["options"]["Q"] = 4
    st, msg = _status(F, bad)
    assert st == F.FTHMS_EINVAL and "shared memory" in msg
    bad = copy.deepcopy(p)                          # unknown cross mode
    bad["options"]["cross_mode"] = 2
    assert _status(F, bad)[0] == F.FTHMS_EINVAL
    assert _status(F, p, precision=3)[0] == F.FTHMS_ENOTIMPL
    bad = copy.deepcopy(p)                          # refinement options out of range
    bad["options"]["refine_max"] = 17
    assert _status(F, bad, precision=1)[0] == F.FTHMS_EINVAL
    bad["options"]["refine_max"] = 3
    bad["options"]["refine_tol"] = -1.0
    assert _status(F, bad, precision=1)[0] == F.FTHMS_EINVAL
    smp = wl.multipulse_samples(t_end=20.0)          # sampled signals: too few samples, bad step or band
    for key, val in (("f", smp["f"][:7]), ("dt", 0.0), ("band", 0.0)):
        bad = wl.with_samples(p, dict(smp, **{key: val}))
        st, msg = _status(F, bad)
        assert st == F.FTHMS_EINVAL and "sampled" in msg
    bad = wl.with_samples(p, dict(smp, f=np.where(np.arange(smp["f"].size) == 5, np.nan, smp["f"])))
    assert _status(F, bad)[0] == F.FTHMS_EINVAL


def test_launch_shapes_in_the_options_are_validated(F):
    """fthms_options.shapes: the autotuner's candidates (0 = default) pass; anything else, and an LU choice in
    the FP64 form (one LU path), is EINVAL; the choices change no device memory."""
    p = wl.random_small(0)
    ok = copy.deepcopy(p)
    ok["options"]["shapes"] = [1, 256, 512, 64, 256]
    assert F.fthms_plan_info(F.Marshalled(ok, precision=1)) == F.fthms_plan_info(F.Marshalled(p, precision=1))
    ok["options"]["shapes"] = [4, 128, 256, 128, 0]
    F.fthms_plan_info(F.Marshalled(ok, precision=0))
    for bad_shapes, prec in (([3, 0, 0, 0, 0], 1), ([0, 32, 0, 0, 0], 1), ([0, 0, 1024, 0, 0], 1),
                             ([0, 0, 0, 512, 0], 1), ([0, 0, 0, 0, 100], 1), ([0, 0, 0, 0, 256], 0)):
        bad = copy.deepcopy(p)
        bad["options"]["shapes"] = bad_shapes
        st, msg = _status(F, bad, precision=prec)
        assert st == F.FTHMS_EINVAL and "shapes" in msg


def test_sampled_signal_plans_like_the_analytic_one(F):
    """A job whose signal is given by samples plans to the same systems; its device memory holds the
    samples as well."""
    p = wl.random_small(3, kind=1)
    smp = wl.multipulse_samples(t_end=30.0)
    b0, n0 = F.fthms_plan_info(F.Marshalled(p))
    b1, n1 = F.fthms_plan_info(F.Marshalled(wl.with_samples(p, smp)))
    assert n0 == n1 and b1 == b0 + 8 * smp["f"].size
