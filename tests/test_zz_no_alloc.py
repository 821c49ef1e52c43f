"""The allocation-free self-matrix entry point gives the same matrices as the allocating one.

fthms_assemble_self_noalloc serves callers that must not allocate device memory (an application whose
allocator owns the device, a process under a fixed memory cap, a pipeline that cannot accept the
device-wide synchronisation of cudaFree): it keeps its temporary data in a static device array of the
library.  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-13   # same bar as the self-matrix parity test (relative to max |A|)


def _matrix(fn, curve, arc, N, kappa):
    A = torch.full((2 * N * N,), float("nan"), dtype=torch.float64, device="cuda")
    fn(curve, arc, N, kappa, A.data_ptr())
    torch.cuda.synchronize()        # the allocation-free call is asynchronous on its stream
    return A.cpu().numpy()


def test_noalloc_matches_allocating_entry_point_twice():
    from paper_2507_05725_gb300 import fthms as F
    torch.cuda.set_device(0)
    cases = [(wl.kite(0.3, -0.2), (-1.9, 1.7), 200, 33.0), (wl.ellipse(1.0, 0.6), (-1.2, 2.4), 48, 0.7)]
    for curve, arc, N, kappa in cases:     # two calls in a row, different sizes
        ref = _matrix(F.fthms_assemble_self, curve, arc, N, kappa)
        got = _matrix(F.fthms_assemble_self_noalloc, curve, arc, N, kappa)
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref)) <= TOL * np.max(np.abs(ref))


@pytest.mark.parametrize("N,kappa", [(256, 41.0), (2, 0.3)])
def test_noalloc_at_the_scratch_limits(N, kappa):
    """N = 256 fills the static array (136 tiles, the whole log table); N = 2 is the smallest system."""
    from paper_2507_05725_gb300 import fthms as F
    torch.cuda.set_device(0)
    curve, arc = wl.star(0.3, 5, 0.4), (-1.1, 1.4)
    ref = _matrix(F.fthms_assemble_self, curve, arc, N, kappa)
    got = _matrix(F.fthms_assemble_self_noalloc, curve, arc, N, kappa)
    assert np.all(np.isfinite(got))
    assert np.max(np.abs(got - ref)) <= TOL * np.max(np.abs(ref))


@pytest.mark.parametrize("N", [1, 257, 300])
def test_noalloc_rejects_sizes_outside_the_scratch(N):
    from paper_2507_05725_gb300 import fthms as F
    A = torch.empty(2 * max(N, 2) ** 2, dtype=torch.float64, device="cuda")
    with pytest.raises(F.FthmsError) as e:
        F.fthms_assemble_self_noalloc(wl.circle(1.0), (-1.0, 1.0), N, 2.0, A.data_ptr())
    assert e.value.status == F.FTHMS_EINVAL and "256" in str(e.value)
