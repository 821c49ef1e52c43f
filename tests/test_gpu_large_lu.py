"""Large systems (N up to 2048) in the mixed forms: FP32 LU with tensor-core (tcgen05, 3xTF32) trailing
updates, refined against the kept matrix, through the C ABI against the FP64 oracle."""
import copy
import math

import numpy as np
import pytest
import torch

import workloads as wl
from oracle import run_oracle

pytestmark = pytest.mark.gpu

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


def _problem(N, kind=1):
    """Two overlapping arcs of one seeded curve, two solved frequencies (omega = 6 and 12), N nodes per arc,
    cross rows evaluated every step (stored rows stop at N = 1427)."""
    p = wl.random_small(13, n_arcs_per_curve=2, N_fixed=N, L=3, H=0.25, M=2, W=12.0, kind=kind, n_period=64)
    p["options"]["cross_mode"] = 1
    return p


@pytest.mark.parametrize("N", [801, 1024, 2048])
@pytest.mark.parametrize("precision", [1, 2])
def test_large_system_parity(F, ctx, N, precision):
    problem = _problem(N)
    job = F.Job(ctx, problem, precision=precision).run().wait()
    ref = run_oracle(problem)
    num = den = 0.0
    for m in (1, 2):
        for j in range(2):
            d = job.densities(j, m, 0)
            for l in (1, 2):
                r = ref.phi[(m, j, l)][0]
                assert d[l].shape == r.shape
                num += float(np.sum(np.abs(d[l] - r) ** 2))
                den += float(np.sum(np.abs(r) ** 2))
    st = job.stats()
    tr = job.traces()
    job.release()
    rel = math.sqrt(num / den)
    assert rel < MIXED_TOL, rel
    assert st["n_unconverged"] == 0 and st["max_refine_resid"] < 1e-12
    # an FP32-accurate factor needs about two refinement passes; a TF32-only one would need many more
    assert st["refine_passes"] <= 3.0, st["refine_passes"]
    assert np.max(np.abs(tr - ref.traces)) < 10 * MIXED_TOL * max(1e-300, np.max(np.abs(ref.traces)))


@pytest.mark.parametrize("precision", [1, 2])
def test_set_shapes_moves_systems_to_the_tensor_core_lu(F, ctx, precision):
    """fthms_set_shapes (or fthms_options.shapes at prepare) with the LU choice 256 factors N = 300 systems
    with tensor-core updates instead of the one-CTA LU; both paths refine to the FP64 oracle's densities."""
    problem = _problem(300)
    ref = run_oracle(problem)
    in_options = copy.deepcopy(problem)
    in_options["options"]["shapes"] = [2, 128, 256, 128, 256]   # the same choices given at prepare
    for prob, shapes, n_tensor in ((problem, [0, 0, 0, 0, 0], 0), (problem, [2, 128, 256, 128, 256], 4),
                                   (in_options, None, 4)):
        job = F.Job(ctx, prob, precision=precision)
        if shapes is not None:
            F.fthms_set_shapes(job.req, shapes)
        job.run().wait()
        num = den = 0.0
        for m in (1, 2):
            for j in range(2):
                d = job.densities(j, m, 0)
                for l in (1, 2):
                    r = ref.phi[(m, j, l)][0]
                    num += float(np.sum(np.abs(d[l] - r) ** 2))
                    den += float(np.sum(np.abs(r) ** 2))
        st = job.stats()
        job.release()
        assert st["lu_tensor_systems"] == n_tensor
        assert st["n_unconverged"] == 0
        assert math.sqrt(num / den) < MIXED_TOL


def test_set_shapes_rejects_choices_outside_the_candidates(F, ctx):
    job = F.Job(ctx, _problem(300), precision=1)
    for bad in ([3, 0, 0, 0, 0], [0, 96, 0, 0, 0], [0, 0, 0, 0, 100], [0, 0, 0, 0, 1024]):
        with pytest.raises(F.FthmsError) as e:
            F.fthms_set_shapes(job.req, bad)
        assert e.value.status == F.FTHMS_EINVAL
    job.release()
    plain = F.Job(ctx, _problem(300), precision=0)
    with pytest.raises(F.FthmsError):
        F.fthms_set_shapes(plain.req, [0, 0, 0, 0, 256])   # the FP64 form has one LU path
    F.fthms_set_shapes(plain.req, [2, 0, 256, 0, 0])
    plain.release()


def test_fp64_form_refuses_the_largest_systems(F, ctx):
    with pytest.raises(F.FthmsError) as e:
        F.Job(ctx, _problem(1024), precision=0)
    assert e.value.status == F.FTHMS_EINVAL and "2048" in str(e.value)


@pytest.mark.parametrize("N,part", [(512, None), (1024, None), (2048, (4, 8))])
def test_config4_sampled_systems(F, ctx, N, part):
    """The mixed-precision configuration (6 arcs of 5 ellipses, N nodes on every arc, 1023 frequencies on
    (0, 400]) in the FP64-kept form, in the bench's launch configuration: m = 1 densities of sampled (arc,
    omega) systems -- the band's edges and the pulse's band around omega = 200 -- against oracle solves
    computed system by system.  N = 2048 (623 GB in full) runs rank 4 of an 8-way frequency partition (its 128
    frequencies from omega = 200 up, 77 GB): the m = 1 densities need no exchange between ranks."""
    import copy
    from oracle import kernels as oker
    from oracle.fthms import Setup
    from oracle.transforms import incident_field
    problem = wl.config4(N, M=1 if part else 2)
    run_problem = copy.deepcopy(problem)
    if part:
        run_problem["options"].update(omega_rank=part[0], omega_ranks=part[1])
    job = F.Job(ctx, run_problem, precision=2)
    if part:
        job.set_allreduce(lambda buf, n, stream: None)      # one rank alone: m = 1 is all that is checked
    job.run()
    st = job.stats()
    own = list(job.own_frequencies())
    assert st["n_unconverged"] == 0, st
    assert st["lu_tensor_systems"] == (len(problem["arcs"]) * len(own) if N > 800 else 0)
    S = Setup(problem)
    tg = S.grid
    sig = problem["signal"]
    num = den = 0.0
    picks = {own[0], own[0] + 4, own[0] + 9, own[-1]} if part else {1, 512, 515, tg.L - 1}
    for j in (0, 2, 5):
        g = sig["sign"] * S.chi[j][:, None] * incident_field(sig, S.X[j], tg.t)
        Gt = tg.forward(g)                                  # [Nmax, Q, L]
        d0, d1 = job.densities(j, 1, 0), job.densities(j, 1, 1)
        for l in sorted(picks):
            A = oker.self_matrix(S.arcs[j], N, tg.omega[l])
            for q, d in ((0, d0), (1, d1)):
                phi = np.linalg.solve(A, Gt[:, q, l])     # N = N_max: no restriction
                num += float(np.sum(np.abs(d[l] - phi) ** 2))
                den += float(np.sum(np.abs(phi) ** 2))
    job.release()
    assert math.sqrt(num / den) < MIXED_TOL, math.sqrt(num / den)
