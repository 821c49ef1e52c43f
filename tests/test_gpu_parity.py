"""GPU (C ABI) vs CPU oracle parity of the FTH-MS hot path.

Bar: densities phi_{j,m,q}(omega_l) within 1e-11 relative L2 of the FP64 oracle (all j, m, q, l
together and per step m); traces within 1e-10 of the trace scale; node counts identical.
"""
import json
import math
import os

import numpy as np
import pytest
import torch
from scipy import special

import workloads as wl
from oracle import kernels as oker
from oracle import run_oracle
from oracle.fthms import Setup
from oracle.transforms import incident_field

pytestmark = pytest.mark.gpu

DENSITY_TOL = 1e-11
TRACE_TOL = 1e-10


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


def test_bessel0_against_scipy(F):
    z = np.concatenate([np.geomspace(1e-6, 4.0, 600), [4.0, np.nextafter(4.0, 5.0), 19.999999, 20.0],
                        np.linspace(4.0, 20.0, 3001), np.linspace(20.0, 3000.0, 4001)])
    zt = torch.tensor(z, dtype=torch.float64, device="cuda")
    j0, y0, yh = (torch.empty_like(zt) for _ in range(3))
    F.fthms_bessel0(zt.data_ptr(), j0.data_ptr(), y0.data_ptr(), yh.data_ptr(), z.size)
    torch.cuda.synchronize()
    j0, y0, yh = j0.cpu().numpy(), y0.cpu().numpy(), yh.cpu().numpy()
    rj, ry = special.j0(z), special.y0(z)
    amp = np.where(z > 1.0, np.sqrt(2.0 / (np.pi * z)), 1.0)
    # scipy's Cephes j0/y0 are themselves off by up to 3.4e-15 of the amplitude on this grid
    # (against 40-digit values); the device functions are within 1.5e-15 there.
    assert np.max(np.abs(j0 - rj) / amp) < 5e-15
    assert np.max(np.abs(y0 - ry) / np.maximum(amp, np.abs(ry))) < 5e-15
    ryh = ry - (2.0 / np.pi) * (np.log(z / 2.0) + np.euler_gamma) * rj
    small = z < 20.0
    assert np.max(np.abs(yh - ryh)[small] / (1.0 + np.abs(np.log(z[small])))) < 5e-15


@pytest.mark.parametrize("case", [("kite", 64, 7.3), ("ellipse", 33, 0.05), ("circle", 96, 24.0),
                                  ("kite", 259, 60.0), ("star", 5, 3.0)])
def test_self_matrix_against_oracle(F, case):
    name, N, kappa = case
    curve = {"kite": wl.kite(0.3, -0.2), "ellipse": wl.ellipse(1.0, 0.6), "circle": wl.circle(1.0),
             "star": wl.star(0.3, 5, 0.4)}[name]
    ta, tb = -1.9, 1.7
    A = torch.empty(2 * N * N, dtype=torch.float64, device="cuda")
    F.fthms_assemble_self(curve, (ta, tb), N, kappa, A.data_ptr())
    torch.cuda.synchronize()
    a = A.cpu().numpy()
    Ag = (a[0::2] + 1j * a[1::2]).reshape(N, N).T
    from oracle.geometry import Arc
    Ao = oker.self_matrix(Arc(0, 0, curve, ta, tb), N, kappa)
    assert np.max(np.abs(Ag - Ao)) < 1e-13 * np.max(np.abs(Ao))


def _parity(F, ctx, problem):
    job = F.Job(ctx, problem).run().wait()
    ref = run_oracle(problem)
    o = problem["options"]
    P, L, M, Q = len(problem["arcs"]), o["L"], o["M"], o["Q"]
    assert np.array_equal(job.node_counts(), ref.Ntab[:, 1:])
    num = den = 0.0
    for m in range(1, M + 1):
        nm = dm = 0.0
        for j in range(P):
            for q in range(Q):
                d = job.densities(j, m, q)
                for l in range(1, L):
                    r = ref.phi[(m, j, l)][q]
                    nm += float(np.sum(np.abs(d[l] - r) ** 2))
                    dm += float(np.sum(np.abs(r) ** 2))
        if dm == 0.0:            # no cross fields (a lone arc): every later step is exactly zero
            assert nm == 0.0, (m, nm)
            continue
        assert math.sqrt(nm / dm) < DENSITY_TOL, (m, math.sqrt(nm / dm))
        num += nm
        den += dm
    # the sum over m (m = 0 in the C ABI), same relative-L2 bar
    ns = ds = 0.0
    for j in range(P):
        d = job.densities(j, 0, 0)
        for l in range(1, L):
            r = sum(ref.phi[(m, j, l)][0] for m in range(1, M + 1))
            ns += float(np.sum(np.abs(d[l] - r) ** 2))
            ds += float(np.sum(np.abs(r) ** 2))
    assert math.sqrt(ns / ds) < DENSITY_TOL
    tr = job.traces()
    scale = max(1e-300, np.max(np.abs(ref.traces)))
    assert np.max(np.abs(tr - ref.traces)) < TRACE_TOL * scale
    st = job.stats()
    job.release()
    return math.sqrt(num / den), st


SMALL = {
    "small-plane": lambda: wl.random_small(0, n_arcs_per_curve=3, kind=1),
    "small-point": lambda: wl.random_small(2, n_arcs_per_curve=3, kind=0, M=3),
    "two-curves-Q2": lambda: wl.random_small(5, n_curves=2, n_arcs_per_curve=2, Q=2, L=65, M=2),
    "four-arcs": lambda: wl.random_small(7, n_arcs_per_curve=4, M=3),
    "fixed-N": lambda: wl.random_small(9, n_arcs_per_curve=3, N_fixed=20, M=2),
    "tiny-L": lambda: wl.random_small(11, n_arcs_per_curve=3, L=17, H=4.0, M=2),
}


@pytest.mark.parametrize("name", sorted(SMALL))
def test_small_problem_parity(F, ctx, name):
    rel, st = _parity(F, ctx, SMALL[name]())
    assert rel < DENSITY_TOL


def test_config1_parity(F, ctx):
    """Disk, 3 arcs, N = 96, 256 solved frequencies, M = 8 (the full first configuration)."""
    rel, st = _parity(F, ctx, wl.config1())
    assert rel < DENSITY_TOL


def test_config2_reduced_parity(F, ctx):
    """Config 2's geometry, signal and node rule on a narrower band (N from 48 to ~140)."""
    rel, st = _parity(F, ctx, wl.config2_reduced(M=2))
    assert rel < DENSITY_TOL


def test_config2_full_size_sampled(F, ctx):
    """Full-size config 2 in the bench's launch configuration: m = 1 densities of sampled (arc,
    omega) systems against the oracle computed system by system (relative L2 over the samples;
    the band where the pulse's spectrum lives, omega in [4, 16], plus both band edges), and finite
    traces."""
    problem = wl.config2(M=2)
    job = F.Job(ctx, problem).run().wait()
    S = Setup(problem)
    assert np.array_equal(job.node_counts(), S.Ntab[:, 1:])   # every (arc, omega), so every transfer mesh
    tg = S.grid
    sig = problem["signal"]
    rng = np.random.default_rng(0)
    num = den = 0.0
    for j in (0, 3, 4, 7):
        g = sig["sign"] * S.chi[j][:, None] * incident_field(sig, S.X[j], tg.t)
        Gt = tg.forward(g)                              # [Nmax, Q, L]
        d = job.densities(j, 1, 0)
        band = rng.integers(int(4.0 / tg.h), int(16.0 / tg.h), size=4).tolist()
        for l in sorted(set(band) | {1, tg.L - 1}):
            n = int(S.Ntab[j, l])
            G = oker.restriction(n, int(S.Nmax[j])) @ Gt[:, 0, l]
            phi = np.linalg.solve(oker.self_matrix(S.arcs[j], n, tg.omega[l]), G)
            num += float(np.sum(np.abs(d[l] - phi) ** 2))
            den += float(np.sum(np.abs(phi) ** 2))
    assert math.sqrt(num / den) < DENSITY_TOL
    tr = job.traces()
    assert np.all(np.isfinite(tr)) and np.max(np.abs(tr)) > 0
    job.release()


# ---- mixed-precision form (FP32 factors, double-float refinement and cross apply) --------------

MIXED_TOL = 1e-10   # density bar of the mixed-precision form (rel. L2 against the FP64 oracle)


def _golden_m2():
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "config2_m2_arc4.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("precision", [0, 1])
def test_config2_full_size_second_step(F, ctx, precision):
    """Full-size config 2: m = 2 densities of arc 4 at sampled frequencies against the stored oracle
    values (tests/golden/make_config2_m2.py: every m = 1 density, the cross fields of all other
    arcs on arc 4's transfer mesh, synthesis, windowed forward transform, restriction, solve), so
    the whole multiple-scattering step is covered at the bench's size."""
    gold = _golden_m2()
    job = F.Job(ctx, wl.config2(M=2), precision=precision).run().wait()
    d = job.densities(gold["arc"], gold["m"], gold["q"])
    num = den = 0.0
    for l, v in gold["samples"].items():
        r = np.asarray(v["re"]) + 1j * np.asarray(v["im"])
        num += float(np.sum(np.abs(d[int(l)] - r) ** 2))
        den += float(np.sum(np.abs(r) ** 2))
    job.release()
    assert math.sqrt(num / den) < (DENSITY_TOL if precision == 0 else MIXED_TOL)




def _parity_mixed(F, ctx, problem):
    job = F.Job(ctx, problem, precision=1).run().wait()
    ref = run_oracle(problem)
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
    tr = job.traces()
    st = job.stats()
    job.release()
    assert st["precision"] == 1
    assert 0.0 <= st["max_refine_resid"] < MIXED_TOL
    scale = max(1e-300, np.max(np.abs(ref.traces)))
    assert np.max(np.abs(tr - ref.traces)) < MIXED_TOL * scale
    return math.sqrt(num / den)


@pytest.mark.parametrize("name", ["small-point", "two-curves-Q2", "four-arcs"])
def test_mixed_small_parity(F, ctx, name):
    assert _parity_mixed(F, ctx, SMALL[name]()) < MIXED_TOL


def test_mixed_config1_parity(F, ctx):
    assert _parity_mixed(F, ctx, wl.config1()) < MIXED_TOL


def test_mixed_config2_reduced_parity(F, ctx):
    assert _parity_mixed(F, ctx, wl.config2_reduced(M=2)) < MIXED_TOL


def test_mixed_matches_plain_at_full_size(F, ctx):
    """Full-size config 2: the mixed form's summed densities against the FP64 form's."""
    problem = wl.config2(M=3)
    a = F.Job(ctx, problem, keep_densities=False, precision=0).run().wait()
    b = F.Job(ctx, problem, keep_densities=False, precision=1).run().wait()
    num = den = 0.0
    for j in range(len(problem["arcs"])):
        x, y = a.densities(j, 0, 0), b.densities(j, 0, 0)
        for l in x:
            num += float(np.sum(np.abs(x[l] - y[l]) ** 2))
            den += float(np.sum(np.abs(x[l]) ** 2))
    a.release()
    b.release()
    assert math.sqrt(num / den) < MIXED_TOL


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_replay_matches_direct_launches(F, ctx, precision):
    """A job captured into a CUDA graph and replayed gives the same densities and traces (both forms)."""
    problem = wl.random_small(5, n_curves=2, n_arcs_per_curve=2, Q=2, L=65, M=2)
    a = F.Job(ctx, problem, precision=precision).run().wait()
    b = F.Job(ctx, problem, precision=precision)
    try:
        F.fthms_use_graph(b.req, True)
        b.run().wait()
        b.run().wait()                       # replay
        assert np.array_equal(a.traces(), b.traces())
        for j in range(len(problem["arcs"])):
            da, db = a.densities(j, 2, 1), b.densities(j, 2, 1)
            for l in da:
                assert np.array_equal(da[l], db[l])
        assert b.stats()["gpu_ms"] > 0.0
    finally:
        a.release()
        b.release()


# ---- edge cases ---------------------------------------------------------------------------------

def _edge(name):
    if name == "no-observation-points":
        p = wl.random_small(1)
        p["options"]["obs"] = np.zeros((0, 2))
        return p
    if name == "single-step":
        return wl.random_small(2, M=1)
    if name == "four-windows":
        return wl.random_small(4, Q=4, L=129, H=5.0, M=2)
    if name == "two-frequencies":
        return wl.random_small(6, L=3, H=0.5, M=2)
    if name == "open-arc-obstacle":
        p = wl.random_small(8, M=2)
        p["arcs"] = [(0, -1.0, 1.3)]                 # one arc alone on its curve: chi = 1, no cross pairs
        return p
    raise KeyError(name)


@pytest.mark.parametrize("name", ["no-observation-points", "single-step", "four-windows", "two-frequencies",
                                  "open-arc-obstacle"])
def test_edge_case_parity(F, ctx, name):
    p = _edge(name)
    if p["options"]["obs"].size == 0:
        job = F.Job(ctx, p).run().wait()
        ref = run_oracle(p)
        assert job.traces().size == 0
        num = den = 0.0
        for (m, j, l), r in ref.phi.items():
            d = job.densities(j, m, 0)[l]
            num += float(np.sum(np.abs(d - r[0]) ** 2))
            den += float(np.sum(np.abs(r[0]) ** 2))
        job.release()
        assert math.sqrt(num / den) < DENSITY_TOL
        return
    rel, st = _parity(F, ctx, p)
    assert rel < DENSITY_TOL


def test_largest_supported_system(F, ctx):
    """N = 800 on every system (the largest node count the LU panel supports), two frequencies."""
    p = wl.random_small(12, n_arcs_per_curve=2, N_fixed=800, L=3, H=0.5, M=2, W=10.0)
    rel, st = _parity(F, ctx, p)
    assert rel < DENSITY_TOL
    big = wl.random_small(12, n_arcs_per_curve=2, N_fixed=801, L=3, H=0.5, M=1)
    with pytest.raises(F.FthmsError) as e:
        F.Job(ctx, big)
    assert e.value.status == F.FTHMS_EINVAL and "800" in str(e.value)


# ---- cross rows evaluated every step (cross_mode 1) ------------------------------------------------

def _cross_mode(problem, mode):
    problem["options"]["cross_mode"] = mode
    return problem


@pytest.mark.parametrize("name", ["small-plane", "two-curves-Q2", "four-arcs"])
@pytest.mark.parametrize("precision", [0, 1])
def test_on_the_fly_cross_matches_stored(F, ctx, name, precision):
    """Evaluating the cross rows in every step gives the densities and traces of the stored rows (the same
    entries, summed in another order; the mixed form's stored rows are double-float)."""
    tol = 1e-12 if precision == 0 else 1e-11
    a = F.Job(ctx, _cross_mode(SMALL[name](), 0), precision=precision).run().wait()
    b = F.Job(ctx, _cross_mode(SMALL[name](), 1), precision=precision).run().wait()
    P = len(SMALL[name]()["arcs"])
    num = den = 0.0
    for j in range(P):
        da, db = a.densities(j, 0, 0), b.densities(j, 0, 0)
        for l in da:
            num += float(np.sum(np.abs(da[l] - db[l]) ** 2))
            den += float(np.sum(np.abs(da[l]) ** 2))
    ta, tb = a.traces(), b.traces()
    a.release()
    b.release()
    assert math.sqrt(num / den) < tol
    assert np.max(np.abs(ta - tb)) < tol * max(1e-300, np.max(np.abs(ta)))


def test_on_the_fly_cross_parity(F, ctx):
    rel, st = _parity(F, ctx, _cross_mode(wl.random_small(7, n_arcs_per_curve=4, M=3), 1))
    assert rel < DENSITY_TOL


def test_config3_reduced_parity(F, ctx):
    """Config 3's 12-arc star cavity (one curve: every arc sees every other, near rows on both sides) on
    omega <= 16 with two windows, cross rows evaluated every step."""
    rel, st = _parity(F, ctx, wl.config3_reduced())
    assert rel < DENSITY_TOL


def test_config3_reduced_mixed_parity(F, ctx):
    assert _parity_mixed(F, ctx, wl.config3_reduced()) < MIXED_TOL


# ---- autotuned launch shapes -------------------------------------------------------------------------

@pytest.mark.parametrize("precision", [0, 1])
def test_autotune_keeps_results_bitwise(F, ctx, precision):
    """Tuned launch shapes change no number: densities and traces identical to the default shapes."""
    problem = wl.random_small(5, n_curves=2, n_arcs_per_curve=2, Q=2, L=65, M=2)
    a = F.Job(ctx, problem, precision=precision).run().wait()
    b = F.Job(ctx, problem, precision=precision)
    try:
        shapes = F.fthms_autotune(b.req, 2)
        assert shapes[0] in (1, 2, 4) and shapes[1] in (64, 128, 256)
        assert shapes[2] in (128, 256, 512) and shapes[3] in (64, 128, 256)
        b.run().wait()
        assert np.array_equal(a.traces(), b.traces())
        for j in range(len(problem["arcs"])):
            for q in range(2):
                da, db = a.densities(j, 0, q), b.densities(j, 0, q)
                for l in da:
                    assert np.array_equal(da[l], db[l])
    finally:
        a.release()
        b.release()


# ---- full-size third configuration (12-arc star cavity) against stored oracle values --------------

def _golden_c3():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "config3_m2.json")
    with open(path) as f:
        return json.load(f)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_config3_full_size_second_step(F, ctx, precision):
    """Full-size 12-arc star cavity (N 32..760, 2048 solved frequencies, Q = 4 windows, point-source data,
    cross rows evaluated every step, in the bench's launch configuration): m = 2 densities of two receiving
    arcs, all four windows, at six frequencies across (0, 200] including the largest system, against the
    oracle values of tests/golden/make_config3_m2.py (every m = 1 density, the cross fields of all other
    arcs, synthesis, windowed forward transform, restriction and solve)."""
    gold = _golden_c3()
    job = F.Job(ctx, wl.config3(M=2), precision=precision).run().wait()
    num = den = 0.0
    for key, v in gold["samples"].items():
        k, l = (int(x) for x in key.split(":"))
        ref = np.asarray(v["re"]) + 1j * np.asarray(v["im"])          # (Q, N)
        for q in range(ref.shape[0]):
            d = job.densities(k, 2, q)[l]
            assert d.shape == ref[q].shape
            num += float(np.sum(np.abs(d - ref[q]) ** 2))
            den += float(np.sum(np.abs(ref[q]) ** 2))
    st = job.stats()
    job.release()
    rel = math.sqrt(num / den)
    assert rel < (DENSITY_TOL if precision == 0 else MIXED_TOL), rel
    if precision:
        assert st["n_unconverged"] == 0
