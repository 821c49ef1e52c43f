"""Seeded synthetic FTH-MS problem descriptions shared by the oracle, the tests and the bench.

This module only *describes* problems: curve coefficients, arc parameter intervals, signal and
discretisation parameters, observation points.  It holds none of the method's arithmetic (no
nodes, windows, kernels, transforms), so that the CPU oracle and the CUDA path can both consume
the same inputs while sharing no computation.

A problem is a plain dict:

* ``curves``: list of trig-polynomial curves ``X(theta) = sum_k (ax[k] cos k theta + bx[k] sin k theta,
  ay[k] cos k theta + by[k] sin k theta)``, k = 0..degree (the ``b[0]`` entries are unused).
* ``arcs``: list of ``(curve_index, theta_a, theta_b)`` with ``theta_b > theta_a`` (may exceed 2 pi);
  consecutive arcs of one closed curve overlap their neighbours only (Section 3.1).
* ``signal``: incident field ``u^i``; ``kind`` 0 = point source at ``z0``, 1 = plane wave along ``dir``;
  time signal ``f(t) = amp sin(carrier t) exp(-((t - centre)/width)^2)``, or samples of f given by an
  optional ``samples`` entry ``{"t0", "dt", "f", "band"}``; boundary data is ``sign * u^i``
  (``sign = -1`` for scattering, ``+1`` when the boundary carries the field itself).
* ``options``: ``W`` (max frequency), ``L`` (frequencies ``omega_l = l W/(L-1)``, l = 0..L-1),
  the per-arc node-count rule ``N = N_fixed`` if nonzero else
  ``max(N_min, ceil(N_ppw * omega * arclength) + N_off)``, ``M`` multiple-scattering steps,
  ``Q`` time windows of half-width ``H``, ``n_period`` time samples per period ``2 pi/h`` of the
  uniform frequency grid, observation points and output times.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "circle", "ellipse", "kite", "star", "split_closed_curve", "config1", "config2",
    "config2_reduced", "config3", "config3_reduced", "config4", "random_small", "served_requests", "problem_summary",
    "multipulse_samples", "with_samples",
]


def circle(r, cx=0.0, cy=0.0):
    return {"ax": [cx, r], "bx": [0.0, 0.0], "ay": [cy, 0.0], "by": [0.0, r]}


def ellipse(a, b, cx=0.0, cy=0.0):
    return {"ax": [cx, a], "bx": [0.0, 0.0], "ay": [cy, 0.0], "by": [0.0, b]}


def kite(cx=0.0, cy=0.0):
    # x(s) = cos s + 0.65 cos 2s - 0.65, y(s) = 1.5 sin s
    return {"ax": [cx - 0.65, 1.0, 0.65], "bx": [0.0, 0.0, 0.0],
            "ay": [cy, 0.0, 0.0], "by": [0.0, 1.5, 0.0]}


def star(amp=0.3, lobes=5, phase=0.0, cx=0.0, cy=0.0):
    """r(theta) = 1 + amp cos(lobes theta + phase), written as a trig polynomial of degree lobes+1."""
    deg = lobes + 1
    ax = [0.0] * (deg + 1); bx = [0.0] * (deg + 1); ay = [0.0] * (deg + 1); by = [0.0] * (deg + 1)
    ax[0] += cx; ay[0] += cy
    ax[1] += 1.0; by[1] += 1.0
    # amp cos(n t + p) cos t = amp/2 [cos((n+1)t + p) + cos((n-1)t + p)]
    # amp cos(n t + p) sin t = amp/2 [sin((n+1)t + p) - sin((n-1)t + p)]
    c, s = math.cos(phase), math.sin(phase)
    for m, sgn in ((lobes + 1, 1.0), (lobes - 1, -1.0)):
        ax[m] += 0.5 * amp * c; bx[m] += -0.5 * amp * s
        by[m] += sgn * 0.5 * amp * c; ay[m] += sgn * 0.5 * amp * s
    return {"ax": ax, "bx": bx, "ay": ay, "by": by}


def split_closed_curve(curve_index, n, span_factor=1.25, theta_off=0.0):
    """n overlapping arcs of span span_factor*2pi/n centred at theta_off + 2 pi k/n."""
    span = span_factor * 2.0 * math.pi / n
    arcs = []
    for k in range(n):
        c = theta_off + 2.0 * math.pi * k / n
        arcs.append((curve_index, c - 0.5 * span, c + 0.5 * span))
    return arcs


def _signal(kind, sign, amp, carrier, centre, width, z0=(0.0, 0.0), direction=(1.0, 0.0)):
    return {"kind": int(kind), "z0": [float(z0[0]), float(z0[1])],
            "dir": [float(direction[0]), float(direction[1])], "sign": float(sign),
            "amp": float(amp), "carrier": float(carrier), "centre": float(centre), "width": float(width)}


def _options(W, L, M, Q, H, n_period, obs, tout0, dtout, n_tout, N_fixed=0, N_min=0, N_off=0,
             N_ppw=0.0, interior=0):
    return {"W": float(W), "L": int(L), "N_fixed": int(N_fixed), "N_min": int(N_min), "N_off": int(N_off),
            "N_ppw": float(N_ppw), "M": int(M), "Q": int(Q), "H": float(H), "n_period": int(n_period),
            "interior": int(interior), "obs": np.asarray(obs, dtype=np.float64).reshape(-1, 2),
            "tout0": float(tout0), "dtout": float(dtout), "n_tout": int(n_tout)}


def config1(L=257, M=8, N=96):
    """Unit disk, 3 arcs of 150 deg at 0/120/240 deg, interior point source at (2, 0.5),
    f(t) = sin(4t) exp(-((t-4)/1.5)^2), boundary data = +field (exact interior solution = u^i),
    N = 96, omega in [0, 24] with 257 points, M = 8, 5 interior observation points, t in [0, 10]."""
    curves = [circle(1.0)]
    arcs = split_closed_curve(0, 3, 1.25, 0.0)
    signal = _signal(0, +1.0, 1.0, 4.0, 4.0, 1.5, z0=(2.0, 0.5))
    obs = [(0.5, 0.0), (0.0, 0.0), (-0.3, 0.4), (0.2, -0.6), (-0.5, -0.2)]
    options = _options(24.0, L, M, 1, 20.0, 2048, obs, 0.0, 0.05, 201, N_fixed=N, interior=1)
    return {"name": "disk3-pointsource", "curves": curves, "arcs": arcs, "signal": signal, "options": options}


def _min_gap(c1, c2, n=720):
    th = np.linspace(0.0, 2.0 * math.pi, n, endpoint=False)

    def pts(c):
        x = np.zeros_like(th); y = np.zeros_like(th)
        for k in range(len(c["ax"])):
            x += c["ax"][k] * np.cos(k * th) + c["bx"][k] * np.sin(k * th)
            y += c["ay"][k] * np.cos(k * th) + c["by"][k] * np.sin(k * th)
        return np.stack([x, y], 1)

    a, b = pts(c1), pts(c2)
    return float(np.min(np.linalg.norm(a[:, None, :] - b[None, :, :], axis=2)))


def config2(seed=2, L=1025, M=12, W=60.0, Q=1, H=40.0, n_period=4096, n_tout=201, T=20.0):
    """Exterior problem, 4 obstacles (ellipses (1,0.6) and (0.8,0.5), kite, circle r=0.7) at seeded
    positions with pairwise gap >= 0.5, each split into 2 overlapping arcs (8 arcs), plane-wave pulse
    f(t) = sin(10t) exp(-((t-6)/2)^2) at a seeded angle, N = max(48, ceil(2 omega len/pi) + 16),
    omega in [0, 60] with 1025 points, M = 12, outputs at 5 points on a circle of radius 6."""
    rng = np.random.default_rng(seed)
    makers = [lambda cx, cy: ellipse(1.0, 0.6, cx, cy), lambda cx, cy: ellipse(0.8, 0.5, cx, cy),
              lambda cx, cy: kite(cx, cy), lambda cx, cy: circle(0.7, cx, cy)]
    curves = []
    for mk in makers:
        for _ in range(10000):
            cx, cy = rng.uniform(-2.5, 2.5, size=2)
            c = mk(float(cx), float(cy))
            if all(_min_gap(c, o) >= 0.5 for o in curves):
                curves.append(c)
                break
        else:
            raise RuntimeError("could not place obstacle")
    arcs = []
    for ci in range(len(curves)):
        arcs += split_closed_curve(ci, 2, 1.25, 0.0)
    ang = float(rng.uniform(0.0, 2.0 * math.pi))
    signal = _signal(1, -1.0, 1.0, 10.0, 6.0, 2.0, direction=(math.cos(ang), math.sin(ang)))
    ph = float(rng.uniform(0.0, 2.0 * math.pi))
    obs = [(6.0 * math.cos(ph + 2 * math.pi * k / 5), 6.0 * math.sin(ph + 2 * math.pi * k / 5)) for k in range(5)]
    options = _options(W, L, M, Q, H, n_period, obs, 0.0, T / (n_tout - 1), n_tout,
                       N_min=48, N_off=16, N_ppw=2.0 / math.pi, interior=0)
    return {"name": "4obstacles-planewave", "curves": curves, "arcs": arcs, "signal": signal, "options": options}


def config2_reduced(seed=2, L=129, M=3, W=30.0, H=12.0, n_period=1024):
    """Config 2's geometry, signal and node-count rule on a band omega <= 30 (N from 48 to ~140)
    with 129 frequencies, H = 12 and fewer steps, sized for the oracle to finish in seconds."""
    return config2(seed=seed, L=L, M=M, W=W, H=H, n_period=n_period, T=14.0)


def config3(seed=3, L=2049, M=8, W=200.0, Q=4, H=12.0, n_period=8192, carrier=30.0, centre=20.0, width=8.0,
            N_min=32, N_off=16, N_ppw=3.6, n_tout=601, T=60.0):
    """Interior problem in a seeded star-shaped cavity r(theta) = 1 + 0.3 cos(5 theta + phi), split into 12
    overlapping arcs; boundary data = +field of a point source at (2.5, 0.7) outside the cavity (so the
    exact interior solution is u^i); f(t) = sin(30t) exp(-((t-20)/8)^2) on t in [0, 60] with 4 windows
    (H = 12); N = max(32, ceil(3.6 omega len) + 16) from 32 to ~760 over omega in [0, 200] with 2049 points
    (dt = pi/400 internally); M = 8; 5 interior observation points.  Its cross rows (~10^11 entries) do not
    fit in device memory, so the job evaluates them every step (cross_mode = 1)."""
    rng = np.random.default_rng(seed)
    curves = [star(0.3, 5, float(rng.uniform(0.0, 2.0 * math.pi)))]
    arcs = split_closed_curve(0, 12, 1.25, 0.0)
    signal = _signal(0, +1.0, 1.0, carrier, centre, width, z0=(2.5, 0.7))
    obs = [(0.0, 0.0), (0.3, 0.2), (-0.4, 0.1), (0.1, -0.5), (-0.2, -0.3)]
    options = _options(W, L, M, Q, H, n_period, obs, 0.0, T / (n_tout - 1), n_tout, N_min=N_min, N_off=N_off,
                       N_ppw=N_ppw, interior=1)
    options["cross_mode"] = 1
    return {"name": "star12-cavity", "curves": curves, "arcs": arcs, "signal": signal, "options": options}


def config3_reduced(seed=3, L=129, M=2, W=16.0, Q=2, n_period=1024):
    """Config 3's cavity, arcs and node rule on omega in [0, 16] (N from 32 to ~76), the carrier moved
    into that band (sin(6t) exp(-((t-8)/3)^2)), Q = 2 windows."""
    return config3(seed=seed, L=L, M=M, W=W, Q=Q, H=12.0, n_period=n_period, carrier=6.0, centre=8.0,
                   width=3.0, n_tout=121, T=30.0)


def config4(N=512, seed=4, L=1024, M=8, W=400.0, Q=2, H=4.0, n_period=4096, carrier=200.0, centre=3.0, width=0.5,
            n_tout=201, T=8.0, cross_mode=None):
    """Mixed-precision configuration: 6 arcs of a seeded exterior configuration of 5 ellipses with semi-axes
    uniform in [0.4, 1.2] at seeded positions with pairwise gap >= 0.5 -- the first ellipse closed and split
    into 2 overlapping arcs, the other four open elliptic-arc obstacles of 270 deg span at seeded
    orientations (6 arcs cannot cover 5 closed curves) -- N nodes on every arc (512, 1024 or 2048 per batch),
    1024 frequencies on [0, 400] (1023 solved), M = 8, Q = 2 windows with H = 4 on t in [0, 8] (dt = pi/800
    internally), plane-wave pulse sin(200t) exp(-((t-3)/0.5)^2) at a seeded angle, 5 observation points on a
    circle of radius 6.  Cross rows stored for N <= 512 (121 GB), evaluated every step above.  Up to 8
    refinement passes: at N = 512 the top of the band has ~1.6 nodes per wavelength and a few of those
    systems need more than 3."""
    rng = np.random.default_rng(seed)
    curves = []
    for _ in range(5):
        a, b = (float(v) for v in rng.uniform(0.4, 1.2, size=2))
        for _ in range(10000):
            cx, cy = rng.uniform(-3.0, 3.0, size=2)
            c = ellipse(a, b, float(cx), float(cy))
            if all(_min_gap(c, o) >= 0.5 for o in curves):
                curves.append(c)
                break
        else:
            raise RuntimeError("could not place obstacle")
    arcs = split_closed_curve(0, 2, 1.25, 0.0)
    for ci in range(1, 5):
        c0 = float(rng.uniform(0.0, 2.0 * math.pi))
        arcs.append((ci, c0 - 0.75 * math.pi, c0 + 0.75 * math.pi))
    ang = float(rng.uniform(0.0, 2.0 * math.pi))
    signal = _signal(1, -1.0, 1.0, carrier, centre, width, direction=(math.cos(ang), math.sin(ang)))
    ph = float(rng.uniform(0.0, 2.0 * math.pi))
    obs = [(6.0 * math.cos(ph + 2 * math.pi * k / 5), 6.0 * math.sin(ph + 2 * math.pi * k / 5)) for k in range(5)]
    options = _options(W, L, M, Q, H, n_period, obs, 0.0, T / (n_tout - 1), n_tout, N_fixed=N, interior=0)
    options["cross_mode"] = (0 if N <= 512 else 1) if cross_mode is None else cross_mode
    options["refine_max"] = 8          # some systems at the band's top (~1.6 nodes per wavelength) converge slowly
    return {"name": f"5ellipses6arcs-N{N}", "curves": curves, "arcs": arcs, "signal": signal, "options": options}


def random_small(seed, n_arcs_per_curve=3, n_curves=1, L=33, M=2, Q=1, N_fixed=0, W=10.0, kind=None,
                 H=8.0, n_period=256):
    """Tiny seeded problems for edge-case parity (few frequencies, small N, ragged sizes)."""
    rng = np.random.default_rng(seed)
    curves = []
    for ci in range(n_curves):
        cx, cy = 4.0 * ci, 0.0
        t = rng.integers(0, 3)
        if t == 0:
            curves.append(circle(float(rng.uniform(0.6, 1.2)), cx, cy))
        elif t == 1:
            curves.append(ellipse(float(rng.uniform(0.7, 1.2)), float(rng.uniform(0.4, 0.7)), cx, cy))
        else:
            curves.append(star(0.2, 5, float(rng.uniform(0, 2 * math.pi)), cx, cy))
    arcs = []
    for ci in range(n_curves):
        arcs += split_closed_curve(ci, n_arcs_per_curve, 1.25, float(rng.uniform(0, 2 * math.pi)))
    if kind is None:
        kind = int(rng.integers(0, 2))
    if kind == 0:
        signal = _signal(0, -1.0, 1.0, float(rng.uniform(3, 6)), 2.5, 1.0, z0=(4.0 * (n_curves - 1) + 2.2, 0.8))
    else:
        a = float(rng.uniform(0, 2 * math.pi))
        signal = _signal(1, -1.0, 1.0, float(rng.uniform(3, 6)), 2.5, 1.0, direction=(math.cos(a), math.sin(a)))
    obs = [(0.0, 3.0), (4.0 * (n_curves - 1) + 3.0, 0.0)]
    options = _options(W, L, M, Q, H, n_period, obs, 0.0, 0.1, 61,
                       N_fixed=N_fixed, N_min=12, N_off=6, N_ppw=1.0 / math.pi)
    return {"name": f"small-{seed}", "curves": curves, "arcs": arcs, "signal": signal, "options": options}


def served_requests(seed, n, wmax=(20.0, 60.0), Ls=(129, 257), arcs=(2, 6)):
    """Seeded request mix shaped like the served stream of the fifth configuration, scaled to a bounded
    sample: each request draws a disk (interior), a star cavity (interior) or 1-5 separated ellipse
    obstacles (exterior, 2 arcs each) with a number of arcs in the `arcs` range, a band omega_max uniform in
    `wmax`, a frequency count from `Ls`, the config-2 node rule, a Gaussian-modulated sinusoid with carrier in
    [2, min(40, omega_max - 8/b)] and width b in [1, 3], and 3-6 steps."""
    rng = np.random.default_rng(seed)
    lo, hi = arcs
    out = []
    for r in range(n):
        kind = int(rng.integers(0, 3))
        W = float(rng.uniform(*wmax))
        L = int(rng.choice(list(Ls)))
        b = float(rng.uniform(1.0, 3.0))
        a = float(rng.uniform(2.0, max(2.5, min(40.0, W - 8.0 / b))))
        M = int(rng.integers(3, 7))
        period = 2.0 * math.pi * (L - 1) / W
        H = float(min(12.0, 0.45 * period))
        if kind == 0:
            curves = [circle(float(rng.uniform(0.8, 1.2)))]
            na = int(rng.integers(max(2, lo), min(6, hi) + 1))
            arcs_ = split_closed_curve(0, na, 1.25, float(rng.uniform(0, 2 * math.pi)))
            signal = _signal(0, +1.0, 1.0, a, 3.0 * b, b, z0=(2.5, float(rng.uniform(-1, 1))))
            obs = [(0.2, 0.1), (-0.3, 0.2)]
            interior = 1
        elif kind == 1:
            curves = [star(0.3, 5, float(rng.uniform(0, 2 * math.pi)))]
            na = int(rng.integers(max(4, lo), max(4, min(12, hi)) + 1))
            arcs_ = split_closed_curve(0, na, 1.25, float(rng.uniform(0, 2 * math.pi)))
            signal = _signal(0, +1.0, 1.0, a, 3.0 * b, b, z0=(2.6, 0.3))
            obs = [(0.1, 0.0), (0.0, 0.3)]
            interior = 1
        else:
            k = int(rng.integers(max(1, lo // 2), max(1, min(5, hi // 2)) + 1))
            curves = [ellipse(float(rng.uniform(0.5, 1.0)), float(rng.uniform(0.3, 0.6)), 3.0 * i, 0.0)
                      for i in range(k)]
            arcs_ = []
            for ci in range(k):
                arcs_ += split_closed_curve(ci, 2, 1.25, 0.0)
            ang = float(rng.uniform(0, 2 * math.pi))
            signal = _signal(1, -1.0, 1.0, a, 3.0 * b + 4.0, b, direction=(math.cos(ang), math.sin(ang)))
            obs = [(1.5 * k, 3.0), (-3.0, -1.0)]
            interior = 0
        options = _options(W, L, M, 1, H, 1024, obs, 0.0, 0.1, 61, N_min=24, N_off=16, N_ppw=2.0 / math.pi,
                           interior=interior)
        out.append({"name": f"served-{seed}-{r}", "curves": curves, "arcs": arcs_, "signal": signal,
                    "options": options})
    return out


def multipulse_samples(t0=0.0, dt=0.01, t_end=60.0, t_lag=2.0, pulses=5, spacing=10.0):
    """Samples of the multi-pulse time profile of Section 5 (eq. multi: five copies of the pulse u3 of eq.
    planewave, 10 time units apart): f(s) = sum_j -sin(4 (s - t_lag - spacing j)) exp(-1.6 (s - t_lag -
    spacing j - 3)^2) at s = t0 + i dt, for a plane wave u = f(t - x.d).  Returns the "samples" entry of a
    signal dict; band = 4 + 8 sqrt(1.6) is the carrier plus eight Gaussian widths."""
    n = int(round((t_end - t0) / dt)) + 1
    s = t0 + dt * np.arange(n)
    f = np.zeros(n)
    for j in range(pulses):
        ell = s - t_lag - spacing * j
        f += -np.sin(4.0 * ell) * np.exp(-1.6 * (ell - 3.0) ** 2)
    return {"t0": float(t0), "dt": float(dt), "f": f, "band": 4.0 + 8.0 * math.sqrt(1.6)}


def with_samples(problem, samples):
    """The same problem with its signal given by samples (the analytic parameters are then unused)."""
    q = dict(problem)
    q["signal"] = dict(problem["signal"], samples=samples)
    return q


def problem_summary(p):
    o = p["options"]
    return (f"{p['name']}: {len(p['curves'])} curves, {len(p['arcs'])} arcs, L={o['L']}, W={o['W']}, "
            f"M={o['M']}, Q={o['Q']}, H={o['H']}, n_period={o['n_period']}")
