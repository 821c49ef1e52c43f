"""Geometry of the overlapping-arc decomposition (Section 3.1) for the oracle.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import math

import numpy as np

TWO_PI = 2.0 * math.pi


def curve_eval(curve, theta):
    """Trig-polynomial curve X(theta) and its derivative X'(theta); theta any shape -> (..., 2)."""
    theta = np.asarray(theta, dtype=np.float64)
    x = np.zeros(theta.shape); y = np.zeros(theta.shape)
    dx = np.zeros(theta.shape); dy = np.zeros(theta.shape)
    for k in range(len(curve["ax"])):
        c = np.cos(k * theta); s = np.sin(k * theta)
        x += curve["ax"][k] * c + curve["bx"][k] * s
        y += curve["ay"][k] * c + curve["by"][k] * s
        dx += k * (-curve["ax"][k] * s + curve["bx"][k] * c)
        dy += k * (-curve["ay"][k] * s + curve["by"][k] * c)
    return np.stack([x, y], -1), np.stack([dx, dy], -1)


def wrap_pi(a):
    """Representative of an angle in (-pi, pi]."""
    a = np.asarray(a, dtype=np.float64)
    r = np.mod(a + math.pi, TWO_PI) - math.pi
    return np.where(r <= -math.pi, r + TWO_PI, r)


def cheb_nodes(n):
    """First-kind Chebyshev nodes t_i = cos((2i+1) pi/(2n)), i = 0..n-1 (decreasing)."""
    i = np.arange(n, dtype=np.float64)
    return np.cos((2.0 * i + 1.0) * math.pi / (2.0 * n))


def eta(t, t0, t1):
    """Smooth cut-off of eq. eta: 1 for |t| <= t0, exp(2 e^{-1/s}/(s-1)) with
    s = (|t|-t0)/(t1-t0) for t0 < |t| < t1, and 0 for |t| >= t1."""
    t = np.abs(np.asarray(t, dtype=np.float64))
    out = np.zeros(t.shape)
    out[t <= t0] = 1.0
    mid = (t > t0) & (t < t1)
    s = (t[mid] - t0) / (t1 - t0)
    out[mid] = np.exp(2.0 * np.exp(-1.0 / s) / (s - 1.0))
    return out


class Arc:
    """Open arc Gamma_j = X([theta_a, theta_b]) parametrised by t in [-1, 1]:
    theta(t) = theta_c + half * t (the arc parametrisation assumed by the open-arc solver,
    Section 4.3)."""

    def __init__(self, index, curve_index, curve, theta_a, theta_b):
        self.index = index
        self.curve_index = curve_index
        self.curve = curve
        self.theta_a = float(theta_a)
        self.theta_b = float(theta_b)
        self.theta_c = 0.5 * (self.theta_a + self.theta_b)
        self.half = 0.5 * (self.theta_b - self.theta_a)
        self.prev = None  # neighbour overlapping the theta_a end
        self.next = None  # neighbour overlapping the theta_b end

    def point(self, t):
        X, dX = curve_eval(self.curve, self.theta_c + self.half * np.asarray(t, dtype=np.float64))
        return X, dX * self.half

    def length(self):
        """Arc length int_{-1}^{1} |x'(t)| dt by 128-point Gauss-Legendre quadrature."""
        s, w = np.polynomial.legendre.leggauss(128)
        _, d = self.point(s)
        return float(np.sum(w * np.linalg.norm(d, axis=-1)))

    def local_param(self, theta):
        """t* such that theta = theta_c + half*t*, using the periodic representative of theta
        nearest to the arc's centre."""
        return wrap_pi(np.asarray(theta, dtype=np.float64) - self.theta_c) / self.half


def build_arcs(problem):
    """Arcs with their cyclic neighbours on each curve (Section 3.1: each patch overlaps only
    Gamma_{j-1} and Gamma_{j+1}).  A curve with a single arc is an open-arc obstacle (no
    neighbours, chi = 1)."""
    arcs = [Arc(i, ci, problem["curves"][ci], ta, tb) for i, (ci, ta, tb) in enumerate(problem["arcs"])]
    by_curve = {}
    for a in arcs:
        by_curve.setdefault(a.curve_index, []).append(a)
    for lst in by_curve.values():
        if len(lst) < 2:
            continue
        lst.sort(key=lambda a: float(np.mod(a.theta_c, TWO_PI)))
        n = len(lst)
        for k, a in enumerate(lst):
            a.next = lst[(k + 1) % n]
            a.prev = lst[(k - 1) % n]
    return arcs


def chi(arc, t, c0=1.0 / 3.0, c1=2.0 / 3.0):
    """Boundary partition of unity chi_j of eq. POU1 at the points x_j(t) of arc j.

    Reading: the overlap diameter A is the chord between the overlap's two ends and d(x) is the
    chord from x to the endpoint of the arc that lies in that overlap (equal to the set diameters
    for the arcs used here).  Right overlap (with next): eta(A - d; c0 A, c1 A) with d measured to
    x(theta_b); left overlap (with prev): 1 - eta(A - d; c0 A, c1 A) with d measured to prev's
    theta_b end.  c0 = 1/3, c1 = 2/3 as in Section 3.1."""
    t = np.asarray(t, dtype=np.float64)
    out = np.ones(t.shape)
    if arc.next is None:
        return out
    X, _ = arc.point(t)
    theta = arc.theta_c + arc.half * t
    # right overlap: theta in [next.theta_a, theta_b]
    nxt = arc.next
    d_right = wrap_pi(theta - nxt.theta_a)       # >= 0 inside the overlap
    span_r = wrap_pi(arc.theta_b - nxt.theta_a)
    in_r = (d_right >= 0.0) & (d_right <= span_r) & (t > 0)
    end_r = curve_eval(arc.curve, arc.theta_b)[0]
    far_r = curve_eval(arc.curve, nxt.theta_a)[0]
    A_r = float(np.linalg.norm(far_r - end_r))
    if np.any(in_r):
        d = np.linalg.norm(X[in_r] - end_r, axis=-1)
        out[in_r] = eta(A_r - d, c0 * A_r, c1 * A_r)
    # left overlap: theta in [theta_a, prev.theta_b]
    prv = arc.prev
    d_left = wrap_pi(prv.theta_b - theta)
    span_l = wrap_pi(prv.theta_b - arc.theta_a)
    in_l = (d_left >= 0.0) & (d_left <= span_l) & (t < 0)
    end_l = curve_eval(arc.curve, prv.theta_b)[0]
    far_l = curve_eval(arc.curve, arc.theta_a)[0]
    A_l = float(np.linalg.norm(far_l - end_l))
    if np.any(in_l):
        d = np.linalg.norm(X[in_l] - end_l, axis=-1)
        out[in_l] = 1.0 - eta(A_l - d, c0 * A_l, c1 * A_l)
    return out


def node_count(problem, arc_len, omega):
    """Per-arc node count: N_fixed, else max(N_min, ceil(N_ppw * omega * length - 1e-9) + N_off).
    The ceiling is taken 1e-9 below the product so that a product that is an integer in exact
    arithmetic (equal arcs of a circle at a grid frequency) gives that integer whatever the last bit
    of the quadrature length."""
    o = problem["options"]
    if o["N_fixed"] > 0:
        return int(o["N_fixed"])
    return max(int(o["N_min"]), int(math.ceil(o["N_ppw"] * omega * arc_len - 1e-9)) + int(o["N_off"]))


def delta_min(problem, samples=4001):
    """delta_min of eq. dist: the smallest distance between a truncated patch Gamma_j^tr (the points of
    Gamma_j where chi_j > 0) and the rest of the boundary Gamma minus Gamma_j, over the patches of every
    closed curve; by dense sampling of the curve (an upper bound within the sampling step)."""
    arcs = build_arcs(problem)
    best = math.inf
    for a in arcs:
        if a.next is None:
            continue
        theta = np.linspace(0.0, TWO_PI, samples, endpoint=False)
        X = curve_eval(a.curve, theta)[0]
        ts = a.local_param(theta)
        inside = np.abs(ts) <= 1.0
        tr = inside.copy()
        tr[inside] = chi(a, ts[inside]) > 0.0
        if not np.any(tr) or np.all(inside):
            continue
        d = np.linalg.norm(X[tr][:, None, :] - X[~inside][None, :, :], axis=-1)
        best = min(best, float(np.min(d)))
    return best
