"""Time signals, incident fields, time windows and the omega <-> t transforms for the oracle.

Test infrastructure only (see the package docstring).

Paper passages: Fourier convention of eqs. forwardFT/backwardFT (Section 2.1); windowing and
recentring of eqs. windowing, Fourierk and TDsol (Section 2.1); the window sqcap built from eta
with s_q = (3/2)(q-1)H (Section 5); the slow transform viewed as a periodic expansion of the
windowed integrand (Section 4.1).

Discrete form (our reading; the paper's FC/FCC transforms are replaced by a uniform grid):
  omega_l = l h, h = W/(L-1), l = 1..L-1 solved (omega = 0 is not solved and contributes nothing)
  t_n = t_0 + n dt, t_0 = -H, dt = 2 pi/(h n_period), n = 0..N_T-1 covering [-H, s_Q + H]
  forward   G_q(omega_l) = dt sum_n g(t_n) sqcap_q(t_n) e^{i omega_l (t_n - s_q)}
  inverse   v(t) = sum_q [valid_q(t)] (1/pi) Re sum_l w_l V_q(omega_l) e^{-i omega_l (t - s_q)}
            with w_l = h (l < L-1), h/2 (l = L-1), valid_q(t): -H <= t - s_q < 2 pi/h - H.
  Phases: e^{i omega_l (t_n - s_q)} = e^{i l*c_q} e^{2 pi i (l n mod n_period)/n_period} with
  c_q = h*(t_0 - s_q): the same number, with the integer part of the phase reduced exactly.
"""
from __future__ import annotations

import math

import numpy as np

from .geometry import eta


def sampled_signal(smp, t):
    """Sampled signal f[i] = f(t0 + i dt) read between the samples (our reading of "a boundary time
    signal" given as data; the paper's own signals are analytic): the degree-7 Lagrange interpolant through
    the samples floor(s) - 3 .. floor(s) + 4, s = (t - t0)/dt, a sample index outside 0..n-1 counting as a
    zero sample, and f = 0 outside [t0, t0 + (n-1) dt].  Weight of sample i0 + k at x = s - i0:
    prod_{m != k} (x - m)/(k - m)."""
    t = np.asarray(t, dtype=np.float64)
    f = np.asarray(smp["f"], dtype=np.float64)
    n = f.size
    t0, dt = float(smp["t0"]), float(smp["dt"])
    tend = t0 + (n - 1) * dt
    out = np.zeros(t.shape)
    inside = (t >= t0) & (t <= tend)
    s = (t[inside] - t0) / dt
    fl = np.floor(s)
    i0 = fl.astype(np.int64) - 3
    x = s - fl + 3.0
    acc = np.zeros(x.shape)
    for k in range(8):
        w = np.ones(x.shape)
        for m in range(8):
            if m != k:
                w *= (x - m) / (k - m)
        idx = i0 + k
        ok = (idx >= 0) & (idx < n)
        acc += w * np.where(ok, f[np.clip(idx, 0, n - 1)], 0.0)
    out[inside] = acc
    return out


def signal_f(sig, t):
    """f(t) = amp sin(carrier t) exp(-((t - centre)/width)^2), or the sampled signal of sig["samples"]."""
    t = np.asarray(t, dtype=np.float64)
    if sig.get("samples") is not None:
        return sampled_signal(sig["samples"], t)
    return sig["amp"] * np.sin(sig["carrier"] * t) * np.exp(-((t - sig["centre"]) / sig["width"]) ** 2)


def signal_F(sig, omega):
    """Closed-form transform F(omega) = int f(t) e^{i omega t} dt of signal_f (eq. forwardFT):
    (amp b sqrt(pi)/(2i)) [e^{i(omega+a)c - b^2(omega+a)^2/4} - e^{i(omega-a)c - b^2(omega-a)^2/4}]."""
    a, b, c, A = sig["carrier"], sig["width"], sig["centre"], sig["amp"]
    w = np.asarray(omega, dtype=np.float64)
    e1 = np.exp(1j * (w + a) * c - b * b * (w + a) ** 2 / 4.0)
    e2 = np.exp(1j * (w - a) * c - b * b * (w - a) ** 2 / 4.0)
    return A * b * math.sqrt(math.pi) / 2j * (e1 - e2)


def point_source_rule(sig, r, t):
    """Integration range and node count of the trapezoid rule in v for the 2-D retarded field
    u(r, t) = (1/(2 pi)) int_0^inf f(t - r cosh v) dv (tau = r cosh v in the convolution of f with
    H(t-r)/(2 pi sqrt(t^2 - r^2))).  The analytic f is below e^{-64} outside |tau - (t - centre)| <=
    8 width, with bandwidth B = |carrier| + 8/width; a sampled f vanishes outside its sample range and
    carries its stated bandwidth B = band.  Returns (v_lo, v_hi, n_intervals) or None when the integrand
    vanishes."""
    smp = sig.get("samples")
    if smp is not None:
        tau_hi = t - smp["t0"]
        tau_lo_c = t - (smp["t0"] + (len(smp["f"]) - 1) * smp["dt"])
        band = smp["band"]
    else:
        tau_hi = t - sig["centre"] + 8.0 * sig["width"]
        tau_lo_c = t - sig["centre"] - 8.0 * sig["width"]
        band = abs(sig["carrier"]) + 8.0 / sig["width"]
    if tau_hi <= r:
        return None
    tau_lo = max(r, tau_lo_c)
    if tau_lo >= tau_hi:
        return None
    v_lo = math.acosh(tau_lo / r)
    v_hi = math.acosh(tau_hi / r)
    rate = band * r * math.sinh(v_hi) + 1.0
    n = int(math.ceil((v_hi - v_lo) * (1.25 * rate + 24.0) / (2.0 * math.pi) * 2.0)) + 16
    return v_lo, v_hi, n


def incident_field(sig, x, t):
    """u^i(x, t) at points x (P, 2) and times t (T,) -> (P, T).
    kind 1: plane wave f(t - x.d).  kind 0: point source at z0, trapezoid rule in v (even
    integrand: half weight at v = 0 when the range starts there)."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, 2)
    t = np.asarray(t, dtype=np.float64)
    if sig["kind"] == 1:
        d = np.asarray(sig["dir"], dtype=np.float64)
        return signal_f(sig, t[None, :] - (x @ d)[:, None])
    z0 = np.asarray(sig["z0"], dtype=np.float64)
    out = np.zeros((x.shape[0], t.shape[0]))
    for p in range(x.shape[0]):
        r = float(np.linalg.norm(x[p] - z0))
        for n_, tn in enumerate(t):
            rule = point_source_rule(sig, r, float(tn))
            if rule is None:
                continue
            v_lo, v_hi, n = rule
            v = np.linspace(v_lo, v_hi, n + 1)
            f = signal_f(sig, tn - r * np.cosh(v))
            dv = (v_hi - v_lo) / n
            wts = np.full(n + 1, dv)
            wts[-1] = 0.5 * dv
            wts[0] = 0.5 * dv          # v_lo = 0: half weight of the symmetric rule; else f ~ 0 there
            out[p, n_] = np.dot(wts, f) / (2.0 * math.pi)
    return out


def window(s, H):
    """sqcap(s) of Section 5: eta(s/H; 1/2, 1) for -H/2 <= s <= H, 1 - eta(s/H + 3/2; 1/2, 1) for
    -H < s < -H/2, 0 for |s| >= H."""
    s = np.asarray(s, dtype=np.float64)
    out = np.zeros(s.shape)
    a = (s >= -H / 2.0) & (s <= H)
    out[a] = eta(s[a] / H, 0.5, 1.0)
    b = (s > -H) & (s < -H / 2.0)
    out[b] = 1.0 - eta(s[b] / H + 1.5, 0.5, 1.0)
    out[np.abs(s) >= H] = 0.0
    return out


class TimeGrid:
    """Frequency grid and internal time grid of one problem (see the module docstring)."""

    def __init__(self, options):
        o = options
        self.W = o["W"]; self.L = o["L"]; self.Q = o["Q"]; self.H = o["H"]; self.K = o["n_period"]
        self.h = self.W / (self.L - 1)
        self.omega = np.array([l * self.h for l in range(self.L)])
        self.dt = 2.0 * math.pi / (self.h * self.K)
        if 2.0 * math.pi / self.h < 2.0 * self.H:
            raise ValueError("window support 2H exceeds the period 2 pi/h of the frequency grid")
        self.t0 = -self.H
        self.s = np.array([1.5 * q * self.H for q in range(self.Q)])      # s_q, q = 1..Q (0-based)
        self.NT = int((self.s[-1] + 2.0 * self.H) / self.dt) + 1
        self.t = self.t0 + np.arange(self.NT) * self.dt
        self.period = 2.0 * math.pi / self.h
        self.wl = np.full(self.L, self.h)
        self.wl[0] = 0.0
        self.wl[-1] = 0.5 * self.h
        self.c = np.array([self.h * (self.t0 - sq) for sq in self.s])     # c_q = h (t_0 - s_q)
        self.nlo = np.array([int(math.ceil(sq / self.dt - 1e-9)) for sq in self.s])
        self.win = np.stack([window(self.t - sq, self.H) for sq in self.s])   # sqcap_q(t_n)

    def _phase_grid(self, q, sign):
        """e^{sign * i omega_l (t_n - s_q)} = e^{sign i l c_q} e^{sign 2 pi i (l n mod K)/K} for
        l = 0..L-1, n = 0..N_T-1 (the integer part of the phase reduced exactly)."""
        l = np.arange(self.L, dtype=np.int64)
        n = np.arange(self.NT, dtype=np.int64)
        m = np.mod(np.outer(l, n), self.K).astype(np.float64)
        a = np.exp(sign * 1j * (l.astype(np.float64) * self.c[q]))
        return a[:, None] * np.exp(sign * 2j * math.pi * m / self.K)

    def forward(self, g):
        """Slow forward transform (eq. Fourierk) of real samples g[..., N_T] -> [..., Q, L]."""
        out = []
        for q in range(self.Q):
            E = self._phase_grid(q, +1.0)                  # (L, N_T)
            out.append(self.dt * (g * self.win[q]) @ E.T)
        return np.stack(out, axis=-2)

    def inverse(self, V):
        """Recentred inverse transform (eq. TDsol) of V[..., Q, L] on the internal grid -> [..., N_T],
        each window used on its valid range only."""
        v = np.zeros(V.shape[:-2] + (self.NT,))
        for q in range(self.Q):
            E = self._phase_grid(q, -1.0)                  # (L, N_T)
            vq = ((V[..., q, :] * self.wl) @ E).real / math.pi
            valid = np.zeros(self.NT, dtype=bool)
            valid[self.nlo[q]:self.nlo[q] + self.K] = True
            v += np.where(valid, vq, 0.0)
        return v

    def inverse_at(self, V, tout):
        """Recentred inverse transform at arbitrary output times (direct evaluation, T4)."""
        tout = np.asarray(tout, dtype=np.float64)
        v = np.zeros(V.shape[:-2] + tout.shape)
        l = np.arange(self.L, dtype=np.float64)
        for q in range(self.Q):
            c = self.h * (tout - self.s[q])                    # h (t - s_q)
            E = np.exp(-1j * np.outer(l, c))                   # (L, T): phase l * c
            vq = ((V[..., q, :] * self.wl) @ E).real / math.pi
            rel = tout - self.s[q]
            valid = (rel >= -self.H) & (rel < self.period - self.H)
            v += np.where(valid, vq, 0.0)
        return v
