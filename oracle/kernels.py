"""Single-layer kernel, its log split and the open-arc Chebyshev product-integration rule.

Test infrastructure only (see the package docstring).

Paper passages: the fundamental solution Phi_omega = (i/4) H0^(1)(kappa|x-y|) (Section 2.1), the
single-layer operator V_Gamma_j of eq. FDBIEk-interior and potential S_Gamma_j of eq.
FDsolk-interior (Section 3.2), the endpoint form psi = alpha/w of eq. singularity (Section 4.3) and
the decomposition of the singular kernel that Section 4.2 takes over for many frequencies.

Discrete form (our reading of those passages, single-patch Chebyshev):
  unknown   phi(t) = Psi(x(t)) |x'(t)| sqrt(1 - t^2)  (smooth alpha of eq. singularity)
  equation  int_{-1}^{1} K(t, s) phi(s) / sqrt(1 - s^2) ds = G(x(t)),  K = Phi(x(t), x(s))
  split     K = K1 log|t - s| + K2,  K1 = -J0(kappa R)/(2 pi)
  rule      A_il = K1(t_i, t_l) Rlog_il + K2(t_i, t_l) pi/N   on first-kind nodes
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

from .geometry import cheb_nodes

EULER_GAMMA = 0.57721566490153286060651209008240243


def phi_kernel(z):
    """(i/4) H0^(1)(z) = (i/4) (J0(z) + i Y0(z)) for z > 0 (Section 2.1)."""
    return 0.25j * (special.j0(z) + 1j * special.y0(z))


def rlog_self(n):
    """Weights of int_{-1}^{1} log|t_i - s| p(s)/sqrt(1-s^2) ds for the degree-(n-1) interpolant p
    on the first-kind nodes, from int log|t-s| T_k(s)/sqrt(1-s^2) ds = -pi ln 2 (k = 0) and
    -(pi/k) T_k(t) (k >= 1):
        Rlog_il = -(pi/n) [ln 2 + 2 sum_{k=1}^{n-1} T_k(t_i) T_k(t_l) / k]."""
    t = cheb_nodes(n)
    k = np.arange(1, n, dtype=np.float64)
    T = np.cos(np.outer(np.arccos(t), k))          # T_k(t_i), k = 1..n-1
    return -(math.pi / n) * (math.log(2.0) + 2.0 * (T / k) @ T.T)


def log_moments_outside(tstar, n):
    """lambda_k(t*) = int_{-1}^{1} log|t* - s| T_k(s)/sqrt(1-s^2) ds for |t*| > 1, k = 0..n-1:
    pi ln((|t*| + sqrt(t*^2-1))/2) for k = 0 and -(pi/k) z^k, z = t* - sgn(t*) sqrt(t*^2 - 1),
    for k >= 1 (from the generating function of the Chebyshev polynomials)."""
    tstar = np.asarray(tstar, dtype=np.float64)
    r = np.sqrt(tstar * tstar - 1.0)
    z = tstar - np.sign(tstar) * r
    k = np.arange(n, dtype=np.float64)
    lam = np.empty(tstar.shape + (n,))
    lam[..., 0] = math.pi * np.log((np.abs(tstar) + r) / 2.0)
    lam[..., 1:] = -(math.pi / k[1:]) * z[..., None] ** k[1:]
    return lam


def rlog_outside(tstar, n):
    """Product-integration weights for a target parameter |t*| > 1 (the near rule):
    Rlog(t*)_l = (1/n) [lambda_0 + 2 sum_{k=1}^{n-1} lambda_k(t*) T_k(t_l)]."""
    t = cheb_nodes(n)
    lam = log_moments_outside(tstar, n)
    T = np.cos(np.outer(np.arange(n, dtype=np.float64), np.arccos(t)))   # T_k(t_l)
    w = 2.0 * (lam @ T)
    w -= lam[..., :1] * T[0]            # the k = 0 term enters once
    return w / n


def self_matrix(arc, n, kappa):
    """Nystrom matrix A (n x n, complex) of V_Gamma_j on arc j at wavenumber kappa (S1-S3):
    off-diagonal K2 = K - K1 log|t_i - t_l| (the definition); diagonal K2 = i/4 -
    (1/(2 pi)) [gamma + ln(kappa |x'(t_i)|/2)] (the limit t -> s of the same definition)."""
    t = cheb_nodes(n)
    X, dX = arc.point(t)
    R = np.linalg.norm(X[:, None, :] - X[None, :, :], axis=-1)
    dt = np.abs(t[:, None] - t[None, :])
    off = ~np.eye(n, dtype=bool)
    z = kappa * R[off]
    J0 = special.j0(z)
    K1 = np.zeros((n, n))
    K2 = np.zeros((n, n), dtype=np.complex128)
    K1[off] = -J0 / (2.0 * math.pi)
    K2[off] = phi_kernel(z) - K1[off] * np.log(dt[off])
    speed = np.linalg.norm(dX, axis=-1)
    diag = np.arange(n)
    K1[diag, diag] = -1.0 / (2.0 * math.pi)
    K2[diag, diag] = 0.25j - (EULER_GAMMA + np.log(kappa * speed / 2.0)) / (2.0 * math.pi)
    return K1 * rlog_self(n) + K2 * (math.pi / n)


def cross_rows(arc, n, kappa, targets, tstar, near):
    """Rows E[r, l] of S_Gamma_j at targets y_r (Section 3.2, eq. FDsolk-interior) acting on the
    nodal values phi_l of arc j with n nodes:
      far rule  E = Phi(y_r, x_l) pi/n
      near rule (same curve, 1 < |t*| <= 3) E = K1(t*, t_l) Rlog(t*)_l + K2(t*, t_l) pi/n with
                K2 = K - K1 log|t* - t_l|."""
    t = cheb_nodes(n)
    X, _ = arc.point(t)
    targets = np.asarray(targets, dtype=np.float64).reshape(-1, 2)
    R = np.linalg.norm(targets[:, None, :] - X[None, :, :], axis=-1)
    z = kappa * R
    K = phi_kernel(z)
    E = K * (math.pi / n)
    near = np.asarray(near, dtype=bool)
    if np.any(near):
        ts = np.asarray(tstar)[near]
        zn = z[near]
        K1 = -special.j0(zn) / (2.0 * math.pi)
        K2 = K[near] - K1 * np.log(np.abs(ts[:, None] - t[None, :]))
        E[near] = K1 * rlog_outside(ts, n) + K2 * (math.pi / n)
    return E


def restriction(n, nmax):
    """Values at the n first-kind nodes of the degree-(nmax-1) Chebyshev interpolant through the
    nmax transfer-mesh nodes: R[i, x] = (1/nmax) [1 + 2 sum_{k=1}^{nmax-1} T_k(t_i) T_k(tau_x)]."""
    t = cheb_nodes(n)
    tau = cheb_nodes(nmax)
    k = np.arange(1, nmax, dtype=np.float64)
    Tt = np.cos(np.outer(np.arccos(t), k))
    Ttau = np.cos(np.outer(np.arccos(tau), k))
    return (1.0 + 2.0 * Tt @ Ttau.T) / nmax
