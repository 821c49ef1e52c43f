"""Multiple-scattering driver of the interior/exterior FTH-MS method (Algorithm 1) for the oracle.

Test infrastructure only (see the package docstring).

Paper passages: Definition inductive_int with eqs. criterion_int1 (g_{j,1} = -chi_j u^i, here
sign * chi_j u^i), criterion_int2 (g_{j,m+1} = -chi_j sum_{k != j} vtilde_{k,j,m}) and vtilde (a
neighbour's field is dropped on the overlap, i.e. at points of Gamma_j that lie in Gamma_k); the
open-arc BIE (eqs. FDBIEk-interior, FDsolk-interior, TDsol-interior); Algorithm 1 (loops over m,
arcs and windows: slow transform, BIE solve, potential, inverse transform with shift, output sum
u_M of eq. mult-scatt-int); the exterior variant of Section 3.3 (same steps on the arcs of every
component).

Every arc k carries a fixed "transfer mesh" (its first-kind nodes at N_k^max = N_k(omega_{L-1}))
on which the time-domain data g_{k,m}(x, t) live; the frequency-domain data G_{k,m,q}(omega_l) on
the N_k(omega_l) solve nodes are the values there of the transfer mesh's Chebyshev interpolant.
Cross-arc fields are evaluated only at transfer nodes where chi_k > 0 (g = -chi_k * (...) is 0
elsewhere).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg

from . import geometry as geo
from . import kernels as ker
from .transforms import TimeGrid, incident_field


@dataclass
class OracleResult:
    Ntab: np.ndarray                 # [P, L] node counts (column 0 unused)
    Nmax: np.ndarray                 # [P]
    phi: dict = field(default_factory=dict)   # (m, j, l) -> complex (Q, N) densities, m = 1..M
    traces: np.ndarray = None        # [n_obs, n_tout]
    Vobs: np.ndarray = None          # [n_obs, Q, L] accumulated observation spectra
    G: dict = field(default_factory=dict)     # (m, j, l) -> complex (Q, N) BIE data (if kept)
    g: dict = field(default_factory=dict)     # (m, k) -> real (Nmax_k, N_T) time-domain data g_{k,m} (if kept)
    chi: list = None                 # per arc chi at transfer nodes
    grid: TimeGrid = None


class Setup:
    """Arcs, node counts, transfer meshes, chi and the cross-evaluation target structure."""

    def __init__(self, problem):
        self.problem = problem
        o = problem["options"]
        self.grid = TimeGrid(o)
        self.arcs = geo.build_arcs(problem)
        self.P = len(self.arcs)
        self.lengths = [a.length() for a in self.arcs]
        L = o["L"]
        self.Ntab = np.zeros((self.P, L), dtype=np.int64)
        for j in range(self.P):
            for l in range(1, L):
                self.Ntab[j, l] = geo.node_count(problem, self.lengths[j], self.grid.omega[l])
        self.Nmax = self.Ntab[:, L - 1].copy()
        self.tau, self.X, self.theta, self.chi, self.tgt = [], [], [], [], []
        for k, a in enumerate(self.arcs):
            tau = geo.cheb_nodes(int(self.Nmax[k]))
            self.tau.append(tau)
            self.X.append(a.point(tau)[0])
            self.theta.append(a.theta_c + a.half * tau)
            c = geo.chi(a, tau)
            self.chi.append(c)
            self.tgt.append(np.nonzero(c > 0.0)[0])
        # blocks[(k, j)] = (target rows (indices into transfer mesh of k), tstar, near flags)
        self.blocks = {}
        for k in range(self.P):
            for j in range(self.P):
                if j == k:
                    continue
                rows = self.tgt[k]
                aj, ak = self.arcs[j], self.arcs[k]
                if aj.curve_index == ak.curve_index:
                    ts = aj.local_param(self.theta[k][rows])
                    inc = np.abs(ts) > 1.0          # eq. vtilde: drop points of Gamma_j
                    rows, ts = rows[inc], ts[inc]
                    near = np.abs(ts) <= 3.0
                else:
                    ts = np.zeros(rows.shape)
                    near = np.zeros(rows.shape, dtype=bool)
                self.blocks[(k, j)] = (rows, ts, near)
        self.obs = np.asarray(o["obs"], dtype=np.float64).reshape(-1, 2)


def run_oracle(problem, M=None, keep_G=False, cache_cross=True, arcs_phi=None, omega_part=None, allreduce=None,
               keep_g=False):
    """Run Algorithm 1 on the discrete problem; returns an OracleResult.

    M overrides the number of multiple-scattering steps; ``arcs_phi`` limits which arcs' densities
    are kept (all by default).  ``omega_part = (r, R)`` runs rank r's share of a frequency partition: the
    solved frequencies l in [1 + r (L-1)/R, 1 + (r+1)(L-1)/R) (the per-frequency sub-problems of a step
    are independent, Section 3); the omega -> t synthesis of every step and the traces are then partial
    sums over those frequencies, which ``allreduce(array) -> array`` must sum across the ranks.  ``keep_g``
    keeps the time-domain data g_{k,m} on every transfer mesh (eqs. criterion_int1/2)."""
    S = Setup(problem)
    o = problem["options"]
    sig = problem["signal"]
    tg = S.grid
    L, Q, P = o["L"], o["Q"], S.P
    M = o["M"] if M is None else M
    res = OracleResult(Ntab=S.Ntab, Nmax=S.Nmax, chi=S.chi, grid=tg)
    keep = set(range(P)) if arcs_phi is None else set(arcs_phi)
    if omega_part is None:
        own = range(1, L)
    else:
        r, R = omega_part
        own = range(1 + r * (L - 1) // R, 1 + (r + 1) * (L - 1) // R)
    total = (lambda a: a) if omega_part is None else allreduce

    # Self matrices, factored once per (arc, omega) and reused for every m and q (Alg. 1, line 8).
    lu = {}
    for j in range(P):
        for l in own:
            A = ker.self_matrix(S.arcs[j], int(S.Ntab[j, l]), tg.omega[l])
            lu[(j, l)] = scipy.linalg.lu_factor(A)

    Rcache = {}

    def restrict(k, Gt):
        """Gt [Nmax_k, Q, L] on the transfer mesh -> {l: (Q, N_k(l))} on the solve nodes."""
        out = {}
        nmax = int(S.Nmax[k])
        for l in own:
            n = int(S.Ntab[k, l])
            if (n, nmax) not in Rcache:
                Rcache[(n, nmax)] = ker.restriction(n, nmax)
            out[l] = (Rcache[(n, nmax)] @ Gt[:, :, l]).T
        return out

    # m = 1 data: g_{k,1} = sign chi_k u^i on the transfer mesh (eq. criterion_int1), slow transform.
    G = {}
    for k in range(P):
        g = sig["sign"] * S.chi[k][:, None] * incident_field(sig, S.X[k], tg.t)
        if keep_g:
            res.g[(1, k)] = g
        for l, v in restrict(k, tg.forward(g)).items():
            G[(k, l)] = v

    cross_cache = {}

    def cross_block(l, k, j):
        key = (l, k, j)
        if key in cross_cache:
            return cross_cache[key]
        rows, ts, near = S.blocks[(k, j)]
        E = ker.cross_rows(S.arcs[j], int(S.Ntab[j, l]), tg.omega[l], S.X[k][rows], ts, near)
        if cache_cross:
            cross_cache[key] = E
        return E

    def obs_block(l, j):
        key = (l, -1, j)
        if key in cross_cache:
            return cross_cache[key]
        n_o = S.obs.shape[0]
        E = ker.cross_rows(S.arcs[j], int(S.Ntab[j, l]), tg.omega[l], S.obs,
                           np.zeros(n_o), np.zeros(n_o, dtype=bool))
        if cache_cross:
            cross_cache[key] = E
        return E

    Vobs = np.zeros((S.obs.shape[0], Q, L), dtype=np.complex128)
    for m in range(1, M + 1):
        phi = {}
        for j in range(P):
            for l in own:
                phi[(j, l)] = scipy.linalg.lu_solve(lu[(j, l)], G[(j, l)].T).T     # (Q, N)
                if j in keep:
                    res.phi[(m, j, l)] = phi[(j, l)]
                if keep_G:
                    res.G[(m, j, l)] = G[(j, l)]
        # Potentials of every arc at the other arcs' transfer nodes (masked per eq. vtilde) and at
        # the observation points (output sum of eq. mult-scatt-int, in the frequency domain).
        Wk = [np.zeros((int(S.Nmax[k]), Q, L), dtype=np.complex128) for k in range(P)]
        for l in own:
            for j in range(P):
                Vobs[:, :, l] += obs_block(l, j) @ phi[(j, l)].T
                for k in range(P):
                    if k == j:
                        continue
                    rows = S.blocks[(k, j)][0]
                    if rows.size:
                        Wk[k][rows, :, l] += cross_block(l, k, j) @ phi[(j, l)].T
        if m == M:
            break
        # g_{k,m+1} = -chi_k sum_j vtilde (eq. criterion_int2), back to the frequency domain.
        G = {}
        for k in range(P):
            w = total(tg.inverse(Wk[k]))
            g = -S.chi[k][:, None] * w
            if keep_g:
                res.g[(m + 1, k)] = g
            for l, v in restrict(k, tg.forward(g)).items():
                G[(k, l)] = v
    res.Vobs = Vobs
    tout = o["tout0"] + o["dtout"] * np.arange(o["n_tout"])
    res.traces = total(tg.inverse_at(Vobs, tout))
    return res
