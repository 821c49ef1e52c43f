"""Write config3_m2.json: second-step densities phi_{k,2,q}(omega_l) of the full-size 12-arc star
cavity (the third configuration: N from 32 to 760, 2048 solved frequencies on (0, 200], Q = 4 windows,
point-source boundary data) at two receiving arcs and sampled frequencies, computed by the CPU oracle
alone.

Algorithm 1's second step restricted to two receiving arcs k: the m = 1 data of every arc (eq.
criterion_int1: sign chi_j u^i on its transfer mesh, windowed slow transform of eq. Fourierk,
restriction to the solve nodes), every m = 1 density (the self matrix of every (arc, omega) and its LU
solve), the cross field of every other arc on k's transfer mesh (eq. vtilde masking, near and far rows),
its recentred synthesis (eq. TDsol), g_{k,2} = -chi_k (...) (eq. criterion_int2), the windowed slow
transform and restriction, and the solve at the sampled frequencies.  Every arithmetic step is a call of
`oracle/`; this script only distributes the independent pieces over worker processes (spawned, CPU only).

Usage: python tests/golden/make_config3_m2.py [--workers 8]   (tens of minutes on 8 cores)
"""
import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np
import scipy.linalg

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

RECEIVERS = [0, 6]
SAMPLES = [1, 307, 614, 1024, 1536, 2048 - 1]
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "config3_m2.json")

_S = None


def _setup():
    global _S
    if _S is None:
        import workloads as wl
        from oracle.fthms import Setup
        _S = Setup(wl.config3(M=2))
    return _S


def _incident_chunk(args):
    """sign chi_k u^i(x, t_n) at a chunk of the active transfer nodes of arc k (eq. criterion_int1)."""
    k, nodes = args
    from oracle.transforms import incident_field
    S = _setup()
    sig = S.problem["signal"]
    u = incident_field(sig, S.X[k][nodes], S.grid.t)
    return k, nodes, sig["sign"] * S.chi[k][nodes][:, None] * u


def _solve_chunk(args):
    """m = 1 densities of arc j at frequencies ls: restriction of the transfer-mesh spectra, self matrix,
    LU solve (Algorithm 1, BIE solve)."""
    j, ls, Gt = args
    from oracle import kernels as ker
    S = _setup()
    out = {}
    for l in ls:
        n = int(S.Ntab[j, l])
        G = (ker.restriction(n, int(S.Nmax[j])) @ Gt[:, :, l - ls[0]]).T          # (Q, n)
        A = ker.self_matrix(S.arcs[j], n, S.grid.omega[l])
        out[l] = scipy.linalg.lu_solve(scipy.linalg.lu_factor(A), G.T).T
    return j, out


def _cross_chunk(args):
    """Cross fields sum_{j != k} E_{l,k,j} phi_{j,1}(omega_l) on arc k's transfer nodes (eqs.
    FDsolk-interior, vtilde) at frequencies ls."""
    k, ls, phis = args
    from oracle import kernels as ker
    S = _setup()
    Q = S.grid.Q
    W = np.zeros((int(S.Nmax[k]), Q, len(ls)), dtype=np.complex128)
    for j in range(S.P):
        if j == k:
            continue
        rows, ts, near = S.blocks[(k, j)]
        if rows.size == 0:
            continue
        for b, l in enumerate(ls):
            E = ker.cross_rows(S.arcs[j], int(S.Ntab[j, l]), S.grid.omega[l], S.X[k][rows], ts, near)
            W[rows, :, b] += E @ phis[(j, l)].T
    return k, ls, W


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    S = _setup()
    tg = S.grid
    L, P, Q = tg.L, S.P, tg.Q
    t0 = time.time()
    ctx = mp.get_context("spawn")
    with ctx.Pool(args.workers, initializer=_setup) as pool:
        # m = 1 data on every arc's transfer mesh
        tasks = []
        for k in range(P):
            act = np.nonzero(S.chi[k] > 0.0)[0]
            for c in range(0, act.size, 16):
                tasks.append((k, act[c:c + 16]))
        g = [np.zeros((int(S.Nmax[k]), tg.NT)) for k in range(P)]
        for k, nodes, v in pool.imap_unordered(_incident_chunk, tasks):
            g[k][nodes] = v
        print(f"incident field: {time.time() - t0:.0f} s", flush=True)
        # m = 1 densities of every (arc, omega)
        tasks = []
        for j in range(P):
            Gt = tg.forward(g[j])                                   # [Nmax, Q, L]
            for c in range(1, L, 32):
                ls = list(range(c, min(c + 32, L)))
                tasks.append((j, ls, Gt[:, :, ls[0]:ls[-1] + 1].copy()))
        phi1 = {}
        for j, out in pool.imap_unordered(_solve_chunk, tasks):
            for l, v in out.items():
                phi1[(j, l)] = v
        print(f"m = 1 densities: {time.time() - t0:.0f} s", flush=True)
        # cross fields on the receiving arcs' transfer meshes, all frequencies
        W = {k: np.zeros((int(S.Nmax[k]), Q, L), dtype=np.complex128) for k in RECEIVERS}
        tasks = []
        for k in RECEIVERS:
            for c in range(1, L, 16):
                ls = list(range(c, min(c + 16, L)))
                need = {(j, l): phi1[(j, l)] for j in range(P) if j != k for l in ls}
                tasks.append((k, ls, need))
        for k, ls, Wc in pool.imap_unordered(_cross_chunk, tasks):
            W[k][:, :, ls[0]:ls[-1] + 1] = Wc
        print(f"cross fields: {time.time() - t0:.0f} s", flush=True)
    from oracle import kernels as ker
    out = {"workload": "config3 (seed 3), M = 2: 12-arc star cavity, N 32..760, L = 2049 on [0, 200], Q = 4",
           "m": 2, "receivers": RECEIVERS, "samples": {}}
    for k in RECEIVERS:
        g2 = -S.chi[k][:, None] * tg.inverse(W[k])                  # eq. criterion_int2 on the transfer mesh
        Gt2 = tg.forward(g2)
        for l in SAMPLES:
            n = int(S.Ntab[k, l])
            G2 = (ker.restriction(n, int(S.Nmax[k])) @ Gt2[:, :, l]).T
            A = ker.self_matrix(S.arcs[k], n, tg.omega[l])
            phi2 = scipy.linalg.lu_solve(scipy.linalg.lu_factor(A), G2.T).T     # (Q, n)
            out["samples"][f"{k}:{l}"] = {"N": n, "re": phi2.real.tolist(), "im": phi2.imag.tolist()}
    with open(OUT, "w") as f:
        json.dump(out, f)
    print(f"wrote {OUT} in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
