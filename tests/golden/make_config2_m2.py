"""Write config2_m2_arc4.json: densities phi_{4,2,1}(omega_l) of full-size config 2 at sampled
frequencies, computed by the CPU oracle alone (m = 1 densities of every arc and frequency, the
cross-arc field on arc 4's transfer mesh, its synthesis, windowed forward transform, restriction and
solve: Algorithm 1's second step restricted to one receiving arc).

Usage: python tests/golden/make_config2_m2.py   (about two minutes on 8 cores)
"""
import json
import os
import sys

import numpy as np
import scipy.linalg

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402
from oracle import kernels as ker  # noqa: E402
from oracle.fthms import Setup  # noqa: E402
from oracle.transforms import incident_field  # noqa: E402

ARC = 4
SAMPLES = [1, 150, 200, 256, 300, 400, 512, 700, 1024]


def main():
    problem = wl.config2(M=2)
    S = Setup(problem)
    tg = S.grid
    sig = problem["signal"]
    L, P = tg.L, S.P

    def restrict(k, Gt, l):
        return ker.restriction(int(S.Ntab[k, l]), int(S.Nmax[k])) @ Gt[:, 0, l]

    # m = 1 densities of every arc and frequency
    phi1 = {}
    for j in range(P):
        g = sig["sign"] * S.chi[j][:, None] * incident_field(sig, S.X[j], tg.t)
        Gt = tg.forward(g)
        for l in range(1, L):
            A = ker.self_matrix(S.arcs[j], int(S.Ntab[j, l]), tg.omega[l])
            phi1[(j, l)] = scipy.linalg.solve(A, restrict(j, Gt, l))
    # cross field of every other arc at arc 4's transfer nodes (eq. vtilde masking), all frequencies
    W = np.zeros((int(S.Nmax[ARC]), 1, L), dtype=np.complex128)
    for j in range(P):
        if j == ARC:
            continue
        rows, ts, near = S.blocks[(ARC, j)]
        if rows.size == 0:
            continue
        for l in range(1, L):
            E = ker.cross_rows(S.arcs[j], int(S.Ntab[j, l]), tg.omega[l], S.X[ARC][rows], ts, near)
            W[rows, 0, l] += E @ phi1[(j, l)]
    g2 = -S.chi[ARC][:, None] * tg.inverse(W)
    Gt2 = tg.forward(g2)
    out = {"workload": "config2 (seed 2), M = 2", "arc": ARC, "m": 2, "q": 0, "samples": {}}
    for l in SAMPLES:
        A = ker.self_matrix(S.arcs[ARC], int(S.Ntab[ARC, l]), tg.omega[l])
        phi2 = scipy.linalg.solve(A, restrict(ARC, Gt2, l))
        out["samples"][str(l)] = {"re": phi2.real.tolist(), "im": phi2.imag.tolist()}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "config2_m2_arc4.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print("wrote", path)


if __name__ == "__main__":
    main()
