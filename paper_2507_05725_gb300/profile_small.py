"""Small jobs for ncu captures.  Prints each job's statistics as one JSON line.

  python -m paper_2507_05725_gb300.profile_small [c2|c4|c4-launches]

c2: the 4-obstacle configuration's geometry, signal and node rule on 512 frequencies of [0, 30] with M = 4
    (about 1.8 GB on the device, cross matrices 1.4 GB, above L2), in the plain FP64 and the mixed form.
c4: the mixed-precision configuration (6 arcs of 5 ellipses) at N = 1024 on 64 frequencies of the same grid
    spacing (omega up to 25), M = 2, in the FP64-kept form with tensor-core LU (about 10 GB on the device:
    every kernel's data are far above L2); the launches of interest are k_lu_big_update, k_lu_big_panel,
    k_mresid64, k_msolve and k_cross_otf_df.
c4-launches: one full-size job of the mixed-precision configuration at N = 512 (1023 frequencies, M = 8,
    the bench's headline workload) in the FP64-kept form with the tensor-core LU, for a launch list.
"""
import json
import os
import sys


def main():
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import workloads as wl
    from paper_2507_05725_gb300 import fthms as F
    torch.cuda.set_device(0)
    which = sys.argv[1] if len(sys.argv) > 1 else "c2"
    ctx = F.fthms_create(0, 0, None)
    if which == "c2":
        runs = [(wl.config2(L=513, W=30.0, M=4), 0), (wl.config2(L=513, W=30.0, M=4), 1)]
    elif which == "c4":
        runs = [(wl.config4(1024, L=65, W=400.0 * 64 / 1023, M=2), 2)]
    else:
        runs = [(wl.config4(512), 2)]
    for problem, precision in runs:
        job = F.Job(ctx, problem, keep_densities=False, precision=precision)
        if which.startswith("c4"):
            F.fthms_autotune(job.req, 1)            # the LU path and launch shapes of the bench
        job.run().wait()
        print(json.dumps(job.stats()))
        job.release()
    F.fthms_destroy(ctx)


if __name__ == "__main__":
    main()
