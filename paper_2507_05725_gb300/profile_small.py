"""Small jobs for ncu captures.  Prints each job's statistics as one JSON line.

  python -m paper_2507_05725_gb300.profile_small [c2|c3s|c4|c4s|c4r|c4-launches]

c2: the 4-obstacle configuration's geometry, signal and node rule on 512 frequencies of [0, 30] with M = 4
    (about 1.8 GB on the device, cross matrices 1.4 GB, above L2), in the plain FP64 and the mixed form.
c3s: the 12-arc cavity (cross rows evaluated every step), M = 2, precision 1, as rank 16 of a 32-way frequency
    partition (its 64 frequencies at omega ~ 100, the all-reduce a no-op): the launch of interest is
    k_cross_otf_df.
c4: the mixed-precision configuration (6 arcs of 5 ellipses) at N = 1024 on 64 frequencies of the same grid
    spacing (omega up to 25), M = 2, in the FP64-kept form with tensor-core LU (about 10 GB on the device:
    every kernel's data are far above L2); the launches of interest are k_lu_big_update, k_lu_big_panel,
    k_mresid64, k_msolve and k_cross_otf_df.
c4s: the mixed-precision configuration at N = 512 on 128 frequencies of the same grid spacing (omega up to
    50), M = 2, cross rows evaluated every step, in the FP64-kept form with the bench's tuned shapes
    (tensor-core LU at N = 512): 768 systems, about 5 GB on the device; the launches of interest are k_lu_big_update, k_lu_big_panel,
    k_msolve, k_mresid64 and k_cross_otf_df.
c4r: the same at N = 512 on 16 frequencies (omega up to 6.3), M = 2, stored cross rows (1.75 GB of them, far
    above L2), FP64-kept form with the tuned shapes: the launch of interest is k_cross_rows_df.
c4-launches: one full-size job of the mixed-precision configuration at N = 512 (1023 frequencies, M = 8,
    the bench's headline workload) in the FP64-kept form with the bench's tuned shapes and the tensor-core
    LU, for a launch list.
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
    elif which == "c3s":
        p = wl.config3(M=2)
        p["options"].update(omega_rank=16, omega_ranks=32)
        runs = [(p, 1)]
    elif which == "c4r":
        runs = [(wl.config4(512, L=17, W=400.0 * 16 / 1023, M=2), 2)]
    elif which == "c4s":
        p = wl.config4(512, L=129, W=400.0 * 128 / 1023, M=2)
        p["options"]["cross_mode"] = 1
        runs = [(p, 2)]
    else:
        runs = [(wl.config4(512), 2)]
    for problem, precision in runs:
        job = F.Job(ctx, problem, keep_densities=False, precision=precision)
        if problem["options"].get("omega_ranks", 0) > 1:
            job.set_allreduce(lambda buf, n, stream: None)   # one rank alone
        if which.startswith("c4"):
            # the bench's tuned choices for this form (tensor-core LU from N = 256), applied without timing
            F.fthms_set_shapes(job.req, [1, 256, 512, 256, 256])
        job.run().wait()
        print(json.dumps(job.stats()))
        job.release()
    F.fthms_destroy(ctx)


if __name__ == "__main__":
    main()
