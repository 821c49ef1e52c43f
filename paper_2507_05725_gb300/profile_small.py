"""A small 4-obstacle job for ncu captures: config 2's geometry, signal and node rule on 512 frequencies of
[0, 30] with M = 4 (about 1.8 GB on the device, cross matrices 1.4 GB, above L2), run once in the plain FP64
form and once in the mixed form.  Prints each job's statistics as one JSON line.

Usage: python -m paper_2507_05725_gb300.profile_small
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
    problem = wl.config2(L=513, W=30.0, M=4)
    ctx = F.fthms_create(0, 0, None)
    for precision in (0, 1):
        job = F.Job(ctx, problem, keep_densities=False, precision=precision)
        job.run().wait()
        print(json.dumps(job.stats()))
        job.release()
    F.fthms_destroy(ctx)


if __name__ == "__main__":
    main()
