"""Multi-rank paths on the CPU (gloo, world_size 2): the bench's replica aggregation, and the frequency
partition of one job (Section 3: a step's per-frequency sub-problems are independent; its one coupling is
the omega -> t synthesis, a sum over frequencies that the ranks all-reduce once per step)."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

import workloads as wl


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _init(rank, port):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2")
    dist.init_process_group("gloo", rank=rank, world_size=2)
    return dist


def _aggregation_worker(rank, port, out):
    dist = _init(rank, port)
    import bench
    ms = bench.max_over_ranks(10.0 + rank, device="cpu")
    out[rank] = (ms, bench.job_value(2, 1000, ms))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_aggregation_worker, args=(port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 11.0               # slowest rank's time
    assert abs(res[0][1] - 2 * 1000 / 0.011) < 1e-6     # total solves of both replicas / that time


def _problem():
    return wl.random_small(5, n_curves=2, n_arcs_per_curve=2, Q=2, L=33, M=3)


def _partition_worker(rank, port, out):
    import torch
    dist = _init(rank, port)
    from oracle import run_oracle

    def allreduce(a):
        t = torch.from_numpy(np.ascontiguousarray(a))
        dist.all_reduce(t)
        return t.numpy()

    res = run_oracle(_problem(), omega_part=(rank, 2), allreduce=allreduce)
    out[rank] = ({k: v for k, v in res.phi.items()}, res.traces)
    dist.destroy_process_group()


def test_frequency_partition_matches_one_rank():
    """Two gloo ranks, each with half of the solved frequencies and one all-reduce of the time samples per
    step (and of the traces), reproduce the one-rank job: every density and the traces within 1e-13."""
    from oracle import run_oracle
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_partition_worker, args=(port, out), nprocs=2, join=True)
        res = dict(out)
    ref = run_oracle(_problem())
    L = _problem()["options"]["L"]
    owned = {}
    for rank in (0, 1):
        phi, traces = res[rank]
        assert np.max(np.abs(traces - ref.traces)) < 1e-13 * np.max(np.abs(ref.traces))
        for (m, j, l), v in phi.items():
            owned.setdefault((m, j, l), rank)
            scale = np.max(np.abs(ref.phi[(m, j, l)])) + 1e-300
            assert np.max(np.abs(v - ref.phi[(m, j, l)])) < 1e-13 * max(scale, 1e-12), (m, j, l)
    assert set(owned) == set(ref.phi)                    # every (m, arc, omega) solved by exactly one rank
    assert {l for (_, _, l), r in owned.items() if r == 0} == set(range(1, 1 + (L - 1) // 2))


def test_partition_plans_on_the_host():
    """The library's planning of a partitioned job (no GPU): each rank holds its share of the systems and of
    the device memory, the shares add up to the whole job's systems, and bad ranks are rejected."""
    import copy

    import pytest

    from paper_2507_05725_gb300 import fthms as F
    p = wl.config2_reduced()
    whole_b, whole_n = F.fthms_plan_info(F.Marshalled(p, keep_densities=False))
    parts = []
    for r in range(3):
        q = copy.deepcopy(p)
        q["options"].update(omega_rank=r, omega_ranks=3)
        parts.append(F.fthms_plan_info(F.Marshalled(q, keep_densities=False)))
    assert sum(n for _, n in parts) == whole_n
    assert all(b < 0.5 * whole_b for b, _ in parts)
    bad = copy.deepcopy(p)
    bad["options"].update(omega_rank=3, omega_ranks=3)
    with pytest.raises(F.FthmsError) as e:
        F.fthms_plan_info(F.Marshalled(bad))
    assert e.value.status == F.FTHMS_EINVAL
