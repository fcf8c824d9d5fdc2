"""Replica mode of bench.py on two gloo ranks (CPU): each rank runs its own
crystal and photon stream, the job's time is the slowest rank's, the job's
rate counts every rank's ions, and only rank 0 runs the reference arm."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, value = bench.job_rate(10.0 * (rank + 1), world, 100, 5, dist, "cpu")
        out.put((rank, t, value, bench.replica_seeds(rank)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_job_rate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, v0, s0), (r1, t1, v1, s1) = res
    assert t0 == t1 == 20.0                       # max over ranks
    assert v0 == v1 == 2 * 100 * 5 / 0.020        # both ranks' ions / slowest time
    assert s0 != s1 and s0[0] != s1[0] and s0[1] != s1[1]   # independent replicas


def test_reference_arm_runs_on_rank_zero_only(capsys):
    class Args:
        steps, warmup, p = 1, 3, 12
    assert bench.reference_arm(Args, 1) == 0
    assert capsys.readouterr().out == ""
