"""The multi-GPU path shards particles with no data-path collective; its
host-side aggregation (whole-job units over the slowest rank's time) is
checked here with two gloo ranks on the CPU."""
import os

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    units = [1.0e9, 3.0e9][rank]
    ms = [10.0, 20.0][rank]
    value, t_max = bench.job_rate(dist, units, ms, device="cpu")
    dist.barrier()
    out[rank] = (value, t_max)
    dist.destroy_process_group()


def test_two_ranks_aggregate_to_the_whole_job():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        value, t_max = out[r]
        assert t_max == 20.0                      # slowest rank
        assert value == pytest.approx(4.0e9 / 0.020)   # all units / slowest time
