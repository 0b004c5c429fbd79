"""The multi-GPU path of bench.py is replicas only: each rank solves its own
workload, the ranks meet at a barrier, and the job time is the maximum over
ranks.  Checked here with two gloo ranks on the CPU (no GPU, no data-path
collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    assert (r, w, local) == (rank, world, rank)
    dist.barrier()
    t = bench.max_over_ranks(times[rank], world, torch.device("cpu"))
    out[rank] = t
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    times = [1.25, 2.5]
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == 2.5


def test_whole_job_value_counts_every_rank():
    import bench

    # two replicas of 1e6 cells x 5000 steps in 2.5 s (max over ranks)
    assert bench.job_value(1e6 * 5000, 1, 2.5, 2) == pytest.approx(2 * 1e6 * 5000 / 2.5 / 1e6)
