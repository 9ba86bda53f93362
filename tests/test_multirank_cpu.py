"""The multi-rank logic of bench.py on the CPU: two gloo ranks, one process
each, take the slowest rank's step time and report whole-job throughput, as
``bench.py --gpus 2`` does over NCCL (replicas: one independent matrix per
rank, no collective on the data path)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank                      # rank 1 is the slow one
    got = bench.max_over_ranks(ms, "cpu", world)
    val = bench.job_throughput(world, 18_874_368_000, got)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got, val))


def test_two_gloo_ranks_report_the_slowest_step():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in res] == [0, 1]
    for _, got, val in res:
        assert got == 15.0
        assert val == pytest.approx(2 * 18.874368 / 0.015)


def test_single_rank_is_the_identity():
    import bench
    assert bench.max_over_ranks(12.5, "cpu", 1) == 12.5
    assert bench.job_throughput(1, 4e9, 2.0) == pytest.approx(2000.0)
