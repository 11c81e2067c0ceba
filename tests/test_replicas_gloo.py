"""The multi-GPU path of bench.py is replicas only (one independent discharge
per rank, no data-path collective).  Its whole-job aggregation -- the slowest
rank's time, the sum of the ranks' particle-steps -- runs here on two gloo
ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_local = [0.50, 0.75][rank]
    ps_local = [1000, 3000][rank]
    t, ps = bench.aggregate_replicas(t_local, ps_local, world, "cpu")
    out[rank] = (t, ps)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_max_time_and_sum_work():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        t, ps = out[r]
        assert t == pytest.approx(0.75) and ps == pytest.approx(4000.0)


def test_single_rank_is_identity():
    import bench
    assert bench.aggregate_replicas(0.3, 12.0, 1, "cpu") == (0.3, 12.0)
