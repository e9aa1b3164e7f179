"""Host logic of the multi-GPU bench path (replicas, weak scaling) with two
gloo ranks on the CPU: the timed region's maximum over ranks and the
whole-job value."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dist.barrier()
    ms = 10.0 + 2.5 * rank  # the second replica is slower
    m = bench.max_over_ranks(ms, dist, "cpu")
    out[rank] = (m, bench.whole_job_value(world, 128 * 4096, 5, m))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    for m, v in res.values():
        assert m == 12.5
        assert v == world * 128 * 4096 * 5 / (12.5e-3)
