"""The replica path of bench.py on CPU: two gloo ranks aggregate their step
times (max) and Gaussian counts (sum), and draw different inputs."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, value = bench.aggregate_ranks(10.0 + 5.0 * rank, 1000 * (rank + 1), world, device="cpu")
    X, _, _, _ = bench.workload(64, 16, 2, seed_offset=100 * rank, device="cpu")
    out[rank] = (ms, value, float(np.asarray(X)[0, 0]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_aggregate_with_gloo():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms, value, _ = res[r]
        assert ms == 15.0  # the slowest rank
        assert abs(value - 3000 / 15e-3) < 1e-6 * value  # every rank's Gaussians
    assert res[0][2] != res[1][2]  # each replica draws its own signals


def test_single_process_aggregate():
    import bench
    ms, value = bench.aggregate_ranks(20.0, 3_000_000, 1)
    assert ms == 20.0 and abs(value - 1.5e8) < 1e-3
