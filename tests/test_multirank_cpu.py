"""The N > 1 path of bench.py on CPU: two gloo ranks, replica aggregation (total work of all ranks over the
slowest rank's time, max taken across ranks) and the barrier."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp        # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    el = 100.0 + 50.0 * rank                       # rank 1 is the slower replica
    value, el_max = bench.aggregate_replicas(el, n=1000, steps=10, dist=dist, device="cpu")
    dist.barrier()
    out[rank] = (value, el_max)
    dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert set(out.keys()) == {0, 1}
    for r in range(world):
        value, el_max = out[r]
        assert el_max == 150.0
        assert abs(value - world * 1000 * 10 / 0.150) < 1e-6
