"""The N > 1 path of bench.py ("replicas only": one graph per GPU, no
collective on the data path): two gloo ranks on the CPU check that the job's
step time is the slowest rank's and the value counts every rank's edges."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r is slower the higher its rank; each traverses 3e9 edges per step
    out = bench.combine_replicas(10.0 + rank, 20.0 + 2 * rank, 3_000_000_000, world, device="cpu")
    q.put((rank, out))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_combine_replicas_gloo(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        step_ms, e2e_ms, value, e2e_value = res[r]
        assert step_ms == 10.0 + (world - 1) and e2e_ms == 20.0 + 2 * (world - 1)
        assert value == pytest.approx(world * 3.0 / (step_ms * 1e-3))
        assert e2e_value == pytest.approx(world * 3.0 / (e2e_ms * 1e-3))


def test_combine_replicas_single():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.combine_replicas(5.0, 8.0, 1_000_000_000, 1) == (5.0, 8.0, 200.0, 125.0)
