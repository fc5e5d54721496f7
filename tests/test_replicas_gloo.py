"""The N > 1 path of bench.py (replicas: one independent front pipeline per
rank, no data-path collective) on the CPU with two gloo ranks: the process
group comes up from the torchrun environment, the barrier holds, the step time
is the maximum over ranks and the value sums the cells of every rank."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    ws, r, local = bench.dist()
    assert (ws, r, local) == (world, rank, rank)
    bench.barrier(ws)
    t_ms = 10.0 * (rank + 1)            # rank 1 is the slower replica
    cells = 1000 * (rank + 1)           # each replica processes its own fronts
    tmax = bench.allmax(ws, t_ms)
    total = bench.allsum(ws, cells * 5)
    out[rank] = (tmax, total, total / (tmax * 1e-3))
    import torch.distributed as td
    td.destroy_process_group()


def test_two_gloo_replicas():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        tmax, total, value = res[rank]
        assert tmax == 20.0
        assert total == 5 * (1000 + 2000)
        assert abs(value - 15000 / 0.02) < 1e-6


def test_reference_arm_other_ranks_exit(monkeypatch):
    """Under torchrun only rank 0 runs the reference arm; the others return."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class A:
        steps, warmup = 1, 0
    # rank 1 of a one-process "world" skips the group and returns before any work
    assert bench.run_reference(A()) is None
