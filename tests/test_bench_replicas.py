"""Host logic of the N-replica benchmark, on CPU with a world-size-2 gloo group:
the timing is the maximum over ranks and the value counts every rank's work;
the reference arm runs on rank 0 only."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_max, value = bench.aggregate(10.0 * (rank + 1), npts=1000, steps=2, ws=world, device="cpu")
    out[rank] = (t_max, value)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_gloo():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        t_max, value = out[r]
        assert t_max == 20.0
        assert abs(value - world * 1000 * 5 * 2 / 0.020 / 1e9) < 1e-15


def test_reference_arm_only_on_rank0(monkeypatch, capsys):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup, gpus = 1, 0, 2
    assert bench.run_reference(A()) == 0
    assert capsys.readouterr().out == ""
