"""The multi-process path of bench.py on the CPU: N independent replicas, one
per rank, with no data-path collective.  World size 2 over gloo checks the
whole-job totals (Newton iterations summed, the slowest rank's time) and that
only rank 0 of the reference arm does any work."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        its, ms = bench.replica_totals(3 + rank, 10.0 * (rank + 1), world, torch.device("cpu"))
        out[rank] = (its, ms)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replica_totals_over_two_gloo_ranks():
    port = free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    # each rank sees the same totals: 3 + 4 iterations, the slower rank's 20 ms
    assert res == {0: (7, 20.0), 1: (7, 20.0)}
    its, ms = res[0]
    assert its / (ms * 1e-3) == pytest.approx(350.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    assert bench.main() == 0
    assert capsys.readouterr().out == ""
