"""The N > 1 path of bench.py on CPU: N independent replicas, whole-job value =
cell-updates of all ranks over the slowest rank's time (max over ranks, sum of
work), over a world-size-2 gloo process group; and the reference arm's rule that
only rank 0 runs and prints."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [2.0, 5.0][rank]          # rank 1 is the slow one
        cells = [1.0e6, 3.0e6][rank]   # replicas need not do equal work
        dist.barrier()
        ms_max, value = bench.aggregate_ranks(ms, cells, world, torch.device("cpu"))
        q.put((rank, ms_max, value))
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_gloo_world2():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms_max, value in got:
        assert ms_max == 5.0
        assert value == pytest.approx((1.0e6 + 3.0e6) / 5.0e-3)


def test_single_rank_aggregation_needs_no_group():
    import torch

    sys.path.insert(0, ROOT)
    import bench

    ms_max, value = bench.aggregate_ranks(4.0, 2.0e6, 1, torch.device("cpu"))
    assert ms_max == 4.0 and value == pytest.approx(2.0e6 / 4.0e-3)


def test_reference_arm_runs_on_rank_0_only(monkeypatch, capsys):
    """Under torchrun the reference arm (the oracle on the host) runs on rank 0
    alone; the other ranks return at once and print nothing."""
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.run_reference(None) is None
    assert capsys.readouterr().out == ""
