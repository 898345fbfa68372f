"""The multi-process (N > 1) bench plumbing on CPU: world-size-2 gloo process
groups on 127.0.0.1.  The path has no exchange step (replicas only), so what
crosses ranks is the job's time: the maximum over the ranks."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, values, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, rk, local = bench.dist_info()
    got = bench.max_over_ranks(values[rank], dist, torch.device("cpu"))
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, ws, rk, local, got))


def test_max_over_ranks_gloo():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    values = [0.0842, 0.0917]
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, values, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, (r, ws, rk, local, got) in enumerate(res):
        assert (r, ws, rk, local) == (rank, 2, rank, rank)
        assert got == max(values)


def test_max_over_ranks_without_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(0.5, None, None) == 0.5


def test_reference_arm_rank_nonzero_does_no_work(monkeypatch, capsys):
    """Under torchrun only rank 0 runs and prints the reference arm."""
    sys.path.insert(0, ROOT)
    import argparse

    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.run_reference(argparse.Namespace(gpus=2, steps=1, warmup=1)) is None
    assert capsys.readouterr().out == ""
