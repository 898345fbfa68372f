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


def test_reference_arm_json_line(monkeypatch, capsys):
    """`bench.py --impl reference` (the FP64 oracle timed on the host cores)
    prints one JSON line with the benchmark's keys, its own e2e figure and a
    cpu_baseline describing the run; it needs no GPU.  Run here on the small
    exact 20^3 workload (the full 400^3 solve takes minutes on these cores)."""
    import argparse
    import json

    import bench

    monkeypatch.setenv("OMP_NUM_THREADS", "4")
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    monkeypatch.setattr(bench, "WORKLOAD", "exact20")
    bench.run_reference(argparse.Namespace(gpus=1, steps=2, warmup=1))
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["n_gpus"] == 1 and line["steps"] == 2 and line["warmup"] == 1
    assert line["value"] > 0 and line["higher_is_better"] is False
    assert abs(line["ms_per_step"] - 1e3 * line["value"]) <= 1e-9 * line["ms_per_step"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 4 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    # the reference arm reports the benchmark's own config (same keys as the GPU arm's line)
    assert line["config"] == dict(bench.CONFIG, parallelism="replicas x1")
