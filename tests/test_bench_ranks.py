"""The benchmark's multi-rank host logic on the CPU (gloo, world size 2).

With several GPUs every rank solves its own independent instance of the
workload (replicas, no collective on the data path); the only collective is
the reduction of the per-rank times to the slowest rank.  These tests run
that reduction over a two-rank gloo group, and the reference arm under
torchrun, where rank 0 alone times the oracle and prints the line."""
import json
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, per_rank, expected):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks(per_rank[rank], dist)
        assert got == expected, (rank, got, expected)
        # one rank alone: the values pass through unchanged
        assert bench.max_over_ranks(per_rank[rank]) == per_rank[rank]
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    per_rank = [[57.0, 39.5, 120.25, 0.0], [58.5, 38.0, 120.5, 1e-3]]
    expected = [max(a, b) for a, b in zip(*per_rank)]
    mp.start_processes(_rank_main, args=(2, free_port(), per_rank, expected), nprocs=2, join=True,
                       start_method="spawn")


def test_reference_arm_under_torchrun_prints_once_from_rank_0():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={free_port()}", os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["steps"] == 1
    assert d["value"] > 0 and d["e2e"]["value"] == d["value"]
