"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2).

The product path has no exchange step: with N ranks every rank runs its own
replica of the workload, the job time is the maximum over ranks and the
whole-job rate counts every rank's work.  These tests run that logic in two
gloo processes, and check that the reference arm does its work on rank 0
only.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as tmp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, loc = bench.dist_info()
        ms = bench.max_over_ranks(1.0 + 2.5 * rank, torch.device("cpu"))   # rank 1 is slower
        val = bench.replica_value(w, 2.0 * 64 ** 3, ms)
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as fh:
            json.dump({"dist": [w, r, loc], "ms": ms, "value": val}, fh)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_replica_value(tmp_path):
    world = 2
    tmp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    for r, d in enumerate(res):
        assert d["dist"] == [world, r, r]
        assert d["ms"] == pytest.approx(3.5)                      # the slower rank's time
        assert d["value"] == pytest.approx(world * 2.0 * 64 ** 3 / 3.5e-3)


def test_single_process_helpers():
    sys.path.insert(0, ROOT)
    import bench
    import torch
    assert bench.max_over_ranks(1.25, torch.device("cpu")) == 1.25
    assert bench.replica_value(1, 2e9, 1.0) == pytest.approx(2e12)


def test_reference_arm_nonzero_rank_does_no_work():
    """Under torchrun only rank 0 times the oracle; other ranks exit 0 silently."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--gpus", "2", "--steps", "1", "--warmup", "3"],
                         env=env, cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == ""
