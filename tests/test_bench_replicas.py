"""Replica bookkeeping of bench.py at world size 2 over gloo on CPU (the multi-GPU form runs
independent replicas: one barrier, the slowest rank's time, every rank's units)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [1200.0, 1500.0][rank]                       # rank 1 is the slow one
    mx = bench.world_max(ms, world, "cpu")
    val = bench.replica_value(4444, mx, world)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"max_ms": mx, "value": val}, f)


def test_world_max_and_value_gloo(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        d = json.load(open(tmp_path / f"r{r}.json"))
        assert d["max_ms"] == 1500.0
        assert d["value"] == pytest.approx(2 * 4444 / 1.5)


def test_single_rank_is_identity():
    import bench
    assert bench.world_max(3.25, 1, "cpu") == 3.25
    assert bench.replica_value(100, 500.0, 1) == pytest.approx(200.0)


def test_reference_arm_nonzero_rank_exits_without_work(tmp_path):
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "3",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
