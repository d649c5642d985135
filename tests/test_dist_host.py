"""The multi-process path of bench.py on CPU (gloo, world size 2): the max-over-ranks
timing, the weak-scaling aggregate, and the reference arm's rank > 0 exit."""

import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, out_path):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    d = bench.dist_init(ws, "gloo")
    local_time = 1.0 + rank  # rank 1 is the slow one
    bench.barrier(d, ws)
    t_max = bench.max_over_ranks(d, ws, local_time, torch.device("cpu"))
    value = bench.weak_scaling_value(ws, 1000, 10, t_max)
    with open(f"{out_path}.{rank}", "w") as f:
        json.dump({"t_max": t_max, "value": value}, f)
    dist.destroy_process_group()


def test_gloo_two_ranks_max_and_weak_scaling(tmp_path):
    port = _free_port()
    out = str(tmp_path / "r")
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    res = [json.load(open(f"{out}.{r}")) for r in range(2)]
    for r in res:
        assert r["t_max"] == 2.0  # the slowest rank's time, seen by every rank
        assert r["value"] == 2 * 1000 * 10 / 2.0


def test_reference_arm_rank1_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "3", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
