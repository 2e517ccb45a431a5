"""Multi-rank bookkeeping of the benchmark, run as two gloo ranks on the CPU.

Replicas exchange nothing on the data path; what crosses ranks is the barrier,
the maximum of the per-rank times and the whole-job rate derived from it.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      LOCAL_RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    from paper_1410_3464_gb300 import replicas
    ws, r, local = replicas.env()
    replicas.init(ws)
    replicas.barrier(ws)
    my_seconds = 1.0 + 0.5 * r                     # rank 1 is the slower one
    slowest = replicas.max_over_ranks(my_seconds, ws)
    rate = replicas.whole_job_rate(1000, ws, slowest)
    mine = replicas.share(list(range(7)), r, ws)
    replicas.finish(ws)
    with open(os.path.join(out, f"rank{r}.json"), "w") as f:
        json.dump(dict(ws=ws, rank=r, local=local, slowest=slowest, rate=rate, mine=mine), f)


def test_two_gloo_ranks_max_time_and_whole_job_rate(tmp_path):
    port = free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for r, d in enumerate(res):
        assert d["ws"] == 2 and d["rank"] == r and d["local"] == r
        assert d["slowest"] == 1.5                  # the max over ranks, seen by both
        assert d["rate"] == pytest.approx(2000 / 1.5)
    # every item goes to exactly one rank
    assert sorted(res[0]["mine"] + res[1]["mine"]) == list(range(7))
    assert not set(res[0]["mine"]) & set(res[1]["mine"])


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    from paper_1410_3464_gb300 import replicas
    replicas.init(1)
    replicas.barrier(1)
    assert replicas.max_over_ranks(2.5, 1) == 2.5
    assert replicas.whole_job_rate(10, 1, 2.0) == 5.0
    assert replicas.share([1, 2, 3], 0, 1) == [1, 2, 3]
    replicas.finish(1)


def test_reference_arm_only_rank0_prints():
    """Under torchrun the reference arm runs on rank 0 alone; another rank
    exits 0 without work and prints nothing."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "1"], env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0
    assert p.stdout.strip() == ""
