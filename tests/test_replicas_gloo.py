"""The N > 1 path of bench.py on CPU: two gloo ranks (no GPU).

bench.py runs one independent replica of the workload per GPU; the job's
time is the slowest rank's (all-reduce MAX) and its throughput counts the
work of every rank.  Under torchrun the reference arm runs on rank 0 only;
the other ranks exit 0 without output.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [130.0, 250.0][rank]
    worst = bench.max_over_ranks(local_ms, dist, "cpu")
    value = bench.replica_value(world, 4 * 1000 * 1000, 3, worst)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"worst": worst, "value": value}, f)


def test_two_gloo_ranks_agree_on_the_slowest_time(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as tmp

    port = _free_port()
    tmp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    got = [json.load(open(tmp_path / f"rank{r}.json")) for r in (0, 1)]
    assert got[0]["worst"] == got[1]["worst"] == 250.0
    # two replicas of 4e6 pairs x 3 steps in 0.25 s
    assert got[0]["value"] == pytest.approx(2 * 4e6 * 3 / 0.25)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--gpus", "2"], env=env, capture_output=True, text=True, timeout=300)
    assert res.returncode == 0
    assert res.stdout.strip() == ""
