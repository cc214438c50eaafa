"""The N > 1 path of bench.py on CPU: two gloo ranks (one process each) take the job's time
as the slowest rank's, give every rank its own independent TT, and only rank 0 prints;
the reference arm does no work on the other ranks.  No GPU is used."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(100.0 + 50.0 * rank, dist, "cpu")  # rank 1 is the slowest
    dist.barrier()
    with open(os.path.join(out, f"r{rank}.json"), "w") as f:
        json.dump({"ms": ms, "seed": bench.rank_seed(rank), "rate": bench.job_rate(world, 10, ms)}, f)
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp

    port = free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    r = [json.load(open(tmp_path / f"r{k}.json")) for k in range(2)]
    # the job's time is the slowest rank's, on every rank
    assert r[0]["ms"] == r[1]["ms"] == 150.0
    # independent problems: distinct seeds, rank 0 keeps the single-GPU workload's
    import bench

    assert r[0]["seed"] == bench.SEED and r[1]["seed"] != r[0]["seed"]
    # whole-job throughput: 2 ranks x 10 rounds in 0.15 s
    assert r[0]["rate"] == pytest.approx(2 * 10 / 0.150)


def test_single_process_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.job_rate(1, 4, 500.0) == pytest.approx(8.0)


def test_reference_arm_other_ranks_do_nothing():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, env=env, timeout=300)
    assert p.returncode == 0
    assert p.stdout.strip() == ""
