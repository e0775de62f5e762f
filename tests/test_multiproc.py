"""The host logic of bench.py's N > 1 path on CPU, with two processes.

Every run on this hardware uses one GPU, and N ranks of bench.py are
independent replicas of the step (the torus shards into independent problems;
no data-path collective). What the ranks share is the timing: each times its
own K steps, the job's time is the slowest rank's (an all-reduce max), and the
throughput counts the zones of every rank over that time. Here two gloo ranks
on CPU check that reduction and the throughput formula, and the reference arm
is launched under torchrun with two ranks: rank 0 alone times the oracle and
prints the one JSON line, rank 1 exits 0 without work."""
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


def _rank_main(rank, world, port, out_path):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [12.5, 20.0][rank]  # rank 1 is the slower replica
        job_ms = bench.max_over_ranks(ms, dist, torch.device("cpu"))
        value = bench.throughput(1000, 10, world, job_ms)
        with open(f"{out_path}.{rank}", "w") as f:
            json.dump({"ms": job_ms, "value": value}, f)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_throughput_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp

    port = _free_port()
    out = str(tmp_path / "r")
    mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
    for rank in range(2):
        with open(f"{out}.{rank}") as f:
            r = json.load(f)
        assert r["ms"] == 20.0  # every rank sees the slowest rank's time
        assert r["value"] == pytest.approx(1000 * 10 * 2 / 20.0e-3)  # both ranks' zones over it


def test_single_process_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(7.25, None, None) == 7.25
    assert bench.throughput(1769472, 50, 1, 60.0) == pytest.approx(1769472 * 50 / 0.06)


@pytest.mark.slow
def test_reference_arm_under_torchrun_two_ranks():
    """bench.py --impl reference launched as the driver launches N > 1 arms:
    one JSON line (rank 0), exit status 0 on every rank."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
