"""The N > 1 host logic of bench.py on CPU with the gloo backend, world size 2:
the rendezvous, the barrier and the max-over-ranks timing, the whole-job
throughput of independent replicas, and the reference arm under torchrun
(rank 0 alone runs and prints one JSON line; the other rank exits 0)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench

    dist = bench.dist_init(world, use_cuda=False)
    bench.barrier(dist)
    m = bench.max_over_ranks(dist, 1.5 + rank, use_cuda=False)
    bench.barrier(dist)
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as fh:
        json.dump({"rank": rank, "max": m}, fh)


def test_gloo_barrier_and_max_over_ranks(tmp_path):
    import torch.multiprocessing as mp

    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    got = [json.load(open(tmp_path / f"r{r}.json")) for r in range(2)]
    assert [g["max"] for g in got] == [2.5, 2.5]


def test_replica_throughput_is_whole_job():
    sys.path.insert(0, ROOT)
    import bench

    # 2 replicas x 3 steps x 100 solves in 1.5 s (max over ranks)
    assert bench.replica_throughput(2, 3, 100, 1500.0) == pytest.approx(400.0)
    assert bench.replica_throughput(1, 3, 100, 1500.0) == pytest.approx(200.0)


def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--workload", "small", "--steps", "1", "--warmup", "0", "--time-steps", "2"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2 and out["value"] > 0
    assert out["cpu_baseline"]["kind"] == "oracle"
