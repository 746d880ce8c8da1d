"""Host logic of bench.py's multi-rank (replica) path on CPU: two gloo ranks, no GPU.

With N > 1 every rank times its own replica; the job's time is the slowest rank's and the
reported value is the whole job's unknowns/s.  The reference arm runs on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ms = 10.0 * (rank + 1)  # rank 1 is the slower one
    job_ms = bench.max_over_ranks(dist, ms, "cpu")
    out[rank] = (job_ms, bench.job_throughput(world, 4, 8, 1000, job_ms))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        job_ms, value = out[rank]
        assert job_ms == 20.0  # the slowest rank
        assert value == world * 4 * 8 * 1000 / 0.020
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, 3.5, "cpu") == 3.5


def test_reference_arm_two_ranks_prints_one_line():
    """`bench.py --impl reference` under torchrun with two ranks: rank 0 times the oracle and prints one
    JSON line, rank 1 exits without work."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={_free_port()}", os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["n_gpus"] == 2
