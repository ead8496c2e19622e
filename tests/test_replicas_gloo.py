"""The multi-GPU path of bench.py is N independent replicas (the wave path
has no exchange step): each rank times its own work, the job takes the
slowest rank, and the value is the whole job's throughput. These tests run
that reduction on world_size-2 gloo process groups on the CPU."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seconds = [1.5, 2.0][rank]  # rank 1 is the slowest replica
    slowest = bench.replica_max(seconds, "cpu")
    value = bench.replica_value(1000, 10, slowest, world)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, slowest, value))


def test_replica_timing_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, value in res:
        assert slowest == 2.0
        assert value == pytest.approx(2 * 1000 * 10 / 2.0 / 1e9)


def test_replica_max_without_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_max(3.25, "cpu") == 3.25


def test_reference_arm_runs_on_rank_zero_only():
    # A non-zero rank of the reference arm exits 0 without work or output.
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "3", "--warmup", "3"], env=env, capture_output=True,
                         text=True, timeout=300)
    assert out.returncode == 0
    assert out.stdout.strip() == ""


def test_reference_arm_prints_its_line():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "64cube", "--steps", "3", "--warmup", "3"], env=env,
                         capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
