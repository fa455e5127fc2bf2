"""bench.py's multi-GPU form is replicas only (one independent problem per
rank, no data-path collective): the timing is the slowest rank's and the
value counts every rank's units.  Checked here with two gloo ranks on CPU;
and the reference arm (the CPU oracle) prints its line on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [120.0, 95.0][rank]        # rank 0 is the slowest
        m = bench.replica_max(dist, local_ms, "cpu")
        v = bench.replica_value(world, 1000.0, m)
        out.put((rank, m, v))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_and_count_all():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, v in res:
        assert m == 120.0
        assert abs(v - 2 * 1000.0 / 0.120) < 1e-9


def test_replica_helpers_alone():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_max(None, 3.5) == 3.5
    assert bench.replica_value(1, 500.0, 250.0) == 2000.0


def _run_reference(rank: str):
    env = dict(os.environ, RANK=rank, WORLD_SIZE="2")
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--workload", "grid2d_64", "--steps", "1", "--warmup", "0"],
                          capture_output=True, text=True, env=env, cwd=ROOT, timeout=300)


def test_reference_arm_prints_on_rank0_only():
    r0 = _run_reference("0")
    assert r0.returncode == 0, r0.stderr[-2000:]
    line = json.loads(r0.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "cpu_baseline", "e2e", "config"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    r1 = _run_reference("1")
    assert r1.returncode == 0 and r1.stdout.strip() == ""
