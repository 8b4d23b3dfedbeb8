"""The multi-rank logic of bench.py on CPU (gloo, world size 2). The fill
does not shard (replicas only): no data-path collective; the job's step time
is the max over ranks and `value` the whole-job throughput; the reference arm
runs on rank 0 alone."""
import json
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        step_ms = 10.0 + rank  # rank 1 is the slow one
        t = bench.reduce_max_over_ranks(step_ms, dist, "cpu")
        v = bench.job_throughput(world, 1000, t / 1e3)
        dist.barrier()
        q.put((rank, t, v))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in res] == [0, 1]
    for _, t, v in res:
        assert t == 11.0  # every rank reports the slowest rank's time
        assert abs(v - 2 * 1000 / 0.011) < 1e-6 * v  # units of both replicas over that time


def test_single_rank_helpers_are_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max_over_ranks(3.5) == 3.5
    assert bench.job_throughput(1, 10, 2.0) == 5.0


def test_reference_arm_runs_on_rank0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                          "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip() == ""
    for wl in ("ellipsoid_batch", "adjoint_3072", "cube_near_field"):  # single-mesh arm only: one line
        out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", wl],
                             capture_output=True, text=True, timeout=300)
        assert out.returncode == 0
        assert "unavailable" in json.loads(out.stdout.strip().splitlines()[-1])
