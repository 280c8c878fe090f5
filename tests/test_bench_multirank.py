"""The benchmark's multi-process path on CPU (gloo, world size 2): the work is sharded by camera
with no data exchange, the timings are reduced with a max over ranks, the job's time per step
divides that by the number of ranks, and only rank 0 prints the result line."""
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


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bench.rank_env()
        mx = bench.max_over_ranks(1.5 + 2.0 * r, w)
        dist.barrier()
        q.put((rank, r, w, lr, mx, bench.view_azimuth(r), bench.job_ms_per_step(mx, w)))
    finally:
        dist.destroy_process_group()


def test_rank_helpers_world_size_two():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [0, 1] and all(g[2] == 2 for g in got)
    assert [g[3] for g in got] == [0, 1]
    assert all(g[4] == 3.5 for g in got)               # every rank sees the slowest rank's time
    assert got[0][5] != got[1][5]                       # each rank renders its own view
    assert all(g[6] == pytest.approx(1.75) for g in got)  # two steps per 3.5 ms


def test_single_process_helpers_need_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, 1) == 2.5
    assert bench.job_ms_per_step(4.0, 1) == 4.0


def test_reference_arm_under_torchrun_two_ranks():
    """Launched as the driver launches it for N = 2: rank 0 alone times the oracle and prints
    one JSON line; rank 1 exits 0 without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--gaussians", "20000", "--width", "64", "--height", "48"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["unit"] == "ms/step"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["value"] > 0
