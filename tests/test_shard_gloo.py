"""Camera sharding of one scene (paper_2507_23006_gb300.shard) on CPU: the camera split covers
every camera exactly once and balances pixels, and the gradient exchange of world size 2 (gloo)
sums every array of the flat buffer, each rank's appearance rows landing at its cameras' launch
indices, in one collective call."""
import os
import socket
import sys

import numpy as np
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2507_23006_gb300 import shard  # noqa: E402

SIZES = [1600 * 1067] * 4 + [960 * 640] * 4  # the mixed-resolution launch of the 8-camera city


def test_shard_cameras_covers_each_camera_once_and_balances():
    for world in (1, 2, 3, 4, 8):
        parts = shard.shard_cameras(SIZES, world)
        flat = sorted(c for p in parts for c in p)
        assert flat == list(range(len(SIZES)))
        loads = [sum(SIZES[c] for c in p) for p in parts]
        assert max(loads) - min(loads) <= max(SIZES)
    assert shard.shard_cameras(SIZES, 2) == [[0, 2, 4, 6], [1, 3, 5, 7]]
    assert shard.shard_cameras([], 2) == [[], []]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _fill(buf, rank, mine, n, K):
    """What rank `rank`'s local backward would leave in its buffer: deterministic values."""
    rng = np.random.default_rng(100 + rank)
    for k in ("means", "scales", "quats", "opacities", "sh"):
        buf[k].copy_(torch.tensor(rng.normal(size=tuple(buf[k].shape)), dtype=torch.float32))
    buf["appearance"].zero_()
    for c in mine:
        buf["appearance"][c] = torch.tensor(rng.normal(size=(3, 4)), dtype=torch.float32)


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2507_23006_gb300 import shard as sh
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        n, K = 7, 16
        mine = sh.shard_cameras(SIZES, world)[rank]
        buf = sh.GradBuffer(n, K, len(SIZES), device="cpu")
        _fill(buf, rank, mine, n, K)
        buf.all_reduce()
        q.put((rank, mine, {k: v.numpy().copy() for k, v in buf.views.items()}))
    finally:
        dist.destroy_process_group()


def test_gradient_all_reduce_world_size_two():
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
    n, K = 7, 16
    expect = None
    for rank, mine, _ in got:
        b = shard.GradBuffer(n, K, len(SIZES), device="cpu")
        _fill(b, rank, mine, n, K)
        vals = {k: v.numpy().astype(np.float64) for k, v in b.views.items()}
        expect = vals if expect is None else {k: expect[k] + vals[k] for k in vals}
    for rank, mine, res in got:
        for k in expect:
            np.testing.assert_allclose(res[k], expect[k], rtol=1e-6, atol=1e-6)
    # every camera's appearance row came from exactly one rank
    owners = [set(m) for _, m, _ in got]
    assert owners[0].isdisjoint(owners[1]) and owners[0] | owners[1] == set(range(len(SIZES)))


def test_grad_buffer_views_share_one_flat_array():
    b = shard.GradBuffer(5, 9, 3, device="cpu")
    b["sh"].fill_(2.0)
    b["appearance"][1].fill_(3.0)
    assert b.flat.numel() == 5 * (3 + 3 + 4 + 1 + 27) + 3 * 12
    assert float(b.flat.sum()) == 5 * 27 * 2.0 + 12 * 3.0
