"""Camera sharding on one GPU: the ranks of a camera-sharded step are run one after another in
this process (each renders its share of the launch's cameras through the library into its own
gradient buffer); the sum of their buffers, which is what the all-reduce computes, equals the
gradient of the launch rendered at once, and both match the oracle at the gradient bar."""
import numpy as np
import pytest
import torch

import oracle
from paper_2507_23006_gb300 import native, scenes, shard
from tests import parity_util as pu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return native.Context(0)


def test_sharded_gradients_sum_to_the_whole_launch(ctx):
    scene, cam = pu.scene_box(5000, seed=41)
    cams = [cam, scenes.box_camera(160, 96, f=200.0), scenes.box_camera(200, 136, f=180.0),
            scenes.pinhole(scenes.look_at((3.0, -2.0, -1.0), (0.0, 0.0, 10.0), up=(0, -1, 0)), 128, 128, fx=150.0)]
    rng = np.random.default_rng(2)
    affs = [np.concatenate([np.eye(3) + rng.normal(0, 0.1, (3, 3)), rng.normal(0, 0.1, (3, 1))], 1) for _ in cams]
    apps = [torch.tensor(a, dtype=torch.float32, device="cuda") for a in affs]
    nopts, oopts = pu.opts_pair(tile_cull=True, bg=(0.1, 0.1, 0.1))
    g = native.Gaussians.from_scene(scene)
    res = oracle.render(scene, cams, oopts, affines=np.stack(affs), want_pairs=False)
    up = pu.upstream(res, res.img.shape[0], seed=3)
    offs = np.cumsum([0] + [c.width * c.height for c in cams])

    def d_out_of(mine):
        rows = np.concatenate([np.arange(offs[c], offs[c + 1]) for c in mine])
        u = up[rows]
        return dict(rgb=torch.tensor(u[:, 0:3], dtype=torch.float32, device="cuda").contiguous(),
                    depth_acc=torch.tensor(u[:, 3], dtype=torch.float32, device="cuda").contiguous(),
                    depth_exp=torch.tensor(u[:, 4], dtype=torch.float32, device="cuda").contiguous(),
                    alpha=torch.tensor(u[:, 5], dtype=torch.float32, device="cuda").contiguous())

    world = 2
    parts = shard.shard_cameras([c.width * c.height for c in cams], world)
    assert all(parts)
    total = None
    for rank in range(world):
        buf = shard.GradBuffer(g.n, 16, len(cams))
        shard.local_grads(ctx, g, cams, parts[rank], d_out_of(parts[rank]), nopts, buf, appearances=apps)
        torch.cuda.synchronize()
        total = buf.flat.clone() if total is None else total + buf.flat
    summed = shard.GradBuffer(g.n, 16, len(cams))
    summed.flat.copy_(total)
    whole = native.render_backward(ctx, g, cams, native.render_forward(ctx, g, cams, nopts, appearances=apps)[1],
                                   d_out_of(range(len(cams))), nopts, appearances=apps)
    ctx.sync_check()
    ref = oracle.backward(scene, cams, up, oopts, affines=np.stack(affs), want_mag=True)
    for k in ("means", "scales", "quats", "opacities", "sh"):
        a = summed[k].cpu().numpy()
        b = whole[k].cpu().numpy()
        pu.grad_close(a, b, f"{k} (ranks summed vs one launch)", mag=ref["mag"][k])
        pu.grad_close(a, ref[k], f"{k} (ranks summed vs oracle)", mag=ref["mag"][k])
    pu.grad_close(summed["appearance"].cpu().numpy().reshape(len(cams), 12),
                  whole["appearance"].cpu().numpy().reshape(len(cams), 12), "appearance (ranks vs launch)")
    pu.grad_close(summed["appearance"].cpu().numpy().reshape(len(cams), 12), ref["affine"], "appearance (oracle)")
