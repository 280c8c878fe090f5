"""Runs a fixed number of training steps (forward + backward through the C ABI) on one
synthetic workload and nothing else: the command to put under a kernel profiler.

    python -m paper_2507_23006_gb300.run_step --gaussians 6000000 --width 1920 --height 1080 --steps 3

Workloads: `city` (a synthetic city grid seen from 150 m up at 45 degrees, the training-step
benchmark), `street` (a street block, one camera 30 m up looking 45 degrees down) and `box`
(uniform Gaussians in a box in front of the camera). `--fwd-only` runs forward renders without
saved state; `--fp16` stores attributes and SH in FP16; `--mlp` turns on the per-Gaussian
appearance transform (random embeddings and weights); `--global-sort` bins through the global
(tile, depth) radix sort instead of the per-tile sort; `--time` prints the device time per
step after the first, and then the mean time of each stage over as many more steps (CUDA events
around every stage).
"""
from __future__ import annotations

import argparse

import torch

from . import native, scenes


def workload(kind: str, n: int, width: int, height: int):
    if kind == "city":
        return scenes.city(2, n), scenes.aerial_camera(width, height, altitude=150.0, pitch_deg=45.0,
                                                       azimuth_deg=90.0)
    if kind == "street":
        return scenes.street_block(0, n), scenes.street_block_camera(width, height)
    if kind == "box":
        scene = scenes.box_scene(0, n)
        return scene, scenes.box_camera(width, height)
    raise ValueError(kind)


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--workload", default="city", choices=["city", "street", "box"])
    p.add_argument("--gaussians", type=int, default=6_000_000)
    p.add_argument("--width", type=int, default=1920)
    p.add_argument("--height", type=int, default=1080)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--fwd-only", action="store_true")
    p.add_argument("--fp16", action="store_true")
    p.add_argument("--mlp", action="store_true")
    p.add_argument("--tile-cull", type=int, default=1)
    p.add_argument("--global-sort", action="store_true")
    p.add_argument("--time", action="store_true")
    a = p.parse_args()
    scene, cam = workload(a.workload, a.gaussians, a.width, a.height)
    dt = torch.float16 if a.fp16 else torch.float32
    ctx = native.Context(0)
    g = native.Gaussians.from_scene(scene, attr_dtype=dt, sh_dtype=dt)
    if a.mlp:
        gm = torch.Generator(device="cuda").manual_seed(4321)
        g.mlp = native.AppearanceMLP(torch.randn((g.n, 16), device="cuda", generator=gm),
                                     torch.randn((1, 32), device="cuda", generator=gm),
                                     0.3 * torch.randn(native.MLP_PARAMS, device="cuda", generator=gm))
    opts = native.Options(tile_cull=bool(a.tile_cull), save_state=not a.fwd_only,
                          global_sort=a.global_sort)
    npix = cam.width * cam.height
    gen = torch.Generator(device="cuda").manual_seed(1234)
    d_out = dict(rgb=torch.randn((npix, 3), device="cuda", generator=gen),
                 depth_acc=torch.randn(npix, device="cuda", generator=gen) * 1e-2,
                 alpha=torch.randn(npix, device="cuda", generator=gen))
    grads = native.param_grads(ctx, g, 1)

    def step():
        if not a.fwd_only:
            native.zero_param_grads(ctx, g, grads)  # the backward zeroes them beside its blend
        out, st = native.render_forward(ctx, g, [cam], opts, want_state=not a.fwd_only)
        if st is not None:
            native.render_backward(ctx, g, [cam], st, d_out, opts, grads=grads)
            st.release()

    step()
    torch.cuda.synchronize()
    if a.time and a.steps > 1:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(a.steps - 1):
            step()
        e1.record()
        torch.cuda.synchronize()
        ctx.profile(True)
        ctx.profile_collect()
        for _ in range(a.steps - 1):
            step()
        torch.cuda.synchronize()
        ms = ctx.profile_collect()["ms"]
        ctx.profile(False)
        print(f"step={e0.elapsed_time(e1) / (a.steps - 1) * 1e3:.1f}us (without stage events); stages:",
              " ".join(f"{k}={v / (a.steps - 1) * 1e3:.1f}us" for k, v in ms.items() if v > 0))
    else:
        for _ in range(a.steps - 1):
            step()
    torch.cuda.synchronize()
    ctx.close()
    print(f"ran {a.steps} steps of {a.workload} n={g.n} {cam.width}x{cam.height}")


if __name__ == "__main__":
    main()
