"""Differentiation (torch.autograd) and reduced-precision storage, against the FP64 oracle.

* `rasterize` applies exp / sigmoid activations in torch and chains them with the library's
  backward; gradients of unconstrained parameters (log-scales, opacity logits, raw quaternions,
  SH, per-image 3x4 appearance) must match the oracle's analytic gradient chained by hand.
* Recompute mode (the state keeps 16 bytes per pixel; backward re-bins) gives the same
  gradients up to the order of the FP32 atomic sums.
* FP16 / BF16 attribute and SH storage: parity against the oracle run on the dequantized values
  (same 1e-4 / 1e-3 bars); the error against the FP32 inputs is reported, not pinned.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2507_23006_gb300 import autograd, native, scenes
from tests import parity_util as pu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return native.Context(0)


def _params(scene, dev="cuda"):
    t = lambda a: torch.tensor(np.asarray(a, np.float32), device=dev)  # noqa: E731
    p = dict(means=t(scene.means), log_scales=t(np.log(scene.scales)), quats=t(scene.quats),
             logits=t(np.log(scene.opacities) - np.log1p(-scene.opacities)), sh=t(scene.sh))
    for v in p.values():
        v.requires_grad_(True)
    return p


def _activated(p):
    return scenes.Scene(p["means"].detach().cpu().numpy(), torch.exp(p["log_scales"]).detach().cpu().numpy(),
                        p["quats"].detach().cpu().numpy(), torch.sigmoid(p["logits"]).detach().cpu().numpy(),
                        p["sh"].detach().cpu().numpy(), 3)


@pytest.mark.parametrize("recompute", [False, True])
def test_autograd_matches_oracle_chain(ctx, recompute):
    base, cam = pu.scene_box(3000, seed=12)
    cam2 = scenes.box_camera(128, 96, f=150.0)
    cams = [cam, cam2]
    p = _params(base)
    rng = np.random.default_rng(3)
    aff = np.stack([np.concatenate([np.eye(3) + rng.normal(0, 0.1, (3, 3)), rng.normal(0, 0.1, (3, 1))], 1)
                    for _ in cams])
    app = torch.tensor(aff, dtype=torch.float32, device="cuda", requires_grad=True)
    opts = native.Options(bg=(0.1, 0.0, 0.2))
    rgb, dacc, dexp, alpha = autograd.rasterize(ctx, p["means"], p["log_scales"], p["quats"], p["logits"], p["sh"],
                                                cams, appearance=app, opts=opts, recompute=recompute)
    scene = _activated(p)
    oopts = oracle.Opts(bg=(0.1, 0.0, 0.2))
    res = oracle.render(scene, cams, oopts, affines=aff, want_pairs=False)
    um = res.mark == 0
    np.testing.assert_allclose(rgb.detach().cpu().numpy()[um], res.img[um, :3], atol=1e-4)
    w = rng.normal(size=(res.img.shape[0], 6))
    w[~um] = 0.0
    w[:, 4] = 0.0
    wt = torch.tensor(w, dtype=torch.float32, device="cuda")
    loss = (rgb * wt[:, :3]).sum() + (dacc * wt[:, 3]).sum() + (alpha * wt[:, 5]).sum()
    loss.backward()
    ref = oracle.backward(scene, cams, w, oopts, affines=aff, want_mag=True)
    s = np.asarray(scene.scales, np.float64)
    o = np.asarray(scene.opacities, np.float64)
    mag = ref["mag"]
    pu.grad_close(p["means"].grad.cpu().numpy(), ref["means"], "means", mag=mag["means"])
    pu.grad_close(p["log_scales"].grad.cpu().numpy(), ref["scales"] * s, "log_scales", mag=mag["scales"] * s)
    pu.grad_close(p["quats"].grad.cpu().numpy(), ref["quats"], "quats", mag=mag["quats"])
    pu.grad_close(p["logits"].grad.cpu().numpy(), ref["opacities"] * o * (1 - o), "logits",
                  mag=mag["opacities"] * o * (1 - o))
    pu.grad_close(p["sh"].grad.cpu().numpy(), ref["sh"], "sh", mag=mag["sh"])
    pu.grad_close(app.grad.cpu().numpy().reshape(2, 12), ref["affine"], "appearance")


def test_recompute_equals_saved_state(ctx):
    """Same pair lists and the same per-pixel walk; the sums differ only in the order of the
    FP32 atomic additions across tiles: 1e-5 relative per element, and for cancelling sums
    1e-5 of the magnitude of their terms (the oracle's, chained through the activations)."""
    scene, cam = pu.scene_box(5000, seed=13)
    grads = []
    for recompute in (False, True):
        p = _params(scene)
        rgb, dacc, _, alpha = autograd.rasterize(ctx, p["means"], p["log_scales"], p["quats"], p["logits"], p["sh"],
                                                 [cam], opts=native.Options(tile_cull=True), recompute=recompute)
        (rgb.sum() + 0.1 * dacc.sum() + alpha.sum()).backward()
        grads.append([p[k].grad.clone() for k in ("means", "log_scales", "quats", "logits", "sh")])
    act = _activated(_params(scene))
    up = np.zeros((cam.width * cam.height, 6))
    up[:, 0:3] = 1.0
    up[:, 3] = 0.1
    up[:, 5] = 1.0
    mag = oracle.backward(act, [cam], up, oracle.Opts(tile_cull=True), want_mag=True)["mag"]
    s = np.asarray(act.scales, np.float64)
    o = np.asarray(act.opacities, np.float64)
    mags = dict(means=mag["means"], log_scales=mag["scales"] * s, quats=mag["quats"],
                logits=mag["opacities"] * o * (1 - o), sh=mag["sh"])
    for name, a, b in zip(("means", "log_scales", "quats", "logits", "sh"), *grads):
        pu.grad_close(a.cpu().numpy(), b.cpu().numpy(), name, rel=1e-5, group_rel=1e-6, mag=mags[name],
                      cancel_rel=1e-5)


@pytest.mark.parametrize("attr,sh", [(torch.float16, torch.float16), (torch.bfloat16, torch.bfloat16),
                                     (torch.float32, torch.float16)])
def test_reduced_precision_storage(ctx, attr, sh):
    scene, cam = pu.scene_box(6000, seed=14)
    g = native.Gaussians.from_scene(scene, attr_dtype=attr, sh_dtype=sh)
    # the dequantized values are what the kernels compute with
    deq = scenes.Scene(g.means.cpu().numpy(), g.scales.float().cpu().numpy(), g.quats.float().cpu().numpy(),
                       g.opacities.float().cpu().numpy(), g.sh.float().cpu().numpy(), 3)
    opts = native.Options(tile_cull=True)
    oopts = oracle.Opts(tile_cull=True)
    out, st = native.render_forward(ctx, g, [cam], opts)
    res = oracle.render(deq, [cam], oopts, want_pairs=False)
    um = res.mark == 0
    assert um.mean() > 0.9
    np.testing.assert_allclose(out["rgb"].cpu().numpy()[um], res.img[um, :3], atol=1e-4)
    np.testing.assert_allclose(out["alpha"].cpu().numpy()[um], res.img[um, 5], atol=1e-4)
    np.testing.assert_allclose(out["depth_acc"].cpu().numpy()[um], res.img[um, 3], atol=1e-4 * 15)
    up = np.random.default_rng(5).normal(size=(res.img.shape[0], 6))
    up[~um] = 0.0
    up[:, 4] = 0.0
    d = dict(rgb=torch.tensor(up[:, :3], dtype=torch.float32, device="cuda"),
             depth_acc=torch.tensor(up[:, 3], dtype=torch.float32, device="cuda"),
             alpha=torch.tensor(up[:, 5], dtype=torch.float32, device="cuda"))
    gr = native.render_backward(ctx, g, [cam], st, d, opts)
    ref = oracle.backward(deq, [cam], up, oopts, want_mag=True)
    for k in ("means", "scales", "quats", "opacities", "sh"):
        pu.grad_close(gr[k].cpu().numpy(), ref[k], f"{k} ({attr}, {sh})", mag=ref["mag"][k])
    # reported, not pinned: error of the reduced-precision render against the FP32 inputs
    full = oracle.render(scene, [cam], oopts, want_pairs=False)
    err = np.abs(out["rgb"].cpu().numpy() - full.img[:, :3])
    print(f"\nstorage attr={attr} sh={sh}: rgb vs FP32 inputs max {err.max():.2e} mean {err.mean():.2e}; "
          f"alpha max {np.abs(out['alpha'].cpu().numpy() - full.img[:, 5]).max():.2e}")
