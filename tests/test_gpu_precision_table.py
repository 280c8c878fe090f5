"""Per-output error of reduced-precision storage against the FP64 oracle on the original inputs.

The workload is the 6M-Gaussian city seen by the eight cameras of one mixed-resolution launch
(four at 1600x1067, four at 960x640). Four storage modes are rendered forward and backward:
everything FP32; FP16 SH with FP32 attributes; FP16 attributes and SH; BF16 attributes and SH
(means are FP32 in every mode; projection, compositing and gradient sums are FP32 throughout).
Each is compared with the FP64 oracle run on the original, un-rounded inputs, on 64 sampled
tiles (six busy and two random per camera): rgb, alpha, accumulated depth and expected depth
over the pixels whose decisions FP32 settles (the oracle's unmarked pixels), and each gradient
group under the same upstream gradients.

The FP32 row must meet the parity bars (images within 1e-4, gradients within the element-wise
bar of the other backward tests). The rounded rows measure what the storage format costs; they
are printed as a table, not pinned, apart from the ordering FP32 < FP16 < BF16 of the image
error and finite values everywhere. Run with `-s` to see the table.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2507_23006_gb300 import native, scenes
from tests import parity_util as pu
from tests.test_gpu_fullsize import _sample_tiles, _tile_pixels
from tests.test_gpu_parity import _gpu_backward

pytestmark = pytest.mark.gpu

MODES = (("fp32", torch.float32, torch.float32),
         ("fp16 SH", torch.float32, torch.float16),
         ("fp16 attr + SH", torch.float16, torch.float16),
         ("bf16 attr + SH", torch.bfloat16, torch.bfloat16))
GROUPS = ("means", "scales", "quats", "opacities", "sh")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return native.Context(0)


def _image_errors(out, res, um):
    rgb = out["rgb"].cpu().numpy().astype(np.float64)[um]
    alpha = out["alpha"].cpu().numpy().astype(np.float64)[um]
    dacc = out["depth_acc"].cpu().numpy().astype(np.float64)[um]
    dexp = out["depth_exp"].cpu().numpy().astype(np.float64)[um]
    ref = res.img[um]
    e_rgb = np.abs(rgb - ref[:, 0:3]).max(axis=1)
    e_alpha = np.abs(alpha - ref[:, 5])
    # depth_exp = depth_acc / alpha is only compared where the pixel is reasonably covered
    cov = ref[:, 5] > 0.05
    e_dacc = np.abs(dacc - ref[:, 3]) / np.maximum(ref[:, 3], 1e-9)
    e_dexp = np.abs(dexp[cov] - ref[cov, 4]) / ref[cov, 4]
    stat = lambda e: (float(e.max()), float(np.percentile(e, 99.9)), float(e.mean()))  # noqa: E731
    return dict(rgb=stat(e_rgb), alpha=stat(e_alpha), depth_acc_rel=stat(e_dacc[cov]),
                depth_exp_rel=stat(e_dexp))


def _grad_errors(gg, ref):
    out = {}
    for k in GROUPS:
        a = np.asarray(gg[k], np.float64).reshape(-1)
        b = np.asarray(ref[k], np.float64).reshape(-1)
        ok, st = pu.grad_stats(a, b, mag=ref["mag"][k])
        rms = np.sqrt(np.mean(b * b))
        out[k] = dict(rel_l2=float(np.linalg.norm(a - b) / np.linalg.norm(b)),
                      max_over_rms=float(np.abs(a - b).max() / rms), strict=float(st["strict_pass"]),
                      bar=float(ok.mean()))
    return out


def test_storage_error_table(ctx):
    scene = scenes.city(2, 6_000_000)
    cams = scenes.city_batch_cameras(2)
    npix = sum(c.width * c.height for c in cams)
    nopts, oopts = pu.opts_pair(tile_cull=True)
    g = native.Gaussians.from_scene(scene)
    _, st = native.render_forward(ctx, g, cams, nopts)
    ctx.sync_check()
    tiles = _sample_tiles(pu.state_arrays(st), cams, 6, 2, seed=9)
    del st, g
    res = oracle.render(scene, cams, oopts, tile_subset=tiles, want_pairs=False)
    pix = _tile_pixels(tiles, cams)
    um = pix[res.mark[pix] == 0]
    assert um.size >= 0.9 * pix.size
    up = pu.upstream_on(um, npix, seed=10, alpha=res.img[:, 5])
    ref = oracle.backward(scene, cams, up, oopts, tile_subset=tiles, want_mag=True)
    rows = {}
    for name, ad, sd in MODES:
        g = native.Gaussians.from_scene(scene, attr_dtype=ad, sh_dtype=sd)
        out, st = native.render_forward(ctx, g, cams, nopts)
        gg = _gpu_backward(ctx, g, cams, st, up, nopts)
        rows[name] = (_image_errors(out, res, um), _grad_errors(gg, ref))
        for k in GROUPS:
            assert np.isfinite(gg[k]).all(), (name, k)
        if name == "fp32":
            img = rows[name][0]
            assert img["rgb"][0] <= 1e-4 and img["alpha"][0] <= 1e-4, img
            for k in GROUPS:
                pu.grad_close(gg[k], ref[k], f"{k} (fp32)", mag=ref["mag"][k])
        del g, st, out, gg
    print(f"\nstorage error against the FP64 oracle on the original inputs: city 6M, 8 cameras, "
          f"{tiles.size} tiles, {um.size} pixels")
    print("| storage | rgb max / p99.9 / mean | alpha max / p99.9 / mean | depth_acc rel max / mean | "
          "depth_exp rel max / mean |")
    print("|---|---|---|---|---|")
    for name, (img, _) in rows.items():
        f = lambda s: f"{s[0]:.1e} / {s[1]:.1e} / {s[2]:.1e}"  # noqa: E731
        print(f"| {name} | {f(img['rgb'])} | {f(img['alpha'])} | {img['depth_acc_rel'][0]:.1e} / "
              f"{img['depth_acc_rel'][2]:.1e} | {img['depth_exp_rel'][0]:.1e} / {img['depth_exp_rel'][2]:.1e} |")
    print("| storage | " + " | ".join(f"{k}: rel L2 / max/rms / strict" for k in GROUPS) + " |")
    print("|---|" + "---|" * len(GROUPS))
    for name, (_, gr) in rows.items():
        print(f"| {name} | " + " | ".join(f"{gr[k]['rel_l2']:.1e} / {gr[k]['max_over_rms']:.1e} / "
                                           f"{gr[k]['strict']:.4f}" for k in GROUPS) + " |")
    e = [rows[n][0]["rgb"][2] for n, _, _ in MODES]
    assert e[0] <= e[1] <= e[3] and e[2] <= e[3], e
