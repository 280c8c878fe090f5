"""Parity of the per-Gaussian appearance transform (Sec. 3.5.1) on the GPU with the FP64 oracle:
the transformed records, the images, and every gradient (the Gaussians' own parameters, the
Gaussian and image embeddings and the four weight arrays), for several cameras of different
sizes in one launch, with the state kept and in recompute mode. Bars as in the other parity
tests: records and images within 1e-4, gradients within 1e-3 of the row plus 1e-3 of the
array's RMS."""
import numpy as np
import pytest
import torch

import oracle
from paper_2507_23006_gb300 import autograd, native, scenes
from tests import parity_util as pu
from tests.test_gpu_fullsize import _check_last_contributor, _tile_pixels
from tests.test_gpu_parity import _check_images, _check_lists, _check_records, _gpu_backward, _upstream

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return native.Context(0)


def _cams():
    cam, cam2 = scenes.box_camera(), scenes.box_camera(160, 96, f=200.0)
    cam3 = scenes.pinhole(scenes.look_at((3.0, -2.0, -1.0), (0.0, 0.0, 10.0), up=(0, -1, 0)), 200, 136, fx=180.0)
    return [cam, cam2, cam3]


def _setup(n, seed, n_cams):
    scene = scenes.box_scene(seed, n)
    mlp = scenes.appearance_mlp(np.random.default_rng(seed + 100), n, n_cams)
    g = native.Gaussians.from_scene(scene)
    g.mlp = native.AppearanceMLP.from_arrays(mlp)
    return scene, mlp, g


def _check_mlp_grads(gg, ref):
    pu.grad_close(gg["gauss_embed"], ref["mlp"]["gemb"], "gauss_embed")
    pu.grad_close(gg["image_embed"], ref["mlp"]["iemb"], "image_embed")
    p = gg["mlp_params"]
    off = 0
    for k, shape in (("w1", (32, 48)), ("b1", (32,)), ("w2", (4, 32)), ("b2", (4,))):
        size = int(np.prod(shape))
        pu.grad_close(p[off:off + size].reshape(shape), ref["mlp"][k], k)
        off += size


@pytest.mark.parametrize("aa,cull", [(True, False), (False, True)])
def test_forward_records_and_images(ctx, aa, cull):
    cams = _cams()
    scene, mlp, g = _setup(8000, 3, len(cams))
    nopts, oopts = pu.opts_pair(antialiased=aa, tile_cull=cull, bg=(0.1, 0.2, 0.3))
    out, st = native.render_forward(ctx, g, cams, nopts)
    ctx.sync_check()
    sa = pu.state_arrays(st)
    res = oracle.render(scene, cams, oopts, mlp=mlp)
    _check_records(sa, scene, cams, oopts, res.gmark, mlp=mlp)
    _check_lists(sa, res, scene, res.gmark)
    _check_images(out, res, cams, 15.0)
    # the last contributor of every unmarked pixel is the same Gaussian (its position in the
    # tile's list can move by one where a near-tie non-contributor sits next to it)
    pix, tile_of = _tile_pixels(np.arange(sa["info"]["n_tiles"]), cams, with_tile=True)
    _check_last_contributor(sa, res, scene.n, pix, tile_of, res.mark[pix] == 0)
    # the transform changes the image (it is not the identity at random weights)
    plain = oracle.render(scene, cams, oopts, want_pairs=False)
    assert np.abs(plain.img[:, 0:3] - res.img[:, 0:3]).max() > 0.05


def test_zero_output_layer_is_the_plain_render_at_half_opacity(ctx):
    """sigmoid(0) = 1/2: colour gain 1, opacity factor 1/2 (both exact in FP32)."""
    cams = _cams()[:1]
    scene, mlp, g = _setup(4000, 5, 1)
    g.mlp.params[32 * 48 + 32:] = 0.0
    nopts, _ = pu.opts_pair(bg=(0.1, 0.2, 0.3))
    out, _ = native.render_forward(ctx, g, cams, nopts, want_state=False)
    half = native.Gaussians.from_scene(scenes.Scene(scene.means, scene.scales, scene.quats,
                                                    np.asarray(scene.opacities) * 0.5, scene.sh, 3))
    ref, _ = native.render_forward(ctx, half, cams, nopts, want_state=False)
    ctx.sync_check()
    for k in ("rgb", "alpha", "depth_acc"):
        torch.testing.assert_close(out[k], ref[k], rtol=0, atol=2e-6)


@pytest.mark.parametrize("save", [True, False])
def test_backward_all_gradients(ctx, save):
    cams = _cams()
    scene, mlp, g = _setup(4000, 7, len(cams))
    nopts, oopts = pu.opts_pair(bg=(0.0, 0.5, 0.0), save_state=save)
    out, st = native.render_forward(ctx, g, cams, nopts)
    res = oracle.render(scene, cams, oopts, mlp=mlp, want_pairs=False)
    up = _upstream(res, res.img.shape[0], seed=9)
    gg = _gpu_backward(ctx, g, cams, st, up, nopts)
    ref = oracle.backward(scene, cams, up, oopts, mlp=mlp, want_mag=True)
    for k in ("means", "scales", "quats", "opacities", "sh"):
        pu.grad_close(gg[k], ref[k], f"{k} (save_state={save})", mag=ref["mag"][k])
    _check_mlp_grads(gg, ref)


def test_autograd_matches_render_backward(ctx):
    """rasterize() with embeddings and weights as leaves: the same gradients as the C-ABI
    backward (chained through the activations for the Gaussians' own parameters)."""
    cams = _cams()[:2]
    scene, mlp, g = _setup(3000, 11, len(cams))
    dev = "cuda"
    leaves = dict(gauss_embed=g.mlp.gauss_embed.clone().requires_grad_(True),
                  image_embed=g.mlp.image_embed.clone().requires_grad_(True),
                  mlp_params=g.mlp.params.clone().requires_grad_(True))
    means = g.means.clone().requires_grad_(True)
    log_scales = torch.log(g.scales).requires_grad_(True)
    logits = torch.logit(g.opacities.double()).float().requires_grad_(True)
    rgb, dacc, dexp, alpha = autograd.rasterize(ctx, means, log_scales, g.quats, logits, g.sh, cams, **leaves)
    w = torch.randn(rgb.shape, generator=torch.Generator(device=dev).manual_seed(3), device=dev)
    (rgb * w).sum().backward()
    nopts = native.Options()
    g2 = native.Gaussians(means.detach(), torch.exp(log_scales.detach()), g.quats,
                          torch.sigmoid(logits.detach()), g.sh, 3, None,
                          native.AppearanceMLP(*(v.detach() for v in leaves.values())))
    out, st = native.render_forward(ctx, g2, cams, nopts)
    ref = native.render_backward(ctx, g2, cams, st, dict(rgb=w), nopts)
    ctx.sync_check()
    # the two runs differ only in the order of their atomic additions
    for a, b in ((leaves["gauss_embed"].grad, ref["gauss_embed"]), (leaves["image_embed"].grad, ref["image_embed"]),
                 (leaves["mlp_params"].grad, ref["mlp_params"]), (means.grad, ref["means"])):
        assert a.shape == b.shape
        assert float(torch.linalg.norm(a - b)) <= 1e-5 * float(torch.linalg.norm(b)) and float(torch.linalg.norm(b)) > 0


def test_empty_and_invisible(ctx):
    """No Gaussian in front of the camera: zero gradients everywhere, embeddings included."""
    cams = _cams()[:1]
    scene, mlp, g = _setup(500, 13, 1)
    g.means[:, 2] = -50.0  # behind the camera
    nopts, _ = pu.opts_pair()
    out, st = native.render_forward(ctx, g, cams, nopts)
    gr = native.render_backward(ctx, g, cams, st, dict(rgb=torch.ones_like(out["rgb"])), nopts)
    ctx.sync_check()
    assert st.info()["n_visible"] == 0
    for k in ("gauss_embed", "image_embed", "mlp_params", "means"):
        assert torch.count_nonzero(gr[k]) == 0, k


def test_fp16_storage_with_the_transform(ctx):
    """FP16 attributes and SH with the transform on: records and images against the oracle on
    the dequantised inputs (what the kernels compute with)."""
    cams = _cams()[:2]
    scene, mlp, g32 = _setup(6000, 17, len(cams))
    g = native.Gaussians.from_scene(scene, attr_dtype=torch.float16, sh_dtype=torch.float16)
    g.mlp = g32.mlp
    deq = scenes.Scene(scene.means, g.scales.float().cpu().numpy(), g.quats.float().cpu().numpy(),
                       g.opacities.float().cpu().numpy(), g.sh.float().cpu().numpy(), 3)
    nopts, oopts = pu.opts_pair(bg=(0.1, 0.2, 0.3))
    out, st = native.render_forward(ctx, g, cams, nopts)
    ctx.sync_check()
    sa = pu.state_arrays(st)
    res = oracle.render(deq, cams, oopts, mlp=mlp)
    _check_records(sa, deq, cams, oopts, res.gmark, mlp=mlp)
    _check_images(out, res, cams, 15.0)


def test_segments_with_the_transform(ctx):
    """A segment list renders the listed Gaussians in list order: the same images as the
    concatenated arrays (embeddings sliced with them), bit for bit, and the same gradients
    (scattered back to the rows of the full arrays; zero elsewhere)."""
    cams = _cams()[:2]
    scene, mlp, g = _setup(5000, 19, len(cams))
    segs = [(3000, 1200), (0, 1700)]
    g.segments = segs
    idx = torch.cat([torch.arange(b, b + c) for b, c in segs]).cuda()
    flat = native.Gaussians(*(getattr(g, k)[idx].contiguous() for k in ("means", "scales", "quats", "opacities", "sh")),
                            3, None, native.AppearanceMLP(g.mlp.gauss_embed[idx].contiguous(), g.mlp.image_embed,
                                                          g.mlp.params))
    nopts, _ = pu.opts_pair(bg=(0.1, 0.2, 0.3))
    out_s, st_s = native.render_forward(ctx, g, cams, nopts)
    out_f, st_f = native.render_forward(ctx, flat, cams, nopts)
    ctx.sync_check()
    for k in ("rgb", "alpha", "depth_acc"):
        assert torch.equal(out_s[k], out_f[k]), k
    w = torch.randn(out_s["rgb"].shape, generator=torch.Generator(device="cuda").manual_seed(5), device="cuda")
    gs = native.render_backward(ctx, g, cams, st_s, dict(rgb=w), nopts)
    gf = native.render_backward(ctx, flat, cams, st_f, dict(rgb=w), nopts)
    ctx.sync_check()
    for k in ("gauss_embed", "means", "sh"):
        full = gs[k]
        assert torch.count_nonzero(full[torch.tensor(sorted(set(range(g.n)) - set(idx.tolist())), device="cuda")]) == 0
        a, b = full[idx], gf[k]
        assert float(torch.linalg.norm(a - b)) <= 1e-5 * float(torch.linalg.norm(b)), k
    for k in ("image_embed", "mlp_params"):
        assert float(torch.linalg.norm(gs[k] - gf[k])) <= 1e-5 * float(torch.linalg.norm(gf[k])), k


def test_cached_outputs_render_the_same_bits(ctx):
    """The transform's outputs cached for one image embedding (gsr_appearance_cache) render the
    same bits as evaluating it, for every camera given that embedding; the cache is for
    rendering only (the backward refuses it)."""
    cams = _cams()
    scene, mlp, g = _setup(6000, 29, len(cams))
    same = g.mlp.image_embed[:1].expand(len(cams), 32).contiguous()
    g.mlp = native.AppearanceMLP(g.mlp.gauss_embed, same, g.mlp.params)
    nopts, _ = pu.opts_pair(bg=(0.1, 0.2, 0.3))
    out_e, _ = native.render_forward(ctx, g, cams, nopts, want_state=False)
    cache = native.appearance_cache(ctx, g, 0)
    gc = native.Gaussians(g.means, g.scales, g.quats, g.opacities, g.sh, 3, None,
                          native.AppearanceMLP(None, None, None, cached=cache))
    out_c, st = native.render_forward(ctx, gc, cams, nopts)
    ctx.sync_check()
    for k in ("rgb", "alpha", "depth_acc"):
        assert torch.equal(out_e[k], out_c[k]), k
    # the cache holds the transform's outputs: sigmoids in (0, 1)
    assert float(cache.min()) > 0.0 and float(cache.max()) < 1.0
    with pytest.raises(native.GsrError):
        native.render_backward(ctx, gc, cams, st, dict(rgb=torch.ones_like(out_c["rgb"])), nopts)
