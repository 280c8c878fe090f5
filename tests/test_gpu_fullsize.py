"""The larger configurations at full size, checked on sampled outputs that the oracle computes
(its preprocess covers every Gaussian and camera; it composites only the sampled tiles):

* the 6M city seen by 8 cameras of mixed resolution in one launch (four 1600x1067, four
  960x640), SH stored in FP16 with FP32 projection, blending and gradients;
* the 30M street-level scene at 3840x2160 with FP16 SH in recompute mode (the state keeps 12
  bytes per pixel and the backward re-bins); peak device memory is reported.

The oracle gets the dequantised SH (what the kernels compute with). Bars: exact visibility,
rectangles, tile lists and last contributors on unmarked items, images within 1e-4, upstream
gradients only on the sampled pixels so that the oracle's gradient restricted to those tiles is
the whole gradient. Gradients: the per-row 1e-3 bar, taken relative to the larger of the row and
the oracle's magnitude of the element's sum: in tiles of hundreds of Gaussians 400-800 m deep
the per-pixel contributions cancel to results far smaller than themselves, and FP32 summation is
accurate relative to their size, not to the result's."""
import numpy as np
import pytest
import torch

import oracle
from paper_2507_23006_gb300 import native, scenes
from tests import parity_util as pu
from tests.test_gpu_parity import _check_records, _gpu_backward

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return native.Context(0)


def _layout(cams):
    """Per camera: (first global tile, tiles_x, tiles_y, first packed pixel)."""
    out, t0, p0 = [], 0, 0
    for c in cams:
        tx, ty = (c.width + 15) // 16, (c.height + 15) // 16
        out.append((t0, tx, ty, p0))
        t0 += tx * ty
        p0 += c.width * c.height
    return out


def _sample_tiles(sa, cams, busy_per_cam, random_per_cam, seed):
    rng = np.random.default_rng(seed)
    counts = np.diff(sa["ranges"], axis=1)[:, 0]
    tiles = []
    for (t0, tx, ty, _), c in zip(_layout(cams), cams):
        local = np.arange(t0, t0 + tx * ty)
        busy = local[counts[local] > 0]
        tiles.append(rng.choice(busy, min(busy_per_cam, busy.size), replace=False))
        tiles.append(rng.choice(local, random_per_cam, replace=False))
    return np.unique(np.concatenate(tiles))


def _tile_pixels(tiles, cams, with_tile=False):
    lay = _layout(cams)
    starts = np.array([l[0] for l in lay])
    pix, tile_of = [], []
    for t in tiles:
        c = int(np.searchsorted(starts, t, side="right") - 1)
        t0, tx, _, p0 = lay[c]
        cam = cams[c]
        ty_, tx_ = divmod(int(t) - t0, tx)
        for y in range(ty_ * 16, min(ty_ * 16 + 16, cam.height)):
            x0, x1 = tx_ * 16, min(tx_ * 16 + 16, cam.width)
            pix.extend(range(p0 + y * cam.width + x0, p0 + y * cam.width + x1))
            tile_of.extend([int(t)] * (x1 - x0))
    pix = np.array(pix, np.int64)
    return (pix, np.array(tile_of, np.int64)) if with_tile else pix


def _check_last_contributor(sa, res, n, pix, tile_of, um_mask):
    """The pixel's last contributor is the same Gaussian. (n_contrib itself is a position in
    the tile's list and moves by one where a Gaussian that does not reach the pixel sits at a
    near-tie depth next to it; the image does not change.)"""
    gl = pu.gpu_tile_lists(sa, n)
    ol = pu.oracle_tile_lists(res.pairs)
    nc_g = sa["n_contrib"][pix]
    nc_o = res.img[pix, 7].astype(np.int64)
    for k in np.nonzero(um_mask)[0]:
        t = int(tile_of[k])
        a = gl[t][nc_g[k] - 1] if nc_g[k] > 0 else -1
        b = ol[t][nc_o[k] - 1] if nc_o[k] > 0 else -1
        assert a == b, (int(pix[k]), t, int(nc_g[k]), int(nc_o[k]))


def _dequantised(scene, g):
    return scenes.Scene(scene.means, scene.scales, scene.quats, scene.opacities, g.sh.float().cpu().numpy(),
                        scene.sh_degree)


def _check_images(out, res, pix, depth_scale, min_compared=0.9):
    """Unmarked pixels within 1e-4 (depth within 1e-4 of the depth scale). Marked pixels, except
    those whose tile list is itself uncertain, within 1e-4 plus the oracle's bound on what their
    uncertain decisions can change (res.bound). At least min_compared of the pixels are compared.
    Returns the unmarked pixels (the only ones that carry upstream gradients)."""
    mark = res.mark[pix]
    um = pix[mark == 0]
    mk = pix[(mark != 0) & ((mark & oracle.MARK_TILE) == 0)]
    compared = (um.size + mk.size) / pix.size
    print(f"\nimages: {um.size} unmarked, {mk.size} marked and compared within their bound, "
          f"{pix.size - um.size - mk.size} in uncertain tile lists, of {pix.size} ({compared:.3f} compared)")
    assert compared >= min_compared, f"{compared:.3f} of the sampled pixels compared"
    rgb = out["rgb"].cpu().numpy().astype(np.float64)
    alpha = out["alpha"].cpu().numpy().astype(np.float64)
    dacc = out["depth_acc"].cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(rgb[um], res.img[um, 0:3], atol=1e-4)
    np.testing.assert_allclose(alpha[um], res.img[um, 5], atol=1e-4)
    np.testing.assert_allclose(dacc[um], res.img[um, 3], atol=1e-4 * depth_scale)
    if mk.size:
        b = res.bound[mk]
        assert np.all(np.abs(rgb[mk] - res.img[mk, 0:3]).max(axis=1) <= 1e-4 + b[:, 0])
        assert np.all(np.abs(alpha[mk] - res.img[mk, 5]) <= 1e-4 + b[:, 2])
        assert np.all(np.abs(dacc[mk] - res.img[mk, 3]) <= 1e-4 * depth_scale + b[:, 1])
    return um


def test_city_8_cameras_mixed_resolution_fp16_sh(ctx):
    scene = scenes.city(2, 6_000_000)
    cams = scenes.city_batch_cameras(2)
    nopts, oopts = pu.opts_pair(tile_cull=True)
    g = native.Gaussians.from_scene(scene, sh_dtype=torch.float16)
    deq = _dequantised(scene, g)
    out, st = native.render_forward(ctx, g, cams, nopts)
    ctx.sync_check()
    sa = pu.state_arrays(st)
    tiles = _sample_tiles(sa, cams, 6, 2, seed=5)
    res = oracle.render(deq, cams, oopts, tile_subset=tiles, want_bound=True)
    _check_records(sa, deq, cams, oopts, res.gmark)
    pix, tile_of = _tile_pixels(tiles, cams, with_tile=True)
    um = _check_images(out, res, pix, depth_scale=400.0)
    _check_last_contributor(sa, res, scene.n, pix, tile_of, res.mark[pix] == 0)
    gl = pu.gpu_tile_lists(sa, scene.n)
    ol = pu.oracle_tile_lists(res.pairs)
    for t in tiles:
        a = gl.get(int(t), np.zeros(0, np.int64))
        b = ol.get(int(t), np.zeros(0, np.int64))
        np.testing.assert_array_equal(np.sort(a[res.gmark[a] == 0]), np.sort(b[res.gmark[b] == 0]))
    up = pu.upstream_on(um, sum(c.width * c.height for c in cams), seed=6, alpha=res.img[:, 5])
    gg = _gpu_backward(ctx, g, cams, st, up, nopts)
    ref = oracle.backward(deq, cams, up, oopts, tile_subset=tiles, want_mag=True)
    for k in ("means", "scales", "quats", "opacities", "sh"):
        pu.grad_close(gg[k], ref[k], k, mag=ref["mag"][k])


def test_large_street_level_4k_fp16_sh_recompute(ctx):
    scene = scenes.large_scene(4, 30_000_000)
    cam = scenes.street_level_camera(3840, 2160)
    nopts, oopts = pu.opts_pair(tile_cull=True, save_state=False)
    g = native.Gaussians.from_scene(scene, sh_dtype=torch.float16)
    deq = _dequantised(scene, g)
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats()
    out, st = native.render_forward(ctx, g, [cam], nopts)
    ctx.sync_check()
    info = st.info()
    npix = cam.width * cam.height
    assert info["n_pixels"] == npix
    # recompute mode: per-pixel state only (n_contrib, T_final, depth) and no pair lists
    nc = st.copy(native.BUF_N_CONTRIB, npix, torch.int32).cpu().numpy().view(np.uint32).astype(np.int64)
    tiles_x = (cam.width + 15) // 16
    rng = np.random.default_rng(7)
    busy = np.unique(np.nonzero(nc > 0)[0] // cam.width // 16 * tiles_x
                     + (np.nonzero(nc > 0)[0] % cam.width) // 16)
    tiles = np.unique(np.concatenate([rng.choice(busy, 32, replace=False),
                                      rng.choice(tiles_x * ((cam.height + 15) // 16), 8, replace=False)]))
    res = oracle.render(deq, [cam], oopts, tile_subset=tiles, want_pairs=False, want_bound=True)
    pix = _tile_pixels(tiles, [cam])
    # Looking down a street, many decisions sit within FP32 reach: facades that face the camera put
    # contributors at nearly equal depth (about 200 contributors per pixel), so the depth order of
    # a pixel's front layers is often not fixed by FP32; those pixels are compared within the
    # oracle's bound on what the order can change.
    um = _check_images(out, res, pix, depth_scale=100.0)
    # no pair lists are kept in recompute mode: n_contrib may differ by near-tie positions
    assert np.abs(nc[um] - res.img[um, 7].astype(np.int64)).max() <= 2
    up = pu.upstream_on(um, npix, seed=8, alpha=res.img[:, 5])
    gg = _gpu_backward(ctx, g, [cam], st, up, nopts)
    peak = torch.cuda.max_memory_allocated() + ctx.workspace_bytes()
    print(f"\n30M / 4K recompute: compared {um.size} of {pix.size} sampled pixels; "
          f"V={info['n_visible']} P={info['n_pairs']} "
          f"peak device memory {peak / 2**30:.2f} GiB (torch {torch.cuda.max_memory_allocated() / 2**30:.2f} GiB)")
    ref = oracle.backward(deq, [cam], up, oopts, tile_subset=tiles, want_mag=True)
    for k in ("means", "scales", "quats", "opacities", "sh"):
        pu.grad_close(gg[k], ref[k], k, mag=ref["mag"][k])
