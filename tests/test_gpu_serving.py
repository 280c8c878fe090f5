"""The continuous-batching server: results in the mix equal results alone, LOD + FP16 serving
stays within 45 dB PSNR of the FP32 render of the same selected set, and memory admission
holds requests back instead of failing them."""
import math

import numpy as np
import pytest
import torch

from paper_2507_23006_gb300 import lod, native, scenes, serve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def city_lod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fine = scenes.city(3, 400_000)
    mid = lod.merge_to_count(fine, 100_000)
    coarse = lod.merge_to_count(mid, 25_000)
    return lod.build_lod([coarse, mid, fine])


def _camera(rng):
    w, h = [(320, 180), (480, 270), (640, 360)][int(rng.integers(0, 3))]
    if rng.uniform() < 0.5:
        return scenes.walkthrough_camera(rng, w, h)
    return scenes.aerial_camera(w, h, altitude=rng.uniform(80, 300), pitch_deg=rng.uniform(30, 89),
                                target=(rng.uniform(-400, 400), rng.uniform(-400, 400), 0.0),
                                azimuth_deg=rng.uniform(0, 360))


def test_distinct_views_in_one_launch_equal_alone(city_lod):
    """Views of different resolutions whose detail selections differ, rendered in one launch
    (the union of their segments, each marked with the views that selected it), give each view
    the image it gets alone: bit for bit (the same records, depth order and blend)."""
    ctx = native.Context(0)
    srv = serve.RenderServer(slots=1, gaussian_budget=150_000)
    srv.add_scene("city", city_lod)
    g = srv.scenes["city"].g
    rng = np.random.default_rng(5)
    cams = [_camera(rng) for _ in range(6)]
    sels = [srv.select_levels("city", c) for c in cams]
    assert len({tuple(map(tuple, s[0])) for s in sels}) >= 3  # the views select differently
    segs, masks = native.union_segments([s[3] for s in sels])
    assert any(m & (m - 1) for m in masks) and any(not m & (m - 1) for m in masks)  # shared and own segments
    opts = native.Options(tile_cull=True)
    gb = native.Gaussians(g.means, g.scales, g.quats, g.opacities, g.sh, 3, segs, segment_cams=masks)
    out, st = native.render_forward(ctx, gb, cams, opts)
    ctx.sync_check()
    off = 0
    for cam, sel in zip(cams, sels):
        ga = native.Gaussians(g.means, g.scales, g.quats, g.opacities, g.sh, 3, sel[0])
        alone, _ = native.render_forward(ctx, ga, [cam], opts, want_state=False)
        hw = cam.width * cam.height
        for k in ("rgb", "depth_acc", "alpha"):
            assert torch.equal(alone[k], out[k][off:off + hw]), k
        off += hw
    # the launch read each Gaussian of the union once and made a record only for the views
    # that selected it
    assert st.info()["n_render"] == sum(c for _, c in segs)
    srv.close()
    ctx.close()


def test_results_in_the_mix_equal_results_alone(city_lod):
    rng = np.random.default_rng(0)
    trace = serve.poisson_trace(rng, 150.0, 0.25, "city", _camera)
    # a burst of distinct views arriving together: launches batch views whose resolutions and
    # detail selections differ
    trace += [(0.26, "city", _camera(rng)) for _ in range(12)]
    mixed = serve.RenderServer(slots=3, gaussian_budget=150_000)
    mixed.add_scene("city", city_lod)
    stats = mixed.run_trace(trace)
    mixed.close()
    assert stats["failed"] == 0 and stats["served"] == len(trace)
    assert stats["max_in_flight"] >= 2
    batched = [r for r in stats["requests"] if r.batch_size > 1]
    assert len(batched) >= 4 and stats["mean_batch"] > 1.0
    assert len({tuple(map(tuple, r.segments)) for r in batched}) >= 2
    alone = serve.RenderServer(slots=1, gaussian_budget=150_000)
    alone.add_scene("city", city_lod)
    for r in stats["requests"]:
        a = alone.submit("city", r.camera)
        a.done.wait(60)
        assert a.error is None
        assert a.segments == r.segments
        np.testing.assert_allclose(a.rgb.float().cpu().numpy(), r.rgb.float().cpu().numpy(), atol=1e-4, rtol=0)
    alone.close()
    assert 0 < stats["p50_ms"] <= stats["p99_ms"]


def test_lod_fp16_psnr_against_fp32_same_set(city_lod):
    ctx = native.Context(0)
    g32 = native.Gaussians.from_scene(city_lod.gaussians)
    g16 = native.Gaussians.from_scene(city_lod.gaussians, attr_dtype=torch.float16, sh_dtype=torch.float16)
    rng = np.random.default_rng(1)
    srv = serve.RenderServer(slots=1, gaussian_budget=150_000)
    srv.add_scene("city", city_lod)
    for _ in range(6):
        cam = _camera(rng)
        segs, nsel, _ = srv.select("city", cam)
        o32, _ = native.render_forward(ctx, native.Gaussians(g32.means, g32.scales, g32.quats, g32.opacities, g32.sh,
                                                             3, segs), [cam], native.Options(tile_cull=True),
                                       want_state=False)
        o16, _ = native.render_forward(ctx, native.Gaussians(g16.means, g16.scales, g16.quats, g16.opacities, g16.sh,
                                                             3, segs), [cam], native.Options(tile_cull=True),
                                       want_state=False)
        mse = float(((o32["rgb"].clamp(0, 1) - o16["rgb"].clamp(0, 1)) ** 2).mean())
        psnr = 10 * math.log10(1.0 / max(mse, 1e-20))
        assert psnr >= 45.0, psnr
    srv.close()


def test_memory_admission_serialises_instead_of_failing(city_lod):
    cam = scenes.aerial_camera(640, 360, altitude=150, pitch_deg=45)
    probe = serve.RenderServer(slots=1, gaussian_budget=150_000)
    probe.add_scene("city", city_lod)
    need = probe.submit("city", cam)
    need.done.wait(60)
    probe.close()
    # room for one request at a time: four slots, but never two in flight
    srv = serve.RenderServer(slots=4, gaussian_budget=150_000, memory_budget=int(need.mem_bytes * 1.5))
    srv.add_scene("city", city_lod)
    stats = srv.run_trace([(0.0005 * k, "city", cam) for k in range(8)])
    assert stats["failed"] == 0 and stats["max_in_flight"] == 1
    # a request larger than the whole budget is refused with a reason
    big = scenes.aerial_camera(3840, 2160, altitude=150, pitch_deg=45)
    r = srv.submit("city", big)
    assert r.done.is_set() and r.error is not None
    srv.close()
