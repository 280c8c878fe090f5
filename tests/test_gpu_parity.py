"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element.

Bars: integer work (visibility, rectangles, pair sets, sort order, n_contrib) is exact on
every item the oracle does not mark as a knife edge (an FP32 decision within rounding reach of
its threshold); floating outputs within 1e-4 absolute (depth within 1e-4 of the depth scale);
gradients within 1e-3 relative plus 1e-3 of the group's RMS.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2507_23006_gb300 import native, scenes
from tests import parity_util as pu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return native.Context(0)


# ---- building blocks ----------------------------------------------------------------------------

@pytest.mark.parametrize("n,bits", [(0, 32), (1, 32), (4095, 32), (4096, 32), (4097, 16), (100_003, 13),
                                    (1_000_000, 32), (3_000_001, 24), (65_536, 8)])
def test_sort_matches_stable_numpy(ctx, n, bits):
    rng = np.random.default_rng(n + bits)
    keys = rng.integers(0, 2 ** 32, size=n, dtype=np.uint64).astype(np.uint32)
    if n > 10:
        keys[: n // 10] = keys[n // 3]  # many equal keys: stability matters
    vals = np.arange(n, dtype=np.uint32)
    kt = torch.from_numpy(keys.view(np.int32)).cuda()
    vt = torch.from_numpy(vals.view(np.int32)).cuda()
    ko, vo = native.sort_pairs_u32(ctx, kt, vt, 0, bits)
    ctx.sync_check()
    masked = keys & np.uint32((1 << bits) - 1) if bits < 32 else keys
    order = np.argsort(masked, kind="stable")
    np.testing.assert_array_equal(vo.cpu().numpy().view(np.uint32), vals[order])
    np.testing.assert_array_equal(ko.cpu().numpy().view(np.uint32), keys[order])
    # inputs untouched
    np.testing.assert_array_equal(kt.cpu().numpy().view(np.uint32), keys)


# ---- forward ------------------------------------------------------------------------------------

def _check_records(sa, scene, cams, oopts, gmark, mlp=None):
    n = scene.n
    rec = sa["rec"]
    x0, x1, y0, y1, cam_bits = pu.unpack_rect(rec)
    for c, cam in enumerate(cams):
        ref, flags = oracle.project(scene, cam, oopts, mlp=pu.mlp_for_camera(mlp, c))
        sel = sa["cam_of"] == c
        g = sa["g_of"][sel]
        vis_gpu = np.zeros(n, bool)
        vis_gpu[g] = True
        vis_ref = (flags & 1).astype(bool)
        unmarked = gmark[c * n:(c + 1) * n] == 0
        np.testing.assert_array_equal(vis_gpu[unmarked], vis_ref[unmarked])
        both = vis_gpu & vis_ref
        r = rec[sel]
        order = np.argsort(g)
        g, r = g[order], r[order]
        keep = both[g]
        g, r = g[keep], r[keep]
        R = ref[g]
        np.testing.assert_allclose(r[:, 0:2], R[:, 0:2], rtol=1e-5, atol=1e-3)
        np.testing.assert_allclose(r[:, 2], R[:, 5], rtol=1e-4, atol=1e-6)
        np.testing.assert_allclose(r[:, 3], R[:, 9], rtol=1e-6)
        np.testing.assert_allclose(r[:, 4:7], R[:, 2:5], rtol=1e-4, atol=1e-6 * np.abs(R[:, 2:5]).max())
        np.testing.assert_allclose(r[:, 7:10], R[:, 6:9], rtol=1e-5, atol=1e-5)
        um = unmarked[g]
        xx0, xx1, yy0, yy1, cb = (a[sel][order][keep] for a in (x0, x1, y0, y1, cam_bits))
        np.testing.assert_array_equal(np.stack([xx0, xx1, yy0, yy1], 1)[um], R[um][:, 11:15].astype(np.int64))
        assert np.all(cb == c)


def _check_lists(sa, res, scene, gmark):
    n = scene.n
    gl = pu.gpu_tile_lists(sa, n)
    ol = pu.oracle_tile_lists(res.pairs)
    assert set(gl) <= set(range(int(sa["info"]["n_tiles"])))
    z_of = {}
    rec = sa["rec"]
    ids = sa["cam_of"] * n + sa["g_of"]
    zv = np.zeros(len(gmark))
    zv[ids] = rec[:, 3]
    swaps = 0
    for t in set(gl) | set(ol):
        a = gl.get(t, np.zeros(0, np.int64))
        b = ol.get(t, np.zeros(0, np.int64))
        a_u = a[gmark[a] == 0]
        b_u = b[gmark[b] == 0]
        np.testing.assert_array_equal(np.sort(a_u), np.sort(b_u))
        # the GPU order is sorted by its own FP32 depth, ties to the lower index (exact)
        za = zv[a]
        ok = (za[1:] > za[:-1]) | ((za[1:] == za[:-1]) & (a[1:] > a[:-1]))
        assert ok.all(), f"tile {t} not in (depth, index) order"
        if not np.array_equal(a_u, b_u):
            swaps += 1
            # only swaps of near ties are allowed
            pos = {v: k for k, v in enumerate(b_u)}
            zb = zv[a_u]
            for k in range(len(a_u) - 1):
                if pos[a_u[k]] > pos[a_u[k + 1]]:
                    assert abs(zb[k] - zb[k + 1]) <= 2e-6 * max(zb[k], zb[k + 1])
    return swaps


def _check_images(out, res, cams, depth_scale):
    npix = pu.camera_list(cams)
    mark = res.mark.astype(bool)
    ref = res.img
    rgb = out["rgb"].cpu().numpy().astype(np.float64)
    um = ~mark
    assert um.mean() > 0.9, f"too many marked pixels ({mark.mean():.3f})"
    np.testing.assert_allclose(rgb[um], ref[um, 0:3], rtol=0, atol=1e-4)
    np.testing.assert_allclose(out["alpha"].cpu().numpy()[um], ref[um, 5], rtol=0, atol=1e-4)
    np.testing.assert_allclose(out["depth_acc"].cpu().numpy()[um], ref[um, 3], rtol=0, atol=1e-4 * depth_scale)
    al = ref[:, 5]
    sel = um & (al > 0.05)
    np.testing.assert_allclose(out["depth_exp"].cpu().numpy()[sel], ref[sel, 4], rtol=1e-4, atol=1e-4 * depth_scale)
    return int(mark.sum())


@pytest.mark.parametrize("aa,cull,global_sort", [(True, False, False), (False, True, False), (True, True, False),
                                                 (True, True, True)])
def test_box_scene_forward(ctx, aa, cull, global_sort):
    """10,000 Gaussians in a 10x10x10 box 5-15 units in front of a 256x256 camera (fx = 300);
    both orderings of the pairs (per-tile sorts and global radix sorts)."""
    scene, cam = pu.scene_box()
    nopts, oopts = pu.opts_pair(antialiased=aa, tile_cull=cull, bg=(0.1, 0.2, 0.3))
    nopts.global_sort = global_sort
    g, out, st = pu.gpu_render(ctx, scene, [cam], nopts)
    sa = pu.state_arrays(st)
    res = oracle.render(scene, [cam], oopts)
    assert sa["info"]["n_pairs"] > 0
    _check_records(sa, scene, [cam], oopts, res.gmark)
    _check_lists(sa, res, scene, res.gmark)
    _check_images(out, res, [cam], 15.0)
    um = res.mark == 0
    np.testing.assert_array_equal(sa["n_contrib"][um], res.img[um, 7].astype(np.int64))
    np.testing.assert_allclose(sa["T_final"][um], res.img[um, 6], rtol=1e-4, atol=1e-6)


def test_batched_cameras_and_appearance(ctx):
    scene, cam = pu.scene_box(6000, seed=5)
    cam2 = scenes.pinhole(scenes.look_at((3.0, -2.0, -1.0), (0.0, 0.0, 10.0), up=(0, -1, 0)), 200, 136, fx=180.0)
    cam3 = scenes.box_camera(96, 80, f=120.0)
    cams = [cam, cam2, cam3]
    rng = np.random.default_rng(1)
    aff = np.concatenate([np.eye(3) + rng.normal(0, 0.1, (3, 3)), rng.normal(0, 0.1, (3, 1))], axis=1)
    aff_t = torch.tensor(aff, dtype=torch.float32, device="cuda")
    nopts, oopts = pu.opts_pair(bg=(0.3, 0.3, 0.3))
    g = native.Gaussians.from_scene(scene)
    out, st = native.render_forward(ctx, g, cams, nopts, appearances=[None, aff_t, None])
    torch.cuda.synchronize()
    res = oracle.render(scene, cams, oopts, affines=np.stack([np.eye(3, 4), aff, np.eye(3, 4)]))
    sa = pu.state_arrays(st)
    _check_lists(sa, res, scene, res.gmark)
    _check_images(out, res, cams, 15.0)
    # one camera at a time gives the same bits
    off = 0
    for k, c in enumerate(cams):
        o1, _ = native.render_forward(ctx, g, [c], nopts, appearances=[[None, aff_t, None][k]], want_state=False)
        hw = c.width * c.height
        assert torch.equal(o1["rgb"], out["rgb"][off:off + hw])
        assert torch.equal(o1["depth_acc"], out["depth_acc"][off:off + hw])
        off += hw


def test_tile_cull_and_segments_and_permutation(ctx):
    scene, cam = pu.scene_box(8000, seed=7)
    g = native.Gaussians.from_scene(scene)
    a, _ = native.render_forward(ctx, g, [cam], native.Options(tile_cull=False), want_state=False)
    b, sb = native.render_forward(ctx, g, [cam], native.Options(tile_cull=True))
    assert (a["rgb"] - b["rgb"]).abs().max().item() <= 1e-6
    # segments: render [3000, 8000) then [0, 3000) == concatenation in that order
    g2 = native.Gaussians.from_scene(scene)
    g2.segments = [(3000, 5000), (0, 3000)]
    s1, _ = native.render_forward(ctx, g2, [cam], native.Options(), want_state=False)
    perm = np.concatenate([np.arange(3000, 8000), np.arange(3000)])
    g3 = native.Gaussians.from_scene(scene.subset(perm))
    s2, _ = native.render_forward(ctx, g3, [cam], native.Options(), want_state=False)
    for k in ("rgb", "depth_acc", "alpha"):
        assert torch.equal(s1[k], s2[k])
    # a random permutation changes nothing but exact-depth ties (none here)
    p = np.random.default_rng(2).permutation(scene.n)
    s3, _ = native.render_forward(ctx, native.Gaussians.from_scene(scene.subset(p)), [cam], native.Options(),
                                  want_state=False)
    assert (s3["rgb"] - a["rgb"]).abs().max().item() == 0.0


def test_edge_cases(ctx):
    cam = scenes.box_camera(37, 21, f=30.0)  # ragged tiles on both axes
    empty = scenes.Scene(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32), np.zeros((0, 4), np.float32),
                         np.zeros(0, np.float32), np.zeros((0, 16, 3), np.float32))
    out, st = native.render_forward(ctx, native.Gaussians.from_scene(empty), [cam],
                                    native.Options(bg=(0.25, 0.5, 1.0)))
    torch.cuda.synchronize()
    assert torch.allclose(out["rgb"], torch.tensor([0.25, 0.5, 1.0], device="cuda").expand_as(out["rgb"]))
    assert float(out["alpha"].abs().max()) == 0.0
    # everything culled (behind the camera)
    sc = scenes.box_scene(1, 500)
    sc.means[:, 2] *= -1
    out, st = native.render_forward(ctx, native.Gaussians.from_scene(sc), [cam], native.Options())
    assert st.info()["n_visible"] == 0 and float(out["alpha"].abs().max()) == 0.0
    # degenerate Gaussians are culled silently: zero quaternion, NaN mean
    sc2 = scenes.box_scene(2, 50)
    sc2.quats[0] = 0
    sc2.means[1] = np.nan
    out, st = native.render_forward(ctx, native.Gaussians.from_scene(sc2), [cam], native.Options())
    res = oracle.render(sc2, [cam])
    assert st.info()["n_visible"] == int(sum(1 for p in [oracle.project(sc2, cam)[1]] for f in p if f & 1))
    um = res.mark == 0
    np.testing.assert_allclose(out["rgb"].cpu().numpy()[um], res.img[um, :3], atol=1e-4)
    # invalid arguments are reported, not crashed on
    bad = scenes.box_camera(16, 16)
    bad.fx = -1.0
    with pytest.raises(native.GsrError) as e:
        native.render_forward(ctx, native.Gaussians.from_scene(sc2), [bad], native.Options())
    assert e.value.status == -1


@pytest.mark.parametrize("o", [0.5, 0.95])
def test_stacked_termination_closed_form(ctx, o):
    k = 40
    zs = 2.0 + 0.05 * np.arange(k)
    xw, yw = (40.5 - 32) / 100.0, (24.5 - 32) / 100.0
    n = k
    sc = scenes.Scene(np.stack([xw * zs, yw * zs, zs], 1).astype(np.float32), np.full((n, 3), 0.01, np.float32),
                      np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)), np.full(n, o, np.float32),
                      np.zeros((n, 16, 3), np.float32), 0)
    cam = scenes.box_camera(64, 64, f=100.0)
    out, st = native.render_forward(ctx, native.Gaussians.from_scene(sc), [cam], native.Options(antialiased=False))
    sa = pu.state_arrays(st)
    a = min(0.99, o)
    m = max(i for i in range(k + 1) if (1 - a) ** i >= 1e-4)
    assert sa["n_contrib"][24 * 64 + 40] == m
    assert abs(sa["T_final"][24 * 64 + 40] - (1 - a) ** m) <= 1e-6


# ---- backward -----------------------------------------------------------------------------------

_upstream = pu.upstream


def _gpu_backward(ctx, g, cams, st, up, nopts, appearances=None):
    """Parameter gradients of L = <up, outputs> through render_backward, on the host."""
    dev = "cuda"
    d = dict(rgb=torch.tensor(up[:, 0:3], dtype=torch.float32, device=dev).contiguous(),
             depth_acc=torch.tensor(up[:, 3], dtype=torch.float32, device=dev).contiguous(),
             depth_exp=torch.tensor(up[:, 4], dtype=torch.float32, device=dev).contiguous(),
             alpha=torch.tensor(up[:, 5], dtype=torch.float32, device=dev).contiguous())
    gr = native.render_backward(ctx, g, cams, st, d, nopts, appearances=appearances)
    ctx.sync_check()
    return {k: (v.cpu().numpy() if v is not None else None) for k, v in gr.items()}


@pytest.mark.parametrize("aa,cull,deg", [(True, False, 3), (False, True, 3), (True, True, 1)])
def test_box_scene_backward(ctx, aa, cull, deg):
    scene, cam = pu.scene_box_backward(4000, seed=3)
    scene.sh_degree = deg
    nopts, oopts = pu.opts_pair(antialiased=aa, tile_cull=cull, bg=(0.2, 0.1, 0.0), absgrad=True)
    g, out, st = pu.gpu_render(ctx, scene, [cam], nopts)
    res = oracle.render(scene, [cam], oopts, want_pairs=False)
    up = _upstream(res, cam.width * cam.height, seed=11)
    gg = _gpu_backward(ctx, g, [cam], st, up, nopts)
    ref = oracle.backward(scene, [cam], up, oopts, want_mag=True)
    for k in ("means", "scales", "quats", "opacities", "sh"):
        pu.grad_close(gg[k], ref[k], k, mag=ref["mag"][k])
    pu.grad_close(gg["absgrad"], ref["absgrad"], "absgrad")  # sums of magnitudes: no cancellation
    pu.grad_close(gg["appearance"], ref["affine"], "appearance")


@pytest.mark.parametrize("shift", [1, 2, 3])
def test_gradient_rows_unaligned_and_prefilled(ctx, shift):
    """Gradient arrays that start 4, 8 or 12 bytes past a 16-byte boundary and hold NaN before
    the call: every row is written (rows of Gaussians without a record exactly 0) and the values
    match the oracle's gradient at the usual bar."""
    scene, cam = pu.scene_box(20000, seed=21)
    m = np.array(scene.means, np.float64)
    m[::3, 2] = -5.0  # a third of the Gaussians behind the camera: no record
    scene = scenes.Scene(m, scene.scales, scene.quats, scene.opacities, scene.sh, 3)
    nopts, oopts = pu.opts_pair(tile_cull=True, absgrad=True)
    g, out, st = pu.gpu_render(ctx, scene, [cam], nopts)
    res = oracle.render(scene, [cam], oopts, want_pairs=False)
    up = _upstream(res, cam.width * cam.height, seed=3)
    ref = oracle.backward(scene, [cam], up, oopts, want_mag=True)
    n = g.n
    shapes = dict(means=(n, 3), scales=(n, 3), quats=(n, 4), opacities=(n,), sh=(n, 16, 3), absgrad=(n, 2))
    grads = {}
    for k, shp in shapes.items():
        size = int(np.prod(shp))
        buf = torch.full((size + 8,), float("nan"), device="cuda")
        grads[k] = buf[shift:shift + size].view(shp)
    grads["appearance"] = torch.full((1, 3, 4), float("nan"), device="cuda")
    d = dict(rgb=torch.tensor(up[:, 0:3], dtype=torch.float32, device="cuda").contiguous(),
             depth_acc=torch.tensor(up[:, 3], dtype=torch.float32, device="cuda").contiguous(),
             depth_exp=torch.tensor(up[:, 4], dtype=torch.float32, device="cuda").contiguous(),
             alpha=torch.tensor(up[:, 5], dtype=torch.float32, device="cuda").contiguous())
    native.render_backward(ctx, g, [cam], st, d, nopts, grads=grads)
    hidden = m[:, 2] < 0
    for k in shapes:
        got = grads[k].cpu().numpy().reshape(n, -1)
        assert np.isfinite(got).all(), k
        assert (got[hidden] == 0).all(), k
        pu.grad_close(got, np.asarray(ref[k]).reshape(n, -1), k,
                      mag=None if k == "absgrad" else np.asarray(ref["mag"][k]).reshape(n, -1))


@pytest.mark.parametrize("early", [0.0, 0.37, 1.0])
def test_param_grads_zeroed_ahead_of_the_forward(ctx, early):
    """gsr_param_grads_zero before the forward: the backward with the same arrays zeroes them
    (one fill, of which the forward queued the first `early` share: none, a part ending inside the
    SH array's span, or all); a backward given other arrays zeroes the requested ones too and
    fills its own. Both are checked on NaN-prefilled arrays against the oracle."""
    ctx.set_fill_split(early)
    scene, cam = pu.scene_box(8000, seed=22)
    m = np.array(scene.means, np.float64)
    m[::4, 2] = -5.0
    scene = scenes.Scene(m, scene.scales, scene.quats, scene.opacities, scene.sh, 3)
    hidden = m[:, 2] < 0
    nopts, oopts = pu.opts_pair(tile_cull=True)
    g = native.Gaussians.from_scene(scene)
    res = oracle.render(scene, [cam], oopts, want_pairs=False)
    up = _upstream(res, cam.width * cam.height, seed=4)
    ref = oracle.backward(scene, [cam], up, oopts, want_mag=True)
    d = dict(rgb=torch.tensor(up[:, 0:3], dtype=torch.float32, device="cuda").contiguous(),
             depth_acc=torch.tensor(up[:, 3], dtype=torch.float32, device="cuda").contiguous(),
             depth_exp=torch.tensor(up[:, 4], dtype=torch.float32, device="cuda").contiguous(),
             alpha=torch.tensor(up[:, 5], dtype=torch.float32, device="cuda").contiguous())

    def nan_grads():
        gr = native.param_grads(ctx, g, 1)
        for v in gr.values():
            if v is not None:
                v.fill_(float("nan"))
        return gr

    for same in (True, False):
        a, b = nan_grads(), nan_grads()
        native.zero_param_grads(ctx, g, a)
        out, st = native.render_forward(ctx, g, [cam], nopts)
        got = native.render_backward(ctx, g, [cam], st, d, nopts, grads=a if same else b)
        ctx.sync_check()
        for k in ("means", "scales", "quats", "opacities", "sh"):
            arr = got[k].cpu().numpy().reshape(g.n, -1)
            assert np.isfinite(arr).all(), (k, same)
            assert (arr[hidden] == 0).all(), (k, same)
            pu.grad_close(arr, np.asarray(ref[k]).reshape(g.n, -1), f"{k} (same arrays: {same})",
                          mag=np.asarray(ref["mag"][k]).reshape(g.n, -1))
        if not same:  # the arrays requested for zeroing were not used by the backward, but are zero
            assert all((a[k] == 0).all() for k in ("means", "scales", "quats", "opacities", "sh"))
    ctx.set_fill_split(0.0)


def test_backward_batched_with_appearance_and_recompute(ctx):
    scene, cam = pu.scene_box(3000, seed=4)
    cam2 = scenes.box_camera(160, 96, f=200.0)
    cams = [cam, cam2]
    rng = np.random.default_rng(8)
    aff = np.concatenate([np.eye(3) + rng.normal(0, 0.1, (3, 3)), rng.normal(0, 0.1, (3, 1))], axis=1)
    aff_t = torch.tensor(aff, dtype=torch.float32, device="cuda")
    for save in (True, False):
        nopts, oopts = pu.opts_pair(bg=(0.0, 0.5, 0.0), save_state=save)
        g = native.Gaussians.from_scene(scene)
        out, st = native.render_forward(ctx, g, cams, nopts, appearances=[aff_t, None])
        res = oracle.render(scene, cams, oopts, affines=np.stack([aff, np.eye(3, 4)]), want_pairs=False)
        up = _upstream(res, res.img.shape[0], seed=5)
        gg = _gpu_backward(ctx, g, cams, st, up, nopts, appearances=[aff_t, None])
        ref = oracle.backward(scene, cams, up, oopts, affines=np.stack([aff, np.eye(3, 4)]), want_mag=True)
        for k in ("means", "scales", "quats", "opacities", "sh"):
            pu.grad_close(gg[k], ref[k], f"{k} (save_state={save})", mag=ref["mag"][k])
        pu.grad_close(gg["appearance"].reshape(2, 12), ref["affine"], "appearance")


def test_backward_against_finite_differences(ctx):
    """GPU gradient vs FP64 central differences of the oracle on a tiny scene."""
    scene, cam = scenes.tiny_scene(31, 24, 32, 32, log_scale_mean=-1.8)
    params = {k: np.asarray(getattr(scene, k), np.float64).copy()
              for k in ("means", "scales", "quats", "opacities", "sh")}
    scene = scenes.Scene(params["means"], params["scales"], params["quats"], params["opacities"], params["sh"], 3)
    nopts, oopts = pu.opts_pair(bg=(0.1, 0.1, 0.1))
    g, out, st = pu.gpu_render(ctx, scene, [cam], nopts)
    res = oracle.render(scene, [cam], oopts, want_pairs=False, want_sig=True)
    up = _upstream(res, 32 * 32, seed=2)
    gg = _gpu_backward(ctx, g, [cam], st, up, nopts)
    rng = np.random.default_rng(0)
    fl0 = oracle.project(scene, cam, oopts)[1]
    checked = 0
    for gi in rng.choice(np.nonzero(fl0 & 1)[0], size=6, replace=False):
        for name in ("means", "scales", "quats", "opacities"):
            arr = params[name].reshape(scene.n, -1)
            for j in range(arr.shape[1]):
                th = arr[gi, j]
                h = 1e-6 * max(1.0, abs(th))
                L = []
                same = True
                for sgn in (1, -1):
                    arr[gi, j] = th + sgn * h
                    r = oracle.render(scene, [cam], oopts, want_pairs=False, want_sig=True)
                    same &= np.array_equal(r.sig, res.sig)
                    L.append(float(np.sum(up * r.img[:, :6])))
                arr[gi, j] = th
                if not same:
                    continue
                fd = (L[0] - L[1]) / (2 * h)
                an = gg[name].reshape(scene.n, -1)[gi, j]
                scale = np.sqrt(np.mean(gg[name] ** 2))
                assert abs(an - fd) <= 1e-3 * abs(fd) + 1e-3 * scale, (name, gi, j, an, fd)
                checked += 1
    assert checked >= 40


# ---- the full-size street block, on sampled tiles ----------------------------------------------

@pytest.fixture(scope="module")
def street():
    return scenes.street_block(1, 500_000), scenes.street_block_camera()


def test_street_block_full_size_sampled(ctx, street):
    """500,000 Gaussians, 1920x1080: every record against the oracle; images and gradients on 48
    random tiles (the oracle composites only those)."""
    scene, cam = street
    nopts, oopts = pu.opts_pair(tile_cull=True)
    g, out, st = pu.gpu_render(ctx, scene, [cam], nopts)
    sa = pu.state_arrays(st)
    ntx = (cam.width + 15) // 16
    nty = (cam.height + 15) // 16
    rng = np.random.default_rng(4)
    counts = np.diff(sa["ranges"], axis=1)[:, 0]
    busy = np.nonzero(counts > 0)[0]
    tiles = np.unique(np.concatenate([rng.choice(busy, 40, replace=False), rng.choice(ntx * nty, 8, replace=False)]))
    res = oracle.render(scene, [cam], oopts, tile_subset=tiles)
    _check_records(sa, scene, [cam], oopts, res.gmark)
    # images on the sampled tiles
    pix = []
    for t in tiles:
        ty, tx = divmod(int(t), ntx)
        for y in range(ty * 16, min(ty * 16 + 16, cam.height)):
            for x in range(tx * 16, min(tx * 16 + 16, cam.width)):
                pix.append(y * cam.width + x)
    pix = np.array(pix)
    um = pix[res.mark[pix] == 0]
    assert um.size > 0.8 * pix.size
    rgb = out["rgb"].cpu().numpy()
    np.testing.assert_allclose(rgb[um], res.img[um, 0:3], atol=1e-4)
    np.testing.assert_allclose(out["alpha"].cpu().numpy()[um], res.img[um, 5], atol=1e-4)
    np.testing.assert_allclose(out["depth_acc"].cpu().numpy()[um], res.img[um, 3], atol=1e-4 * 150.0)
    np.testing.assert_array_equal(sa["n_contrib"][um], res.img[um, 7].astype(np.int64))
    # tile lists of the sampled tiles
    gl = pu.gpu_tile_lists(sa, scene.n)
    ol = pu.oracle_tile_lists(res.pairs)
    for t in tiles:
        a = gl.get(int(t), np.zeros(0, np.int64))
        b = ol.get(int(t), np.zeros(0, np.int64))
        np.testing.assert_array_equal(np.sort(a[res.gmark[a] == 0]), np.sort(b[res.gmark[b] == 0]))
    # gradients with upstream only on the sampled, unmarked pixels (depth_exp where alpha > 0.05)
    up = pu.upstream_on(um, cam.width * cam.height, seed=9, alpha=res.img[:, 5])
    gg = _gpu_backward(ctx, g, [cam], st, up, nopts)
    ref = oracle.backward(scene, [cam], up, oopts, tile_subset=tiles, want_mag=True)
    for k in ("means", "scales", "quats", "opacities", "sh"):
        pu.grad_close(gg[k], ref[k], k, mag=ref["mag"][k])


@pytest.mark.parametrize("which", ["box", "street"])
def test_global_sort_gives_the_same_bits(ctx, which):
    """The two orderings of the (tile, Gaussian) pairs, per-tile sorts in shared memory and global
    onesweep radix sorts (depth, then stably by tile), put every tile's list in the same
    (depth, index) order: records, pair lists, ranges, last contributors and images bit for bit;
    gradients equal up to the order of the FP32 atomic sums."""
    if which == "box":
        scene, cam = pu.scene_box(10_000, seed=8)
    else:
        scene, cam = scenes.street_block(1, 500_000), scenes.street_block_camera()
    g = native.Gaussians.from_scene(scene)
    res = {}
    for glob in (False, True):
        opts = native.Options(tile_cull=True, global_sort=glob)
        out, st = native.render_forward(ctx, g, [cam], opts)
        ctx.sync_check()
        sa = pu.state_arrays(st)
        up = np.random.default_rng(3).normal(size=(cam.width * cam.height, 6))
        up[:, 4] = 0.0
        gr = _gpu_backward(ctx, g, [cam], st, up, opts)
        res[glob] = (out, sa, gr)
    (o0, s0, g0), (o1, s1, g1) = res[False], res[True]
    assert s0["info"]["n_pairs"] == s1["info"]["n_pairs"] > 0
    for k in ("rec", "g_of", "pair_vals", "ranges", "n_contrib", "T_final"):
        np.testing.assert_array_equal(s0[k], s1[k], err_msg=k)
    for k in ("rgb", "depth_acc", "depth_exp", "alpha"):
        assert torch.equal(o0[k], o1[k]), k
    up = np.random.default_rng(3).normal(size=(cam.width * cam.height, 6))
    up[:, 4] = 0.0
    mag = oracle.backward(scene, [cam], up, oracle.Opts(tile_cull=True), want_mag=True)["mag"]
    for k in ("means", "scales", "quats", "opacities", "sh"):
        pu.grad_close(g1[k], g0[k], f"{k} (global vs per-tile sort)", rel=1e-5, group_rel=1e-6, mag=mag[k],
                      cancel_rel=1e-5)


@pytest.mark.parametrize("scale,size,f", [(4.0, (256, 256), 300.0), (25.0, (96, 80), 100.0)])
def test_long_tile_lists(ctx, scale, size, f):
    """Tile lists of more than 1024 pairs are sorted by a launch of their own before the forward
    blend (lists over 16384 in runs merged through global memory), the shorter ones by the blend
    itself. The first scene mixes both kinds, the second has lists of up to 19k pairs. Every list
    is in (depth, record) order and has the same bits as the global radix-sort binning (records,
    lists, ranges, last contributors, images); on the mixed scene the image matches the oracle."""
    scene, _ = pu.scene_box(20_000, seed=21)
    scene.scales = (np.asarray(scene.scales) * scale).astype(np.float32)
    cam = scenes.box_camera(size[0], size[1], f=f)
    g = native.Gaussians.from_scene(scene)
    res = {}
    for glob in (False, True):
        opts = native.Options(tile_cull=True, global_sort=glob)
        out, st = native.render_forward(ctx, g, [cam], opts)
        ctx.sync_check()
        res[glob] = (out, pu.state_arrays(st))
    (o0, s0), (o1, s1) = res[False], res[True]
    counts = np.diff(s0["ranges"], axis=1)[:, 0]
    if scale < 10:
        assert (counts > 1024).sum() > 0 and ((counts > 0) & (counts <= 1024)).sum() > 0
    else:
        assert counts.max() > 16384
    assert s0["info"]["max_tile_pairs"] == counts.max()
    depth_bits = s0["rec"][:, 3].view(np.uint32).astype(np.uint64)
    for t in np.nonzero(counts)[0]:
        v = s0["pair_vals"][s0["ranges"][t, 0]:s0["ranges"][t, 1]].astype(np.uint64)
        key = (depth_bits[v] << np.uint64(32)) | v
        assert np.all(key[1:] > key[:-1]), t
    for k in ("rec", "g_of", "pair_vals", "ranges", "n_contrib", "T_final"):
        np.testing.assert_array_equal(s0[k], s1[k], err_msg=k)
    for k in ("rgb", "depth_acc", "depth_exp", "alpha"):
        assert torch.equal(o0[k], o1[k]), k
    if scale < 10:
        ref = oracle.render(scene, [cam], oracle.Opts(tile_cull=True), want_pairs=False)
        um = ref.mark == 0
        assert um.mean() > 0.7
        np.testing.assert_allclose(o0["rgb"].cpu().numpy()[um], ref.img[um, :3], atol=1e-4)
        np.testing.assert_allclose(o0["alpha"].cpu().numpy()[um], ref.img[um, 5], atol=1e-4)


def test_preprocess_record_order_and_repeatability():
    """The cull pass numbers the visible (Gaussian, camera) records in (Gaussian, camera) order and
    the record pass fills them in: over three cameras the owners never decrease and the cameras
    of one Gaussian's records increase; a second launch gives the same bits."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c2 = native.Context(0)
    scene, cam = pu.scene_box(6000, seed=23)
    cams = [cam, scenes.box_camera(200, 120, f=250.0), scenes.box_camera(64, 64, f=120.0)]
    nopts, _ = pu.opts_pair(bg=(0.1, 0.2, 0.3))
    g = native.Gaussians.from_scene(scene)
    out1, st1 = native.render_forward(c2, g, cams, nopts)
    sa1 = pu.state_arrays(st1)
    out2, st2 = native.render_forward(c2, g, cams, nopts)
    sa2 = pu.state_arrays(st2)
    c2.sync_check()
    own, cam_of = sa1["g_of"], sa1["cam_of"]
    assert own.size > 0.25 * scene.n and np.unique(cam_of).size == 3
    key = own * 4 + cam_of
    assert np.all(key[1:] > key[:-1])
    np.testing.assert_array_equal(sa1["rec"].view(np.uint32), sa2["rec"].view(np.uint32))
    np.testing.assert_array_equal(sa1["g_of"], sa2["g_of"])
    for k in ("rgb", "alpha", "depth_acc"):
        assert torch.equal(out1[k], out2[k]), k
    c2.close()
