"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed form, an
invariant, a quadrature identity, an independent brute force, or finite differences.
"""
import math

import numpy as np
import pytest

import oracle
import oracle.brute as brute
from paper_2507_23006_gb300 import scenes

Y00 = 1.0 / (2.0 * math.sqrt(math.pi))


def make_scene(means, scales, quats=None, opac=None, dc=None, deg=0):
    means = np.asarray(means, np.float64).reshape(-1, 3)
    n = means.shape[0]
    scales = np.asarray(scales, np.float64)
    scales = np.broadcast_to(scales[:, None] if scales.ndim == 1 and scales.size == n and n != 3 else scales,
                             (n, 3)).copy()
    quats = np.tile([1.0, 0, 0, 0], (n, 1)) if quats is None else np.asarray(quats, np.float64).reshape(n, 4)
    opac = np.full(n, 0.5) if opac is None else np.broadcast_to(np.asarray(opac, np.float64), (n,)).copy()
    sh = np.zeros((n, 16, 3))
    if dc is not None:
        sh[:, 0, :] = np.broadcast_to(np.asarray(dc, np.float64), (n, 3))
    return scenes.Scene(means, scales, quats, opac, sh, deg)


CAM64 = scenes.box_camera(64, 64, f=100.0)


# --- projection: closed forms (Sec. 3.1 projection, Sec. 3.5.4 filter) ------------------------

@pytest.mark.parametrize("aa", [False, True])
def test_isotropic_on_axis(aa):
    s, z, f, eps = 0.07, 4.0, 100.0, 0.3
    sc = make_scene([[0, 0, z]], s, opac=0.6, dc=[0.3, -0.2, 0.1])
    rec, flags = oracle.project(sc, CAM64, oracle.Opts(antialiased=aa))
    assert flags[0] & 1
    var = (f * s / z) ** 2
    np.testing.assert_allclose(rec[0, 0:2], [32.0, 32.0], rtol=0, atol=1e-12)
    np.testing.assert_allclose(rec[0, 2:5], [1 / (var + eps), 0.0, 1 / (var + eps)], rtol=1e-12, atol=1e-15)
    comp = var / (var + eps) if aa else 1.0   # sqrt(det raw / det dilated) for an isotropic splat
    np.testing.assert_allclose(rec[0, 5], 0.6 * comp, rtol=1e-12)
    # lambda_max = m + sqrt(max(0.1, m^2 - det)); isotropic: m^2 - det = 0
    lam = var + eps + math.sqrt(0.1)
    assert rec[0, 10] == math.ceil(3 * math.sqrt(lam))
    # degree-0 colour is view independent: 0.5 + Y00 * dc, clamped at 0
    np.testing.assert_allclose(rec[0, 6:9], np.maximum(0, 0.5 + Y00 * np.array([0.3, -0.2, 0.1])), rtol=1e-12)
    assert rec[0, 9] == z


def test_axis_aligned_anisotropic_off_axis():
    f, eps = 100.0, 0.3
    x, y, z = 0.4, -0.3, 3.0
    sx, sy, sz = 0.05, 0.11, 0.23
    sc = make_scene([[x, y, z]], [sx, sy, sz])
    rec, _ = oracle.project(sc, CAM64, oracle.Opts(antialiased=False))
    # J rows (f/z, 0, -f x/z^2), (0, f/z, -f y/z^2) applied to diag(sx^2, sy^2, sz^2)
    a = (f / z) ** 2 * sx ** 2 + (f * x / z ** 2) ** 2 * sz ** 2 + eps
    b = (f * x / z ** 2) * (f * y / z ** 2) * sz ** 2
    c = (f / z) ** 2 * sy ** 2 + (f * y / z ** 2) ** 2 * sz ** 2 + eps
    det = a * c - b * b
    np.testing.assert_allclose(rec[0, 2:5], [c / det, -b / det, a / det], rtol=1e-12)
    np.testing.assert_allclose(rec[0, 0:2], [f * x / z + 32, f * y / z + 32], rtol=1e-14)


def test_quaternion_convention():
    # (w, x, y, z) = (cos 45, 0, 0, sin 45): +90 degrees about z maps the x axis to the y axis,
    # so a Gaussian long in its local x becomes long in world y.
    h = math.sqrt(0.5)
    sc = make_scene([[0, 0, 4.0]], [0.21, 0.05, 0.05], quats=[[h, 0, 0, h]])
    rec, _ = oracle.project(sc, CAM64, oracle.Opts(antialiased=False, eps2d=0.0))
    var_long = (100 * 0.21 / 4) ** 2
    var_short = (100 * 0.05 / 4) ** 2
    np.testing.assert_allclose(rec[0, 2:5], [1 / var_short, 0.0, 1 / var_long], rtol=1e-10, atol=1e-12)
    # unnormalised quaternions give the same splat
    sc2 = make_scene([[0, 0, 4.0]], [0.21, 0.05, 0.05], quats=[[3 * h, 0, 0, 3 * h]])
    rec2, _ = oracle.project(sc2, CAM64, oracle.Opts(antialiased=False, eps2d=0.0))
    np.testing.assert_allclose(rec2, rec, rtol=1e-13, atol=1e-14)


def test_culling_rules():
    # behind the camera, beyond far, zero quaternion, non-finite -> culled; far off-screen -> culled
    sc = make_scene([[0, 0, -1.0], [0, 0, 2e10], [0, 0, 3.0], [0, 0, 3.0], [100.0, 0, 3.0]], 0.1,
                    quats=[[1, 0, 0, 0], [1, 0, 0, 0], [0, 0, 0, 0], [np.nan, 0, 0, 0], [1, 0, 0, 0]])
    _, flags = oracle.project(sc, CAM64)
    assert not np.any(flags & 1)


def test_rect_rule():
    # r = ceil(3 sqrt(lambda)), rectangle [floor((m - r)/16), floor((m + r + 15)/16)) clamped
    sc = make_scene([[0.0, 0.0, 4.0]], 0.04)
    rec, _ = oracle.project(sc, CAM64, oracle.Opts(antialiased=False))
    r = rec[0, 10]
    m = 32.0
    x0 = max(0, math.floor((m - r) / 16))
    x1 = min(4, math.floor((m + r + 15) / 16))
    assert rec[0, 11:15].tolist() == [x0, x1, x0, x1]
    assert rec[0, 15] == (x1 - x0) ** 2


# --- compositing: closed forms (Eq. 2) ----------------------------------------------------------

@pytest.mark.parametrize("aa", [False, True])
def test_single_gaussian_image(aa):
    s, z, f, eps, o = 0.06, 4.0, 100.0, 0.3, 0.8
    dc = np.array([0.4, 0.1, -0.3])
    sc = make_scene([[0.05, -0.02, z]], s, opac=o, dc=dc)
    res = oracle.render(sc, [CAM64], oracle.Opts(antialiased=aa)).split(0)
    x_w, y_w = 0.05, -0.02
    # isotropic Sigma = s^2 I through J rows (f/z, 0, -f x/z^2), (0, f/z, -f y/z^2)
    ar = (f / z) ** 2 * s * s + (f * x_w / z ** 2) ** 2 * s * s
    br = (f * x_w / z ** 2) * (f * y_w / z ** 2) * s * s
    cr = (f / z) ** 2 * s * s + (f * y_w / z ** 2) ** 2 * s * s
    a2, b2, c2 = ar + eps, br, cr + eps
    det = a2 * c2 - b2 * b2
    op = o * (math.sqrt((ar * cr - br * br) / det) if aa else 1.0)
    conic = np.array([[c2, -b2], [-b2, a2]]) / det
    mx, my = f * x_w / z + 32, f * y_w / z + 32
    rgb_c = np.maximum(0, 0.5 + Y00 * dc)
    mid = 0.5 * (a2 + c2)
    lam = mid + math.sqrt(max(0.1, mid * mid - det))
    r = math.ceil(3 * math.sqrt(lam))
    tiles = range(max(0, math.floor((mx - r) / 16)), min(4, math.floor((mx + r + 15) / 16)))
    tiles_y = range(max(0, math.floor((my - r) / 16)), min(4, math.floor((my + r + 15) / 16)))
    exp_a = np.zeros((64, 64))
    for y in range(64):
        for x in range(64):
            if x // 16 not in tiles or y // 16 not in tiles_y:
                continue
            d = np.array([mx - x - 0.5, my - y - 0.5])
            a = min(0.99, op * math.exp(-0.5 * d @ conic @ d))
            if a >= 1 / 255:
                exp_a[y, x] = a
    np.testing.assert_allclose(res["alpha"], exp_a, rtol=0, atol=1e-13)
    np.testing.assert_allclose(res["rgb"], exp_a[..., None] * rgb_c, rtol=0, atol=1e-13)
    np.testing.assert_allclose(res["depth_acc"], exp_a * z, rtol=0, atol=1e-12)
    np.testing.assert_allclose(res["T"], 1 - exp_a, rtol=0, atol=1e-13)
    # expected depth equals z wherever anything was blended
    np.testing.assert_allclose(res["depth_exp"][exp_a > 0], z, rtol=1e-12)


def test_two_gaussians_over_operator():
    sc = make_scene([[0.0, 0.0, 3.0], [0.01, 0.0, 5.0]], [0.05, 0.08], opac=[0.7, 0.9],
                    dc=[[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    opts = oracle.Opts(antialiased=False)
    res = oracle.render(sc, [CAM64], opts).split(0)
    rec, _ = oracle.project(sc, CAM64, opts)
    y, x = 31, 32
    a = []
    for g in range(2):
        dx, dy = rec[g, 0] - (x + 0.5), rec[g, 1] - (y + 0.5)
        sig = 0.5 * (rec[g, 2] * dx * dx + rec[g, 4] * dy * dy) + rec[g, 3] * dx * dy
        a.append(min(0.99, rec[g, 5] * math.exp(-sig)))
    c1, c2 = rec[0, 6:9], rec[1, 6:9]
    np.testing.assert_allclose(res["rgb"][y, x], c1 * a[0] + c2 * a[1] * (1 - a[0]), rtol=1e-13)
    np.testing.assert_allclose(res["T"][y, x], (1 - a[0]) * (1 - a[1]), rtol=1e-13)
    np.testing.assert_allclose(res["depth_acc"][y, x], 3.0 * a[0] + 5.0 * a[1] * (1 - a[0]), rtol=1e-13)
    # expected depth (Sec. 3.5.3): the blend weights' mean of the depths, 3 and 5 here
    w0, w1 = a[0], a[1] * (1 - a[0])
    np.testing.assert_allclose(res["depth_exp"][y, x], (3.0 * w0 + 5.0 * w1) / (w0 + w1), rtol=1e-13)
    np.testing.assert_allclose(res["alpha"][y, x], w0 + w1, rtol=1e-13)


@pytest.mark.parametrize("o", [0.5, 0.3, 0.999])
def test_stacked_termination(o):
    # k identical splats centred on pixel (40, 24)'s centre: alpha = min(0.99, o) there. The pixel
    # keeps the m-th splat iff (1 - a)^m >= 1e-4, so m = max{i : (1 - a)^i >= 1e-4}.
    k = 40
    x_w = (40.5 - 32) / 100.0
    y_w = (24.5 - 32) / 100.0
    zs = 2.0 + 0.05 * np.arange(k)
    means = np.stack([x_w * zs, y_w * zs, zs], axis=1)
    sc = make_scene(means, 0.01, opac=o, dc=[0.1, 0.2, 0.3])
    res = oracle.render(sc, [CAM64], oracle.Opts(antialiased=False)).split(0)
    a = min(0.99, o)
    m = max(i for i in range(k + 1) if (1 - a) ** i >= 1e-4)
    assert res["n_contrib"][24, 40] == m
    np.testing.assert_allclose(res["T"][24, 40], (1 - a) ** m, rtol=1e-12)


def test_appearance_affine_identity():
    # c' = A c + b per Gaussian equals A C + b (1 - T) per pixel by linearity of Eq. 2
    sc, cam = scenes.tiny_scene(5, 40, 32, 32)
    rng = np.random.default_rng(0)
    aff = np.concatenate([np.eye(3) + rng.normal(0, 0.1, (3, 3)), rng.normal(0, 0.1, (3, 1))], axis=1)
    plain = oracle.render(sc, [cam]).split(0)
    withA = oracle.render(sc, [cam], affines=aff[None]).split(0)
    expect = plain["rgb"] @ aff[:, :3].T + (1 - plain["T"])[..., None] * aff[:, 3]
    np.testing.assert_allclose(withA["rgb"], expect, rtol=0, atol=1e-13)
    np.testing.assert_array_equal(withA["alpha"], plain["alpha"])


# --- invariants ----------------------------------------------------------------------------------

@pytest.fixture(scope="module")
def mid_scene():
    sc, cam = scenes.tiny_scene(11, 1500, 96, 80, depth=(2.0, 9.0), log_scale_mean=-2.5)
    return sc, cam


def test_weights_telescope(mid_scene):
    # white splats: rgb_out = sum alpha_i T_i must equal 1 - T_final
    sc, cam = mid_scene
    white = scenes.Scene(sc.means, sc.scales, sc.quats, sc.opacities, np.zeros(sc.sh.shape, np.float64), 0)
    white.sh[:, 0, :] = 0.5 / Y00
    res = oracle.render(white, [cam]).split(0)
    for ch in range(3):
        np.testing.assert_allclose(res["rgb"][..., ch], res["alpha"], rtol=0, atol=1e-12)
    assert np.all(res["alpha"] >= 0) and np.all(res["alpha"] < 1)
    assert np.all(res["T"] >= 1e-4 * (1 - 1e-12))


def test_rgb_nonnegative_and_bounds(mid_scene):
    sc, cam = mid_scene
    res = oracle.render(sc, [cam]).split(0)
    assert np.all(res["rgb"] >= 0)
    assert res["n_contrib"].max() > 5


def test_permutation_invariance(mid_scene):
    sc, cam = mid_scene
    perm = np.random.default_rng(3).permutation(sc.n)
    a = oracle.render(sc, [cam]).split(0)
    b = oracle.render(sc.subset(perm), [cam]).split(0)
    for k in ("rgb", "depth_acc", "alpha", "T"):
        np.testing.assert_allclose(a[k], b[k], rtol=0, atol=1e-12)


def test_tile_cull_changes_nothing_but_pairs(mid_scene):
    sc, cam = mid_scene
    a = oracle.render(sc, [cam], oracle.Opts(tile_cull=False))
    b = oracle.render(sc, [cam], oracle.Opts(tile_cull=True))
    for k in ("rgb", "depth_acc", "alpha", "T"):
        np.testing.assert_allclose(a.split(0)[k], b.split(0)[k], rtol=0, atol=1e-12)
    sa = set(map(tuple, a.pairs.tolist()))
    sb = set(map(tuple, b.pairs.tolist()))
    assert sb < sa


def test_batch_equals_single(mid_scene):
    sc, cam = mid_scene
    cam2 = scenes.pinhole(scenes.look_at((1.0, -0.5, -1.0), (0.0, 0.0, 6.0), up=(0, -1, 0)), 64, 48,
                          fx=60.0)
    both = oracle.render(sc, [cam, cam2])
    one = oracle.render(sc, [cam]).split(0)
    two = oracle.render(sc, [cam2]).split(0)
    for k in ("rgb", "depth_acc", "alpha", "T"):
        np.testing.assert_array_equal(both.split(0)[k], one[k])
        np.testing.assert_array_equal(both.split(1)[k], two[k])


def test_pair_lists_are_rect_enumeration_sorted(mid_scene):
    sc, cam = mid_scene
    res = oracle.render(sc, [cam])
    rec, flags = oracle.project(sc, cam)
    tx = (cam.width + 15) // 16
    expect = []
    for g in np.nonzero(flags & 1)[0]:
        x0, x1, y0, y1 = rec[g, 11:15].astype(int)
        for ty in range(y0, y1):
            for txx in range(x0, x1):
                expect.append((ty * tx + txx, np.float32(rec[g, 9]), g))
    expect.sort()
    got = [tuple(p) for p in res.pairs.tolist()]
    assert got == [(t, g) for t, _, g in expect]


# --- spherical harmonics ----------------------------------------------------------------------------

def test_sh_orthonormal_by_quadrature():
    nt, nphi = 24, 48
    xg, wg = np.polynomial.legendre.leggauss(nt)   # exact for polynomials in cos(theta) of degree < 48
    phi = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    ct = np.repeat(xg, nphi)
    w = np.repeat(wg, nphi) * (2 * np.pi / nphi)
    st = np.sqrt(1 - ct ** 2)
    dirs = np.stack([st * np.cos(np.tile(phi, nt)), st * np.sin(np.tile(phi, nt)), ct], axis=1)
    Y = oracle.sh_basis(dirs, 3)
    G = (Y * w[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)
    assert abs(Y[0, 0] - Y00) < 1e-15


def test_sh_matches_independent_polynomials():
    rng = np.random.default_rng(7)
    d = rng.normal(size=(200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = oracle.sh_basis(d, 3)
    B = np.array([brute.sh_poly(*v) for v in d])
    np.testing.assert_allclose(Y, B, atol=1e-14)
    # the common checkpoint layout: Y_1 = (-k y, k z, -k x) with k = sqrt(3 / (4 pi))
    k = math.sqrt(3 / (4 * math.pi))
    np.testing.assert_allclose(Y[:, 1:4], np.stack([-k * d[:, 1], k * d[:, 2], -k * d[:, 0]], 1), atol=1e-15)


# --- whole oracle vs an independent brute force -----------------------------------------------------

@pytest.mark.parametrize("seed,aa,cull,bg,aff", [
    (0, True, False, (0, 0, 0), False),
    (1, False, False, (0.2, 0.1, 0.7), False),
    (2, True, True, (0, 0, 0), True),
    (3, False, True, (1, 1, 1), True),
])
def test_oracle_matches_brute_force(seed, aa, cull, bg, aff):
    sc, cam = scenes.tiny_scene(seed, 45, 32, 32, log_scale_mean=-1.8)
    A = None
    if aff:
        rng = np.random.default_rng(seed)
        A = np.concatenate([np.eye(3) + rng.normal(0, 0.2, (3, 3)), rng.normal(0, 0.2, (3, 1))], axis=1)
    res = oracle.render(sc, [cam], oracle.Opts(antialiased=aa, tile_cull=cull, bg=bg),
                        affines=None if A is None else A[None]).split(0)
    ref = brute.render(sc, cam, aa=aa, tile_cull=cull, bg=bg, affine=A)
    for k in ("rgb", "depth_acc", "alpha", "T"):
        np.testing.assert_allclose(res[k], ref[k], rtol=0, atol=1e-12)
    assert ref["alpha"].max() > 0.3


# --- gradients: FP64 central finite differences ------------------------------------------------------

def _loss(sc, cam, w, opts, aff):
    r = oracle.render(sc, [cam], opts, affines=aff, want_pairs=False, want_sig=True)
    img = r.img
    L = float(np.sum(w * img[:, :6]))
    return L, r.sig.copy()


def _fd_check(sc, cam, opts, aff, n_check, seed, tol=2e-6):
    rng = np.random.default_rng(seed)
    npix = cam.width * cam.height
    w = rng.normal(size=(npix, 6))
    g = oracle.backward(sc, [cam], w, opts, affines=aff)
    L0, sig0 = _loss(sc, cam, w, opts, aff)
    rec0, fl0 = oracle.project(sc, cam, opts)
    # perturb float64 copies: a float32 parameter would round the step h away
    params = {k: np.asarray(v, np.float64).copy() for k, v in
              dict(means=sc.means, scales=sc.scales, quats=sc.quats, opacities=sc.opacities, sh=sc.sh).items()}
    sc = scenes.Scene(params["means"], params["scales"], params["quats"], params["opacities"], params["sh"],
                      sc.sh_degree)
    checked = dropped = 0
    vis = np.nonzero(fl0 & 1)[0]
    for gi in rng.choice(vis, size=min(n_check, vis.size), replace=False):
        for name, arr in params.items():
            flat = arr.reshape(arr.shape[0], -1)[gi]
            nb = (sc.sh_degree + 1) ** 2 * 3 if name == "sh" else flat.size
            for j in range(nb):
                th = float(flat[j])
                h = 1e-6 * max(1.0, abs(th))
                vals = []
                ok = True
                for sgn in (1, -1):
                    p2 = {k: v.copy() for k, v in params.items()}
                    p2[name].reshape(p2[name].shape[0], -1)[gi, j] = th + sgn * h
                    s2 = scenes.Scene(p2["means"], p2["scales"], p2["quats"], p2["opacities"], p2["sh"],
                                      sc.sh_degree)
                    L, sig = _loss(s2, cam, w, opts, aff)
                    rec, fl = oracle.project(s2, cam, opts)
                    if (not np.array_equal(sig, sig0) or not np.array_equal(fl, fl0)
                            or not np.array_equal(rec[:, 10:16], rec0[:, 10:16])):
                        ok = False
                    vals.append(L)
                if not ok:
                    dropped += 1
                    continue
                fd = (vals[0] - vals[1]) / (2 * h)
                an = g[name].reshape(g[name].shape[0], -1)[gi, j]
                scale = np.sqrt(np.mean(g[name] ** 2)) + 1e-12
                assert abs(fd - an) <= tol * (abs(an) + scale) + 1e-7, (name, gi, j, fd, an)
                checked += 1
    return checked, dropped, g, w


@pytest.mark.parametrize("aa,cull,use_aff,deg", [(True, False, False, 3), (False, True, True, 3),
                                                 (True, True, True, 1)])
def test_gradients_match_finite_differences(aa, cull, use_aff, deg):
    sc, cam = scenes.tiny_scene(21 + deg, 24, 32, 32, log_scale_mean=-1.8)
    sc.sh_degree = deg
    opts = oracle.Opts(antialiased=aa, tile_cull=cull, bg=(0.1, 0.2, 0.3))
    aff = None
    if use_aff:
        rng = np.random.default_rng(9)
        aff = np.concatenate([np.eye(3) + rng.normal(0, 0.1, (3, 3)), rng.normal(0, 0.1, (3, 1))], axis=1)[None]
    checked, dropped, g, w = _fd_check(sc, cam, opts, aff, n_check=12, seed=deg)
    assert checked >= 12 * 20 and dropped <= checked // 10
    if use_aff:
        # affine gradient by FD of the whole render
        for j in range(12):
            h = 1e-6
            a1, a2 = aff.copy(), aff.copy()
            a1[0].reshape(-1)[j] += h
            a2[0].reshape(-1)[j] -= h
            fd = (_loss(sc, cam, w, opts, a1)[0] - _loss(sc, cam, w, opts, a2)[0]) / (2 * h)
            an = g["affine"][0, j]
            assert abs(fd - an) <= 1e-6 * (abs(an) + 1.0), (j, fd, an)


def test_colour_gradient_closed_form():
    # dC/dc_i = alpha_i T_i: one splat, degree 0, d rgb_r = 1 at one pixel -> dL/d dc_r = Y00 alpha
    sc = make_scene([[0.0, 0.0, 4.0]], 0.06, opac=0.8, dc=[0.4, 0.1, 0.2])
    opts = oracle.Opts(antialiased=False)
    up = np.zeros((64 * 64, 6))
    y, x = 30, 33
    up[y * 64 + x, 0] = 1.0
    g = oracle.backward(sc, [CAM64], up, opts)
    a = oracle.render(sc, [CAM64], opts).split(0)["alpha"][y, x]
    np.testing.assert_allclose(g["sh"][0, 0, 0], Y00 * a, rtol=1e-12)
    assert g["sh"][0, 0, 1] == 0.0


# --- detail-level selection (Sec. 3.4.2) -------------------------------------------------------------

def _row_partitions(n, size=100.0):
    """n partitions of size x size x 50 along +y, starting at y = 0."""
    aabb = np.array([[0.0, i * size, 0.0, size, (i + 1) * size, 50.0] for i in range(n)])
    return aabb


def test_select_lod_levels_by_distance():
    aabb = _row_partitions(6)
    counts = np.array([[10, 11, 12, 13, 14, 15], [100, 101, 102, 103, 104, 105], [1000, 1001, 1002, 1003, 1004, 1005]])
    lo = np.concatenate([np.zeros((3, 1), np.int64), np.cumsum(counts, axis=1)], axis=1)
    lo[1] += lo[0, -1]
    lo[2] += lo[1, -1]
    # camera at (50, -10, 20) looking along +y: distances to the boxes are 10, 110, 210, ...
    cam = scenes.pinhole(scenes.look_at((50.0, -10.0, 20.0), (50.0, 100.0, 20.0)), 640, 480)
    st, lev, segs, nsel = oracle.select_lod(aabb, lo, cam, [100.0, 200.0])
    assert st == 0
    assert lev.tolist() == [2, 1, 0, 0, 0, 0]
    assert nsel == 1000 + 101 + 12 + 13 + 14 + 15
    assert segs[0].tolist() == [lo[2, 0], 1000] and segs[1].tolist() == [lo[1, 1], 101]


def test_select_lod_culls_behind_and_budget_demotes_farthest():
    aabb = _row_partitions(4)
    counts = np.array([[5, 5, 5, 5], [50, 50, 50, 50], [500, 500, 500, 500]])
    lo = np.concatenate([np.zeros((3, 1), np.int64), np.cumsum(counts, axis=1)], axis=1)
    lo[1] += lo[0, -1]
    lo[2] += lo[1, -1]
    # camera inside partition 1 looking along +y: partition 0 is behind it (culled)
    cam = scenes.pinhole(scenes.look_at((50.0, 150.0, 20.0), (50.0, 300.0, 20.0)), 640, 480)
    st, lev, _, nsel = oracle.select_lod(aabb, lo, cam, [100.0, 200.0])
    assert lev.tolist() == [-1, 2, 2, 1] and nsel == 1050 and st == 0
    # budget 600: demote partition 3 (farthest) to 0 -> 1005; then 2 -> 1 -> 555
    st, lev, _, nsel = oracle.select_lod(aabb, lo, cam, [100.0, 200.0], budget=600)
    assert lev.tolist() == [-1, 2, 1, 0] and nsel == 555 and st == 0
    # impossible budget: everything visible goes to level 0, warning
    st, lev, _, nsel = oracle.select_lod(aabb, lo, cam, [100.0, 200.0], budget=3)
    assert lev.tolist() == [-1, 0, 0, 0] and nsel == 15 and st == 1


@pytest.mark.parametrize("delta,marked", [(5e-6, True), (-5e-6, True), (0.2, False), (-0.2, False)])
def test_rectangle_knife_edge_where_mean2d_cancels(delta, marked):
    """my = fy y/z + cy with the two terms near -535.5 and 533.5: a rectangle bound 5e-6 px from
    an integer is within reach of FP32 rounding (about 1e-4 px here), so the item is marked,
    whichever side of the edge the FP64 value falls; 0.2 px away it is not."""
    fy, cy, z = 1385.640646055102, 533.5, 427.466
    cam = scenes.pinhole(np.hstack([np.eye(3), np.zeros((3, 1))]), 1600, 1067, fx=fy, fy=fy, cx=800.0, cy=cy)
    # radius 3: 3 sqrt(lambda) in (2, 3); the top bound y1 = floor((my + 3 + 15) / 16) sits at 1
    my = -2.0 + delta
    y = (my - cy) * z / fy
    scene = make_scene([[0.0, y, z]], [0.1], opac=[0.9], dc=[0.5])
    rec, flags = oracle.project(scene, cam, oracle.Opts())
    assert rec[0, 10] == 3.0 or not flags[0] & 1  # radius 3 (with the max(0.1, .) floor)
    assert abs(fy * y / z) > 500 and abs(cy) > 500  # the cancelling terms
    assert bool(flags[0] & 2) == marked
    assert bool(flags[0] & 1) == (delta > 0)  # visible only when the FP64 bound reaches row 0


def test_gradient_magnitude_bounds_and_single_pixel_equality():
    """The magnitude returned with the gradient (the per-pixel contributions in absolute value
    through the absolute Jacobian) bounds |gradient| elementwise (triangle inequality), and
    equals it where one pixel of one Gaussian carries the loss and the Jacobian has one term
    per entry (an isotropic Gaussian at the image centre, loss on its centre pixel's alpha)."""
    scene, cam = scenes.box_scene(7, 300), scenes.box_camera(64, 64, f=80.0)
    opts = oracle.Opts(bg=(0.1, 0.2, 0.3))
    res = oracle.render(scene, [cam], opts, want_pairs=False)
    up = np.random.default_rng(1).normal(size=(64 * 64, 6))
    ref = oracle.backward(scene, [cam], up, opts, want_mag=True)
    for k in ("means", "scales", "quats", "opacities", "sh"):
        assert np.all(ref["mag"][k] >= np.abs(ref[k]) * (1 - 1e-12) - 1e-15), k
        assert ref["mag"][k].max() > 0, k
    # one Gaussian, one pixel: the opacity gradient has a single term
    one = make_scene([[0.0, 0.0, 5.0]], [0.3], opac=[0.6], dc=[0.5])
    cam1 = scenes.pinhole(np.hstack([np.eye(3), np.zeros((3, 1))]), 16, 16, fx=40.0, fy=40.0, cx=8.0, cy=8.0)
    up1 = np.zeros((256, 6))
    up1[8 * 16 + 8, 5] = 1.0
    r1 = oracle.backward(one, [cam1], up1, oracle.Opts(), want_mag=True)
    np.testing.assert_allclose(r1["mag"]["opacities"], np.abs(r1["opacities"]), rtol=1e-12)
    assert res.img.shape[0] == 64 * 64


def test_absgrad_is_the_sum_over_pixels_of_the_mean2d_gradient_magnitudes():
    """AbsGS (Sec. 3.5.4) accumulates, per Gaussian and image axis, |dL_p / dmean2d| over the
    pixels p, L_p being the loss's part at pixel p. Brute force from that definition: a backward
    with the upstream gradient of one pixel alone gives dL_p / dmean2d (the 2D gradient the oracle
    returns per camera and Gaussian); the magnitudes summed over every pixel must equal the
    statistic, which in turn bounds the full 2D mean gradient, their signed sum."""
    W, H = 24, 20
    sc, cam = scenes.tiny_scene(3, 40, W, H, depth=(2.0, 6.0), log_scale_mean=-2.0)
    opts = oracle.Opts(bg=(0.1, 0.2, 0.3))
    up = np.random.default_rng(4).normal(size=(W * H, 6))
    full = oracle.backward(sc, [cam], up, opts, want_g2d=True)
    per_pixel = np.zeros((sc.n, 2))
    signed = np.zeros((sc.n, 2))
    for p in range(W * H):
        u = np.zeros_like(up)
        u[p] = up[p]
        g2d = oracle.backward(sc, [cam], u, opts, want_g2d=True)["g2d"][:, 0:2]
        per_pixel += np.abs(g2d)
        signed += g2d
    assert (per_pixel > 0).sum() >= sc.n // 2  # most Gaussians reach some pixel
    np.testing.assert_allclose(full["absgrad"], per_pixel, rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(full["g2d"][:, 0:2], signed, rtol=1e-9, atol=1e-12)
    assert np.all(np.abs(full["g2d"][:, 0:2]) <= full["absgrad"] * (1 + 1e-12) + 1e-15)
    # cancelling pixels make the statistic strictly larger than the gradient somewhere
    assert np.any(full["absgrad"] > np.abs(full["g2d"][:, 0:2]) * 1.01 + 1e-12)


# --- appearance transform (Sec. 3.5.1) ---------------------------------------------------------------

def test_appearance_transform_limits():
    """A zero output layer gives sigmoid(0) = 1/2: colour gain 1 and opacity halved, i.e. the
    plain render of the scene with halved opacities; a very negative opacity bias with zero
    colour logits leaves the Gaussian unchanged."""
    sc, cam = scenes.tiny_scene(3, 30, 32, 32, log_scale_mean=-1.8)
    rng = np.random.default_rng(0)
    mlp = scenes.appearance_mlp(rng, sc.n, 1)
    mlp["w2"][:] = 0.0
    mlp["b2"][:] = 0.0
    opts = oracle.Opts(bg=(0.1, 0.2, 0.3))
    half = scenes.Scene(sc.means, sc.scales, sc.quats, np.asarray(sc.opacities, np.float64) * 0.5, sc.sh, 3)
    a = oracle.render(sc, [cam], opts, mlp=mlp, want_pairs=False).img
    b = oracle.render(half, [cam], opts, want_pairs=False).img
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-12)
    mlp["b2"][3] = -60.0  # opacity factor 1 - sigmoid(-60)
    a = oracle.render(sc, [cam], opts, mlp=mlp, want_pairs=False).img
    b = oracle.render(sc, [cam], opts, want_pairs=False).img
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-12)
    assert b[:, 5].max() > 0.3


@pytest.mark.parametrize("aa,cams", [(True, 1), (False, 2)])
def test_appearance_transform_gradients_match_finite_differences(aa, cams):
    """FP64 central differences of L = <w, outputs> over the whole render, for every kind of
    appearance-transform input (Gaussian and image embeddings, both layers' weights and biases)
    and for the geometric and SH parameters of a few Gaussians."""
    sc, cam = scenes.tiny_scene(11, 20, 32, 32, log_scale_mean=-1.8)
    cam_list = [cam] if cams == 1 else [cam, scenes.box_camera(24, 24, f=25.0)]
    rng = np.random.default_rng(1)
    mlp = scenes.appearance_mlp(rng, sc.n, cams)
    opts = oracle.Opts(antialiased=aa, bg=(0.1, 0.2, 0.3))
    npix = sum(c.width * c.height for c in cam_list)
    w = rng.normal(size=(npix, 6))
    g = oracle.backward(sc, cam_list, w, opts, mlp=mlp)

    def loss(m, scene=sc):
        r = oracle.render(scene, cam_list, opts, mlp=m, want_pairs=False, want_sig=True)
        return float(np.sum(w * r.img[:, :6])), r.sig.copy()

    L0, sig0 = loss(mlp)
    checked = 0
    for key, count in (("gemb", 10), ("iemb", 10), ("w1", 16), ("b1", 6), ("w2", 10), ("b2", 4)):
        arr = mlp[key]
        flat_idx = rng.choice(arr.size, size=min(count, arr.size), replace=False)
        an_all = g["mlp"][key].reshape(-1)
        for j in flat_idx:
            h = 1e-6
            vals = []
            for sgn in (1, -1):
                m2 = {k: v.copy() for k, v in mlp.items()}
                m2[key].reshape(-1)[j] += sgn * h
                L, sig = loss(m2)
                assert np.array_equal(sig, sig0)
                vals.append(L)
            fd = (vals[0] - vals[1]) / (2 * h)
            an = an_all[j]
            scale = np.sqrt(np.mean(an_all ** 2)) + 1e-12
            assert abs(fd - an) <= 2e-6 * (abs(an) + scale) + 1e-8, (key, j, fd, an)
            checked += 1
    assert checked >= 50
    # the geometric and SH gradients through the transformed colour and opacity
    params = {k: np.asarray(v, np.float64).copy() for k, v in
              dict(means=sc.means, scales=sc.scales, quats=sc.quats, opacities=sc.opacities, sh=sc.sh).items()}
    for gi in rng.choice(sc.n, size=4, replace=False):
        for name in ("means", "opacities", "sh"):
            flat = params[name].reshape(sc.n, -1)
            for j in range(min(flat.shape[1], 3)):
                vals = []
                h = 1e-6
                for sgn in (1, -1):
                    p2 = {k: v.copy() for k, v in params.items()}
                    p2[name].reshape(sc.n, -1)[gi, j] += sgn * h
                    s2 = scenes.Scene(p2["means"], p2["scales"], p2["quats"], p2["opacities"], p2["sh"], 3)
                    L, sig = loss(mlp, s2)
                    vals.append(L)
                fd = (vals[0] - vals[1]) / (2 * h)
                an = g[name].reshape(sc.n, -1)[gi, j]
                scale = np.sqrt(np.mean(g[name] ** 2)) + 1e-12
                assert abs(fd - an) <= 1e-5 * (abs(an) + scale) + 1e-8, (name, gi, j, fd, an)


def test_flip_bound_covers_the_other_order_of_a_depth_tie():
    """Two overlapping Gaussians at the same depth (a tie, broken by index) with different
    colours: the render with their indices swapped takes the other order. The image difference
    is nonzero, every pixel where it is nonzero is marked, and it stays within the oracle's
    per-pixel bound (the bound the GPU comparison of marked pixels uses); unmarked pixels have a
    zero bound."""
    sc = make_scene([[0.0, 0.0, 5.0], [0.02, 0.01, 5.0]], [0.3, 0.25], opac=[0.7, 0.6],
                    dc=[[0.9, 0.1, 0.4], [0.1, 0.8, 0.2]])
    r1 = oracle.render(sc, [CAM64], want_bound=True)
    r2 = oracle.render(sc.subset(np.array([1, 0])), [CAM64], want_bound=True)
    d_rgb = np.abs(r1.img[:, 0:3] - r2.img[:, 0:3]).max(axis=1)
    d_dep = np.abs(r1.img[:, 3] - r2.img[:, 3])
    d_alp = np.abs(r1.img[:, 5] - r2.img[:, 5])
    assert d_rgb.max() > 1e-3
    changed = d_rgb > 1e-12
    assert np.all(r1.mark[changed] & (oracle.MARK_TIE | oracle.MARK_SOFT))
    assert np.all(d_rgb <= r1.bound[:, 0] * (1 + 1e-9) + 1e-12)
    assert np.all(d_dep <= r1.bound[:, 1] * (1 + 1e-9) + 1e-12)
    assert np.all(d_alp <= r1.bound[:, 2] + 1e-12)
    assert np.all(r1.bound[r1.mark == 0] == 0.0)
