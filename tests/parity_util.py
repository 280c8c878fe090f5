"""Helpers shared by the GPU parity tests: run the CUDA path and the FP64 oracle on the same
seeded inputs and put their results side by side."""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2507_23006_gb300 import native, scenes


def opts_pair(antialiased=True, tile_cull=False, bg=(0.0, 0.0, 0.0), save_state=True, absgrad=False):
    return (native.Options(antialiased=antialiased, tile_cull=tile_cull, bg=bg, save_state=save_state,
                           absgrad=absgrad),
            oracle.Opts(antialiased=antialiased, tile_cull=tile_cull, bg=bg))


def gpu_render(ctx, scene, cams, nopts, appearances=None, attr_dtype=torch.float32, sh_dtype=torch.float32):
    g = native.Gaussians.from_scene(scene, attr_dtype=attr_dtype, sh_dtype=sh_dtype)
    out, st = native.render_forward(ctx, g, cams, nopts, appearances=appearances)
    torch.cuda.synchronize()
    return g, out, st


def state_arrays(st):
    """Pulls the binning state to the host: records, (camera, Gaussian) of each record,
    sorted pair values, ranges, n_contrib, T_final."""
    info = st.info()
    V, P, T, NP = info["n_visible"], info["n_pairs"], info["n_tiles"], info["n_pixels"]
    R = native.REC_FLOATS
    rec = st.copy(native.BUF_RECORDS, V * R, torch.float32).cpu().numpy().reshape(V, R)
    own = st.copy(native.BUF_OWNER, V, torch.int32).cpu().numpy().view(np.uint32).astype(np.int64)
    pv = st.copy(native.BUF_PAIR_VALS, P, torch.int32).cpu().numpy().view(np.uint32).astype(np.int64)
    rg = st.copy(native.BUF_RANGES, 2 * T, torch.int32).cpu().numpy().view(np.uint32).astype(np.int64).reshape(T, 2)
    nc = st.copy(native.BUF_N_CONTRIB, NP, torch.int32).cpu().numpy().view(np.uint32).astype(np.int64)
    tf = st.copy(native.BUF_T_FINAL, NP, torch.float32).cpu().numpy()
    cam_of = rec[:, 11].view(np.uint32).astype(np.int64) >> 27 if V else np.zeros(0, np.int64)
    return dict(info=info, rec=rec, cam_of=cam_of, g_of=own, pair_vals=pv, ranges=rg, n_contrib=nc, T_final=tf)


def unpack_rect(rec):
    lo = rec[:, 10].view(np.uint32).astype(np.int64)
    hi = rec[:, 11].view(np.uint32).astype(np.int64)
    return lo & 0xFFFF, lo >> 16, hi & 0xFFFF, (hi >> 16) & 0x7FF, hi >> 27


def gpu_tile_lists(sa, n):
    """Per global tile: list of ids c*n + g in blend order."""
    ids = sa["cam_of"] * n + sa["g_of"]
    lists = {}
    for t, (s, e) in enumerate(sa["ranges"]):
        if e > s:
            lists[t] = ids[sa["pair_vals"][s:e]]
    return lists


def oracle_tile_lists(pairs):
    lists = {}
    if pairs is None or len(pairs) == 0:
        return lists
    t = pairs[:, 0]
    cuts = np.nonzero(np.diff(t))[0] + 1
    for chunk in np.split(np.arange(len(t)), cuts):
        lists[int(t[chunk[0]])] = pairs[chunk, 1]
    return lists


# The gradient bar. Per element, |g - g_ref| <= REL |g_ref| + GROUP_REL rms(group): 1e-3 relative
# plus 1e-3 of the parameter group's RMS. An element whose gradient is a cancelling sum of
# per-pixel contributions (cancellation ratio mag / |g_ref| above CANCEL_RATIO, mag = the sum of
# the contributions' magnitudes from the oracle) can be computed by an FP32 implementation only to
# the accuracy of its terms relative to mag, not to |g_ref|: each term carries the FP32 error of
# its alpha, about 1e-4 of itself at pixel coordinates near 1000 (mean2d is rounded to 1e-4 px,
# and alpha moves by |d sigma / d mean2d| times that near a Gaussian's edge). For those elements
# alone the bar adds CANCEL_REL mag (2.5x the largest such error measured on the full-size scenes).
REL = 1e-3
GROUP_REL = 1e-3
CANCEL_RATIO = 4.0
CANCEL_REL = 5e-4
# relative errors are reported over elements whose |g_ref| is at least this fraction of the RMS
REPORT_FLOOR = 0.1

GRAD_REPORT = []  # one dict per grad_close call of this process (printed by the tests)


def grad_stats(g, ref, mag=None, rel=REL, group_rel=GROUP_REL, cancel_ratio=CANCEL_RATIO, cancel_rel=CANCEL_REL,
               rms=None):
    """Element-wise comparison against the bar above; returns (ok mask, stats dict). rms: the
    group's RMS when ref is only part of the group (default: the RMS of ref)."""
    ref = np.asarray(ref, np.float64).reshape(-1)
    g = np.asarray(g, np.float64).reshape(-1)
    assert g.size == ref.size, (g.size, ref.size)
    if rms is None:
        rms = float(np.sqrt(np.mean(ref ** 2))) if ref.size else 0.0
    err = np.abs(g - ref)
    aref = np.abs(ref)
    strict = rel * aref + group_rel * rms + 1e-12
    ok_strict = err <= strict
    ok = ok_strict.copy()
    n_cancel = 0
    n_widened = 0
    if mag is not None:
        mag = np.asarray(mag, np.float64).reshape(-1)
        cancelling = mag > cancel_ratio * aref
        n_cancel = int(cancelling.sum())
        wide_ok = cancelling & (err <= strict + cancel_rel * mag)
        n_widened = int((wide_ok & ~ok_strict).sum())
        ok = ok_strict | wide_ok
    big = aref >= REPORT_FLOOR * rms
    relerr = err[big] / aref[big] if big.any() else np.zeros(0)
    st = dict(n=int(ref.size), rms=rms, strict_pass=float(ok_strict.mean()) if ref.size else 1.0,
              n_cancelling=n_cancel, n_widened=n_widened, n_fail=int((~ok).sum()),
              max_rel_above_floor=float(relerr.max()) if relerr.size else 0.0,
              frac_rel_above_floor_1e3=float((relerr > 1e-3).mean()) if relerr.size else 0.0,
              max_err_over_mag=(float((err[cancelling] / mag[cancelling]).max()) if n_cancel else 0.0)
              if mag is not None else None)
    return ok, st


def grad_close(g, ref, name, rel=REL, group_rel=GROUP_REL, mag=None, cancel_ratio=CANCEL_RATIO,
               cancel_rel=CANCEL_REL, quiet=False, rms=None):
    """Asserts the gradient bar (see REL ... CANCEL_REL above) element by element and records
    the per-element statistics: the fraction within the strict 1e-3 bar, how many elements are
    cancelling sums and how many of those pass only through the CANCEL_REL mag term, and the
    largest relative error over elements above REPORT_FLOOR of the RMS."""
    ok, st = grad_stats(g, ref, mag, rel, group_rel, cancel_ratio, cancel_rel, rms)
    st["name"] = name
    GRAD_REPORT.append(st)
    if not quiet:
        print(f"\n[grad] {name}: {st['n']} elements, strict-bar pass {st['strict_pass']:.6f}, "
              f"cancelling {st['n_cancelling']}, passed only by the cancellation term {st['n_widened']}, "
              f"max rel err (|ref| >= {REPORT_FLOOR} rms) {st['max_rel_above_floor']:.2e}"
              + (f", max err/mag of cancelling {st['max_err_over_mag']:.2e}" if st['max_err_over_mag'] is not None
                 else ""))
    if not ok.all():
        ref = np.asarray(ref, np.float64).reshape(-1)
        g = np.asarray(g, np.float64).reshape(-1)
        err = np.abs(g - ref)
        idx = np.nonzero(~ok)[0]
        worst = idx[np.argsort(-err[idx])[:5]]
        detail = ", ".join(f"[{i}] gpu {g[i]:.6e} ref {ref[i]:.6e}" for i in worst)
        raise AssertionError(f"{name}: {st['n_fail']} / {st['n']} outside tolerance (ref rms {st['rms']:.3e}): "
                             f"{detail}")


def camera_list(cams):
    return list(cams) if isinstance(cams, (list, tuple)) else [cams]


def mlp_for_camera(mlp, c):
    """The appearance-transform inputs as one camera sees them (its own image embedding)."""
    if mlp is None:
        return None
    return dict(mlp, iemb=np.asarray(mlp["iemb"])[c:c + 1])


def scene_box(n=10_000, seed=0):
    return scenes.box_scene(seed, n), scenes.box_camera()


def scene_box_backward(n=4000, seed=3):
    """The box scene of the backward tests: one Gaussian in 16 is made nearly opaque (opacity
    0.9995) and four times larger, so that the 0.99 clamp of alpha is active at some pixels and
    its zero gradient is exercised (with the scene's sigmoid(N(0, 1)) opacities it never is)."""
    scene, cam = scene_box(n, seed)
    op = np.array(scene.opacities, np.float64)
    sc = np.array(scene.scales, np.float64)
    op[::16] = 0.9995
    sc[::16] *= 4.0
    return scenes.Scene(scene.means, sc, scene.quats, op, scene.sh, scene.sh_degree), cam


def upstream(res, npix, seed, alpha_min=0.05):
    """Upstream gradients [npix, 6] ~ N(0, 1) on rgb, depth_acc, depth_exp and alpha, zero on
    the oracle's marked pixels; depth_exp only where alpha > alpha_min (it is ill-conditioned
    where alpha ~ 0)."""
    rng = np.random.default_rng(seed)
    up = rng.normal(size=(npix, 6))
    up[res.mark.astype(bool)] = 0.0
    up[res.img[:, 5] < alpha_min, 4] = 0.0
    return up


def upstream_on(um, npix, seed, alpha=None, alpha_min=0.05):
    """Upstream gradients ~ N(0, 1) on the pixels um only (zero elsewhere); depth_exp only where
    alpha (the oracle's, per pixel) exceeds alpha_min, or nowhere when alpha is None."""
    up = np.zeros((npix, 6))
    w = np.random.default_rng(seed).normal(size=(um.size, 6))
    if alpha is None:
        w[:, 4] = 0.0
    else:
        w[np.asarray(alpha)[um] <= alpha_min, 4] = 0.0
    up[um] = w
    return up
