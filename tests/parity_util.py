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


def grad_close(g, ref, name, rel=1e-3, group_rel=1e-3, mag=None):
    """|g - ref| <= rel * ||ref row|| + group_rel * rms(ref) elementwise, where a row is one
    Gaussian's block of the parameter (its mean, scale, quaternion, opacity or SH block): a
    single component of a row can be a near-cancelling sum of large per-pixel terms, so its
    FP32 error scales with the row, not with the component.

    mag (the oracle's magnitude of each element's sum, oracle.backward(want_mag=True)) widens the
    first term to rel * max(||ref row||, mag): where the per-pixel contributions cancel to a
    result far below their own size, FP32 summation is accurate relative to that size only."""
    ref = np.asarray(ref, np.float64)
    g = np.asarray(g, np.float64).reshape(ref.shape)
    rows = ref.reshape(ref.shape[0], -1) if ref.ndim > 1 else ref.reshape(-1, 1)
    row_norm = np.sqrt((rows ** 2).sum(axis=1, keepdims=True))
    row_norm = np.broadcast_to(row_norm, rows.shape).reshape(-1)
    if mag is not None:
        row_norm = np.maximum(row_norm, np.asarray(mag, np.float64).reshape(-1))
    g = g.reshape(-1)
    ref = ref.reshape(-1)
    rms = np.sqrt(np.mean(ref ** 2)) if ref.size else 0.0
    err = np.abs(g - ref)
    bound = rel * row_norm + group_rel * rms + 1e-12
    bad = err > bound
    if bad.any():
        idx = np.nonzero(bad)[0]
        worst = idx[np.argsort(-(err[idx] / bound[idx]))[:5]]
        detail = ", ".join(f"[{i}] gpu {g[i]:.6e} ref {ref[i]:.6e}" for i in worst)
        raise AssertionError(f"{name}: {bad.sum()} / {bad.size} outside tolerance (ref rms {rms:.3e}): {detail}")


def camera_list(cams):
    return list(cams) if isinstance(cams, (list, tuple)) else [cams]


def mlp_for_camera(mlp, c):
    """The appearance-transform inputs as one camera sees them (its own image embedding)."""
    if mlp is None:
        return None
    return dict(mlp, iemb=np.asarray(mlp["iemb"])[c:c + 1])


def scene_box(n=10_000, seed=0):
    return scenes.box_scene(seed, n), scenes.box_camera()
