"""Detail-level assets for serving (Sec. 3.4): a synthetic stand-in for the trained levels.

The paper trains its levels (Sec. 3.4.1, budgets B_1 < B_2 < B_3) and selects one per partition
by camera distance at render time (Sec. 3.4.2). Without data or training, coarser levels are
made here from a finer scene by opacity-weighted merging over a voxel grid, and the levels are
laid out the way gsr_select_lod reads them: concatenated coarsest first, each sorted by
partition, with per-partition boxes and per-level offsets.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .scenes import Scene


def _quat_to_rot(q):
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    R = np.empty((q.shape[0], 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z); R[:, 0, 1] = 2 * (x * y - w * z); R[:, 0, 2] = 2 * (x * z + w * y)
    R[:, 1, 0] = 2 * (x * y + w * z); R[:, 1, 1] = 1 - 2 * (x * x + z * z); R[:, 1, 2] = 2 * (y * z - w * x)
    R[:, 2, 0] = 2 * (x * z - w * y); R[:, 2, 1] = 2 * (y * z + w * x); R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def _rot_to_quat(R):
    """Unit quaternions (w, x, y, z) of proper rotation matrices (Shepperd's method)."""
    m = R
    tr = m[:, 0, 0] + m[:, 1, 1] + m[:, 2, 2]
    q = np.empty((R.shape[0], 4))
    cands = np.stack([tr, m[:, 0, 0], m[:, 1, 1], m[:, 2, 2]], axis=1)
    k = np.argmax(cands, axis=1)
    s = np.sqrt(np.maximum(1.0 + 2.0 * np.take_along_axis(cands, k[:, None], 1)[:, 0] - tr, 1e-12)) * 2.0
    i0 = k == 0
    q[i0, 0] = 0.25 * s[i0]
    q[i0, 1] = (m[i0, 2, 1] - m[i0, 1, 2]) / s[i0]
    q[i0, 2] = (m[i0, 0, 2] - m[i0, 2, 0]) / s[i0]
    q[i0, 3] = (m[i0, 1, 0] - m[i0, 0, 1]) / s[i0]
    i1 = k == 1
    q[i1, 0] = (m[i1, 2, 1] - m[i1, 1, 2]) / s[i1]
    q[i1, 1] = 0.25 * s[i1]
    q[i1, 2] = (m[i1, 0, 1] + m[i1, 1, 0]) / s[i1]
    q[i1, 3] = (m[i1, 0, 2] + m[i1, 2, 0]) / s[i1]
    i2 = k == 2
    q[i2, 0] = (m[i2, 0, 2] - m[i2, 2, 0]) / s[i2]
    q[i2, 1] = (m[i2, 0, 1] + m[i2, 1, 0]) / s[i2]
    q[i2, 2] = 0.25 * s[i2]
    q[i2, 3] = (m[i2, 1, 2] + m[i2, 2, 1]) / s[i2]
    i3 = k == 3
    q[i3, 0] = (m[i3, 1, 0] - m[i3, 0, 1]) / s[i3]
    q[i3, 1] = (m[i3, 0, 2] + m[i3, 2, 0]) / s[i3]
    q[i3, 2] = (m[i3, 1, 2] + m[i3, 2, 1]) / s[i3]
    q[i3, 3] = 0.25 * s[i3]
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def merge_to_count(scene: Scene, target: int, extent: float = 1000.0, iters: int = 14) -> Scene:
    """Opacity-weighted merging over a voxel grid, voxel size searched so that about `target`
    voxels are occupied. Per voxel with weights w_i = o_i: mean = sum w mu / sum w; covariance =
    sum w (Sigma_i + (mu_i - mean)(mu_i - mean)^T) / sum w (eigendecomposed into rotation and
    scales); SH = sum w sh / sum w; opacity = 1 - prod(1 - o_i), at most 0.99."""
    mu = np.asarray(scene.means, np.float64)
    lo = mu.min(axis=0)

    def keys(size):
        v = np.floor((mu - lo) / size).astype(np.int64)
        return (v[:, 0] * 1_000_003 + v[:, 1]) * 1_000_033 + v[:, 2]

    a, b = 1e-3, extent
    for _ in range(iters):
        mid = np.sqrt(a * b)
        cnt = np.unique(keys(mid)).size
        if cnt > target:
            a = mid
        else:
            b = mid
    _, inv = np.unique(keys(b), return_inverse=True)
    m = int(inv.max()) + 1
    w = np.asarray(scene.opacities, np.float64)
    sw = np.bincount(inv, weights=w, minlength=m)
    sw = np.maximum(sw, 1e-12)
    mean = np.stack([np.bincount(inv, weights=w * mu[:, k], minlength=m) for k in range(3)], 1) / sw[:, None]
    R = _quat_to_rot(np.asarray(scene.quats, np.float64))
    s2 = np.asarray(scene.scales, np.float64) ** 2
    cov = np.einsum("nij,nj,nkj->nik", R, s2, R)
    d = mu - mean[inv]
    cov = cov + d[:, :, None] * d[:, None, :]
    C = np.zeros((m, 3, 3))
    for i in range(3):
        for j in range(3):
            C[:, i, j] = np.bincount(inv, weights=w * cov[:, i, j], minlength=m) / sw
    evals, evecs = np.linalg.eigh(C)
    evecs[np.linalg.det(evecs) < 0, :, 0] *= -1.0
    scales = np.sqrt(np.maximum(evals, 1e-10))
    quats = _rot_to_quat(evecs)
    sh = np.asarray(scene.sh, np.float64).reshape(scene.n, -1)
    shm = np.stack([np.bincount(inv, weights=w * sh[:, k], minlength=m) for k in range(sh.shape[1])], 1) / sw[:, None]
    logt = np.bincount(inv, weights=np.log1p(-np.minimum(w, 0.999999)), minlength=m)
    opac = np.minimum(1.0 - np.exp(logt), 0.99)
    return Scene(mean.astype(np.float32), scales.astype(np.float32), quats.astype(np.float32),
                 opac.astype(np.float32), shm.reshape(m, -1, 3).astype(np.float32), scene.sh_degree)


@dataclasses.dataclass
class LodScene:
    """Levels concatenated (coarsest first), each sorted by partition, with the index select_lod
    reads: aabb [P,6] and level_offsets [L, P+1] into the concatenated arrays."""
    gaussians: Scene
    aabb: np.ndarray
    level_offsets: np.ndarray
    level_sizes: list


def build_lod(levels, part_size: float = 100.0, extent: float = 1000.0) -> LodScene:
    """levels: Scenes from coarsest to finest. Partitions are a part_size grid over the ground;
    each box spans its Gaussians (means +- 3 max scale) of every level."""
    half = extent / 2.0
    nx = int(np.ceil(extent / part_size))
    P = nx * nx
    parts, orders = [], []
    for sc in levels:
        ij = np.clip(np.floor((np.asarray(sc.means[:, :2], np.float64) + half) / part_size).astype(np.int64), 0, nx - 1)
        p = ij[:, 0] * nx + ij[:, 1]
        orders.append(np.argsort(p, kind="stable"))
        parts.append(p)
    aabb = np.zeros((P, 6))
    aabb[:, :3] = np.inf
    aabb[:, 3:] = -np.inf
    for sc, p in zip(levels, parts):
        r = 3.0 * np.asarray(sc.scales, np.float64).max(axis=1)
        lo = np.asarray(sc.means, np.float64) - r[:, None]
        hi = np.asarray(sc.means, np.float64) + r[:, None]
        for k in range(3):
            np.minimum.at(aabb[:, k], p, lo[:, k])
            np.maximum.at(aabb[:, 3 + k], p, hi[:, k])
    empty = ~np.isfinite(aabb[:, 0])
    aabb[empty] = 0.0
    offsets = np.zeros((len(levels), P + 1), np.int64)
    merged = None
    base = 0
    for l, (sc, p, o) in enumerate(zip(levels, parts, orders)):
        offsets[l, 1:] = base + np.cumsum(np.bincount(p, minlength=P))
        offsets[l, 0] = base
        part = sc.subset(o)
        merged = part if merged is None else merged.concat(part)
        base += sc.n
    return LodScene(merged, aabb, offsets, [sc.n for sc in levels])
