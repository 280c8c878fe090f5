"""Detail-level assets for serving (Sec. 3.4): a synthetic stand-in for the trained levels.

The paper trains its levels (Sec. 3.4.1, budgets B_1 < B_2 < B_3) and selects one per partition
by camera distance at render time (Sec. 3.4.2). Without data or training, coarser levels are
made here from a finer scene by opacity-weighted merging over a voxel grid, and the levels are
laid out the way gsr_select_lod reads them: concatenated coarsest first, each sorted by
partition, with per-partition boxes and per-level offsets.
"""
from __future__ import annotations

import dataclasses
import math

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


def merge_to_count(scene: Scene, target: int, extent: float = 1000.0, iters: int = 40, rel_tol: float = 0.02,
                   device=None) -> Scene:
    """Opacity-weighted merging over a voxel grid, voxel size searched (geometric bisection,
    stopping within rel_tol of the target) so that about `target` voxels are occupied. Per voxel
    with weights w_i = o_i: mean = sum w mu / sum w; covariance = sum w (Sigma_i + (mu_i - mean)
    (mu_i - mean)^T) / sum w (eigendecomposed into rotation and scales); SH = sum w sh / sum w;
    opacity = 1 - prod(1 - o_i), at most 0.99. Runs with torch on `device` (the GPU when there
    is one: a 20M-Gaussian level takes seconds there)."""
    import torch
    dev = torch.device(device or ("cuda" if torch.cuda.is_available() else "cpu"))
    f64 = torch.float64
    mu = torch.as_tensor(np.asarray(scene.means, np.float64), device=dev)
    lo = mu.min(dim=0).values

    def keys(size):
        v = torch.floor((mu - lo) / size).long()
        return (v[:, 0] * 1_000_003 + v[:, 1]) * 1_000_033 + v[:, 2]

    a, b = 1e-3, extent
    size = b
    for _ in range(iters):
        mid = math.sqrt(a * b)
        cnt = int(torch.unique(keys(mid)).numel())
        if abs(cnt - target) <= rel_tol * target:
            size = mid
            break
        if cnt > target:
            a = mid
        else:
            b = mid
        size = b
    _, inv = torch.unique(keys(size), return_inverse=True)
    m = int(inv.max().item()) + 1
    w = torch.as_tensor(np.asarray(scene.opacities, np.float64), device=dev).reshape(-1)
    sw = torch.zeros(m, dtype=f64, device=dev).index_add_(0, inv, w).clamp_min(1e-12)
    mean = torch.zeros(m, 3, dtype=f64, device=dev).index_add_(0, inv, w[:, None] * mu) / sw[:, None]
    q = torch.as_tensor(np.asarray(scene.quats, np.float64), device=dev)
    R = torch.as_tensor(_quat_to_rot(q.cpu().numpy()), device=dev) if dev.type == "cpu" else _quat_to_rot_t(q)
    s2 = torch.as_tensor(np.asarray(scene.scales, np.float64), device=dev) ** 2
    cov = torch.einsum("nij,nj,nkj->nik", R, s2, R)
    del R
    d = mu - mean[inv]
    cov += d[:, :, None] * d[:, None, :]
    C = torch.zeros(m, 9, dtype=f64, device=dev).index_add_(0, inv, w[:, None] * cov.reshape(-1, 9))
    del cov, d
    C = (C / sw[:, None]).reshape(m, 3, 3).cpu().numpy()
    evals, evecs = np.linalg.eigh(C)  # on the host (LAPACK): seconds for millions of 3x3 matrices
    evecs[np.linalg.det(evecs) < 0, :, 0] *= -1.0
    scales = torch.as_tensor(np.sqrt(np.maximum(evals, 1e-10)))
    quats = _rot_to_quat(evecs)
    K = np.asarray(scene.sh).shape[1]
    sh = torch.as_tensor(np.asarray(scene.sh, np.float32).reshape(scene.n, -1), device=dev)
    shm = torch.zeros(m, sh.shape[1], dtype=torch.float32, device=dev).index_add_(0, inv, w[:, None].float() * sh)
    shm = shm / sw[:, None].float()
    logt = torch.zeros(m, dtype=f64, device=dev).index_add_(0, inv, torch.log1p(-w.clamp_max(0.999999)))
    opac = torch.clamp(1.0 - torch.exp(logt), max=0.99)
    return Scene(mean.float().cpu().numpy(), scales.float().cpu().numpy(), quats.astype(np.float32),
                 opac.float().cpu().numpy(), shm.reshape(m, K, 3).cpu().numpy(), scene.sh_degree)


def _quat_to_rot_t(q):
    """_quat_to_rot on a torch tensor (same formula, on the tensor's device)."""
    import torch
    q = q / q.norm(dim=1, keepdim=True)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    return torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                        2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                        2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], dim=1).reshape(-1, 3, 3)


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
