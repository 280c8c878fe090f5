"""Seeded synthetic scenes and cameras.

This module only draws random numbers and builds camera poses; it contains none
of the rasterizer's arithmetic, so both the CUDA path and the CPU oracle can be
fed from it without sharing any of the method.

The scenes stand in for the paper's aerial urban captures (Mega-NeRF Rubble,
UrbanScene3D, JNU-ZH, BigCity; Sec. 4.1), which are not available: 0.04-1 km^2 of
ground plus box-building facades, viewed from aerial or street-level poses.

Attribute recipe shared by every scene (the Gaussian record of Sec. 3.1, Eq. 1):
  * scales   = exp(N(-2.5, 0.5)) per axis (linear, world units)
  * quats    = normalize(N(0, I_4)), stored (w, x, y, z)
  * opacity  = sigmoid(N(0, 1))
  * SH (degree 3, 16 coefficients x RGB): DC ~ N(0.5, 0.3), the other 45 ~ N(0, 0.2)

Camera convention: world->camera 3x4 [R|t], OpenCV axes (+x right, +y down,
+z forward), pinhole fx, fy, cx, cy, image width x height.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SH_COEFFS = 16


@dataclasses.dataclass
class Camera:
    viewmat: np.ndarray  # [3,4] float64 world->camera
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    near: float = 0.01
    far: float = 1e10

    def center(self) -> np.ndarray:
        R = self.viewmat[:, :3]
        t = self.viewmat[:, 3]
        return -R.T @ t

    def as_row(self) -> np.ndarray:
        """Flat float64 row: viewmat(12), fx, fy, cx, cy, width, height, near, far."""
        return np.concatenate([
            np.asarray(self.viewmat, np.float64).reshape(12),
            np.array([self.fx, self.fy, self.cx, self.cy, self.width, self.height,
                      self.near, self.far], np.float64)])


@dataclasses.dataclass
class Scene:
    means: np.ndarray      # [N,3] float32
    scales: np.ndarray     # [N,3] float32 (linear)
    quats: np.ndarray      # [N,4] float32 (w,x,y,z), not normalised
    opacities: np.ndarray  # [N]   float32 in (0,1)
    sh: np.ndarray         # [N,16,3] float32, coefficient-major, RGB innermost
    sh_degree: int = 3

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        return Scene(self.means[idx].copy(), self.scales[idx].copy(), self.quats[idx].copy(),
                     self.opacities[idx].copy(), self.sh[idx].copy(), self.sh_degree)

    def concat(self, other: "Scene") -> "Scene":
        return Scene(np.concatenate([self.means, other.means]),
                     np.concatenate([self.scales, other.scales]),
                     np.concatenate([self.quats, other.quats]),
                     np.concatenate([self.opacities, other.opacities]),
                     np.concatenate([self.sh, other.sh]), self.sh_degree)


def fx_for_hfov(width: int, hfov_deg: float = 60.0) -> float:
    return width / (2.0 * math.tan(math.radians(hfov_deg) / 2.0))


def look_at(eye, target, up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """World->camera [R|t] (OpenCV axes) for a camera at `eye` looking at `target`."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    up = np.asarray(up, np.float64)
    if abs(float(np.dot(f, up))) > 0.999:
        up = np.array([0.0, 1.0, 0.0]) if abs(f[1]) < 0.9 else np.array([1.0, 0.0, 0.0])
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f])
    t = -R @ eye
    return np.concatenate([R, t[:, None]], axis=1)


def pinhole(viewmat, width, height, fx=None, fy=None, cx=None, cy=None,
            near=0.01, far=1e10) -> Camera:
    fx = fx_for_hfov(width) if fx is None else fx
    fy = fx if fy is None else fy
    cx = width / 2.0 if cx is None else cx
    cy = height / 2.0 if cy is None else cy
    return Camera(np.asarray(viewmat, np.float64), float(fx), float(fy), float(cx), float(cy),
                  int(width), int(height), float(near), float(far))


def random_attributes(rng: np.random.Generator, n: int, log_scale_mean=-2.5, log_scale_std=0.5):
    scales = np.exp(rng.normal(log_scale_mean, log_scale_std, size=(n, 3))).astype(np.float32)
    q = rng.normal(0.0, 1.0, size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    quats = q.astype(np.float32)
    opac = (1.0 / (1.0 + np.exp(-rng.normal(0.0, 1.0, size=n)))).astype(np.float32)
    sh = rng.normal(0.0, 0.2, size=(n, SH_COEFFS, 3)).astype(np.float32)
    sh[:, 0, :] = rng.normal(0.5, 0.3, size=(n, 3)).astype(np.float32)
    return scales, quats, opac, sh


def appearance_mlp(rng: np.random.Generator, n: int, n_cams: int, scale: float = 0.3) -> dict:
    """Random inputs of the per-Gaussian appearance transform (Sec. 3.5.1): Gaussian embeddings
    [n,16] and image embeddings [n_cams,32] ~ N(0,1); w1 [32,48], b1 [32], w2 [4,32], b2 [4] ~
    N(0, scale). The draws only, in that order."""
    return dict(gemb=rng.normal(0, 1, (n, 16)), iemb=rng.normal(0, 1, (n_cams, 32)),
                w1=rng.normal(0, scale, (32, 48)), b1=rng.normal(0, scale, 32),
                w2=rng.normal(0, scale, (4, 32)), b2=rng.normal(0, scale, 4))


def box_scene(seed: int = 0, n: int = 10_000) -> Scene:
    """Means uniform in x,y in [-5,5], z in [5,15] in front of an identity camera."""
    rng = np.random.default_rng(seed)
    means = np.stack([rng.uniform(-5, 5, n), rng.uniform(-5, 5, n), rng.uniform(5, 15, n)],
                     axis=1).astype(np.float32)
    scales, quats, opac, sh = random_attributes(rng, n)
    return Scene(means, scales, quats, opac, sh)


def box_camera(width=256, height=256, f=300.0) -> Camera:
    vm = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)
    return pinhole(vm, width, height, fx=f, fy=f, cx=width / 2.0, cy=height / 2.0)


def _place_buildings(rng, count, lo, hi, fmin, fmax, hmin, hmax, max_tries=100_000):
    """Non-overlapping axis-aligned boxes [x0,y0,x1,y1,height] inside [lo,hi]^2."""
    boxes = []
    tries = 0
    while len(boxes) < count and tries < max_tries:
        tries += 1
        w, d = rng.uniform(fmin, fmax, 2)
        x0 = rng.uniform(lo, hi - w)
        y0 = rng.uniform(lo, hi - d)
        b = (x0, y0, x0 + w, y0 + d)
        if all(b[2] <= o[0] or o[2] <= b[0] or b[3] <= o[1] or o[3] <= b[1] for o in boxes):
            boxes.append((*b, rng.uniform(hmin, hmax)))
    return np.array(boxes, np.float64).reshape(-1, 5)


def _facade_points(rng, boxes: np.ndarray, n: int) -> np.ndarray:
    """n points uniform by area over the four walls of each box."""
    if n == 0 or len(boxes) == 0:
        return np.zeros((0, 3), np.float32)
    x0, y0, x1, y1, h = boxes.T
    # walls: 0: y=y0, 1: y=y1 (length x1-x0); 2: x=x0, 3: x=x1 (length y1-y0)
    lx = x1 - x0
    ly = y1 - y0
    areas = np.stack([lx * h, lx * h, ly * h, ly * h], axis=1).reshape(-1)
    wall = rng.choice(areas.size, size=n, p=areas / areas.sum())
    b = wall // 4
    side = wall % 4
    u = rng.uniform(0.0, 1.0, n)
    z = rng.uniform(0.0, 1.0, n) * h[b]
    px = np.where(side < 2, x0[b] + u * lx[b], np.where(side == 2, x0[b], x1[b]))
    py = np.where(side < 2, np.where(side == 0, y0[b], y1[b]), y0[b] + u * ly[b])
    return np.stack([px, py, z], axis=1).astype(np.float32)


def street_block(seed: int = 1, n: int = 500_000) -> Scene:
    """60% on the ground plane z=0 over [-100,100]^2, 40% on the facades of 40 boxes."""
    rng = np.random.default_rng(seed)
    n_ground = int(round(0.6 * n))
    ground = np.stack([rng.uniform(-100, 100, n_ground), rng.uniform(-100, 100, n_ground),
                       np.zeros(n_ground)], axis=1).astype(np.float32)
    boxes = _place_buildings(rng, 40, -100.0, 100.0, 10.0, 30.0, 10.0, 60.0)
    fac = _facade_points(rng, boxes, n - n_ground)
    means = np.concatenate([ground, fac])
    scales, quats, opac, sh = random_attributes(rng, n)
    return Scene(means, scales, quats, opac, sh)


def street_block_camera(width=1920, height=1080) -> Camera:
    return pinhole(look_at((0.0, -30.0, 30.0), (0.0, 0.0, 0.0)), width, height)


def city_boxes(rng, extent=1000.0, block=100.0, street=20.0, hmin=10.0, hmax=80.0):
    half = extent / 2.0
    boxes = []
    nb = int(round(extent / block))
    for i in range(nb):
        for j in range(nb):
            bx0 = -half + i * block + street / 2.0
            by0 = -half + j * block + street / 2.0
            size = block - street
            k = int(rng.integers(3, 7))
            sub = _place_buildings(rng, k, 0.0, size, 10.0, 30.0, hmin, hmax, max_tries=2000)
            sub[:, [0, 2]] += bx0
            sub[:, [1, 3]] += by0
            boxes.append(sub)
    return np.concatenate(boxes)


def city(seed: int = 2, n: int = 6_000_000, extent: float = 1000.0) -> Scene:
    """1x1 km grid of 100 m blocks with 20 m streets, 3-6 buildings per block,
    heights U(10, 80) m; 60% ground, 40% facades."""
    rng = np.random.default_rng(seed)
    half = extent / 2.0
    n_ground = int(round(0.6 * n))
    ground = np.stack([rng.uniform(-half, half, n_ground), rng.uniform(-half, half, n_ground),
                       np.zeros(n_ground)], axis=1).astype(np.float32)
    boxes = city_boxes(rng, extent)
    fac = _facade_points(rng, boxes, n - n_ground)
    means = np.concatenate([ground, fac])
    scales, quats, opac, sh = random_attributes(rng, n)
    return Scene(means, scales, quats, opac, sh)


def aerial_camera(width=1920, height=1080, altitude=150.0, pitch_deg=45.0,
                  target=(0.0, 0.0, 0.0), azimuth_deg=90.0) -> Camera:
    """Camera at `altitude` above the target plane looking at `target` with the given pitch
    below the horizon; azimuth is the direction the camera looks (degrees from +x)."""
    p = math.radians(min(pitch_deg, 89.0))
    a = math.radians(azimuth_deg)
    horiz = altitude / math.tan(p)
    tx, ty, tz = target
    eye = (tx - horiz * math.cos(a), ty - horiz * math.sin(a), tz + altitude)
    return pinhole(look_at(eye, target), width, height)


def city_batch_cameras(seed: int = 2, extent: float = 1000.0):
    """Four 1600x1067 and four 960x640 aerial views at altitude U(80,300) m, looking at a
    uniform ground point in the city with pitch U(30,90) degrees."""
    rng = np.random.default_rng(seed + 1000)
    cams = []
    half = extent / 2.0
    for k in range(8):
        w, h = (1600, 1067) if k < 4 else (960, 640)
        target = (rng.uniform(-half, half), rng.uniform(-half, half), 0.0)
        cams.append(aerial_camera(w, h, altitude=rng.uniform(80, 300),
                                  pitch_deg=rng.uniform(30, 90), target=target,
                                  azimuth_deg=rng.uniform(0, 360)))
    return cams


def large_scene(seed: int = 4, n: int = 30_000_000, extent: float = 1000.0) -> Scene:
    """55% ground, 35% facades, 10% vegetation blobs (clusters of 15 Gaussians around a
    centre, positions N(centre, 1.5 m), log-scales offset by +1 on one random axis)."""
    rng = np.random.default_rng(seed)
    half = extent / 2.0
    n_ground = int(round(0.55 * n))
    n_veg = int(round(0.10 * n)) // 15 * 15
    n_fac = n - n_ground - n_veg
    ground = np.stack([rng.uniform(-half, half, n_ground), rng.uniform(-half, half, n_ground),
                       np.zeros(n_ground)], axis=1).astype(np.float32)
    boxes = city_boxes(rng, extent)
    fac = _facade_points(rng, boxes, n_fac)
    n_clusters = n_veg // 15
    centres = np.stack([rng.uniform(-half, half, n_clusters), rng.uniform(-half, half, n_clusters),
                        rng.uniform(1.0, 8.0, n_clusters)], axis=1)
    veg = (np.repeat(centres, 15, axis=0) + rng.normal(0, 1.5, size=(n_veg, 3))).astype(np.float32)
    means = np.concatenate([ground, fac, veg])
    scales, quats, opac, sh = random_attributes(rng, n)
    axis = rng.integers(0, 3, n_veg)
    scales[n_ground + n_fac + np.arange(n_veg), axis] *= np.float32(math.e)
    return Scene(means, scales, quats, opac, sh)


def street_level_camera(width=3840, height=2160, x=0.0, y=-440.0, height_m=1.7) -> Camera:
    """A street-level camera looking horizontally along +y down a street (x on a street)."""
    eye = (x, y, height_m)
    return pinhole(look_at(eye, (x, y + 100.0, height_m)), width, height)


def tiny_scene(seed: int, n: int, width: int = 32, height: int = 32, depth=(2.0, 6.0),
               log_scale_mean=-2.0, spread=None) -> tuple[Scene, Camera]:
    """A small random scene in front of an identity camera, for brute-force checks."""
    rng = np.random.default_rng(seed)
    f = 0.9 * width
    zs = rng.uniform(depth[0], depth[1], n)
    sx = (0.5 * width / f) if spread is None else spread
    xs = rng.uniform(-1.2, 1.2, n) * sx * zs
    ys = rng.uniform(-1.2, 1.2, n) * (0.5 * height / f) * zs
    means = np.stack([xs, ys, zs], axis=1).astype(np.float32)
    scales, quats, opac, sh = random_attributes(rng, n, log_scale_mean=log_scale_mean)
    cam = box_camera(width, height, f=f)
    return Scene(means, scales, quats, opac, sh), cam



def walkthrough_camera(rng, width, height, extent=1000.0, block=100.0, street=20.0):
    """A street-level camera (1.7-10 m up, pitch within 10 degrees of horizontal) on a street of
    the city grid, looking along the street."""
    half = extent / 2.0
    k = int(rng.integers(0, int(extent / block)))
    along = rng.uniform(-half, half)
    pos = -half + k * block  # streets run along the block boundaries
    hgt = rng.uniform(1.7, 10.0)
    pitch = math.radians(rng.uniform(-10.0, 10.0))
    if rng.uniform() < 0.5:
        eye = np.array([pos, along, hgt])
        fwd = np.array([0.0, rng.choice([-1.0, 1.0]), 0.0])
    else:
        eye = np.array([along, pos, hgt])
        fwd = np.array([rng.choice([-1.0, 1.0]), 0.0, 0.0])
    tgt = eye + 50.0 * fwd + np.array([0.0, 0.0, 50.0 * math.tan(pitch)])
    return pinhole(look_at(eye, tgt), width, height)
