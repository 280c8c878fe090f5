"""Tiny pure-Python brute-force renderer, used only to check the C++ oracle.

TEST INFRASTRUCTURE ONLY. It loops over every pixel and, per pixel, over every Gaussian
(no tile lists, no sort kernel: each pixel sorts its own candidates), so it is meant for
N <= 50 Gaussians and images of at most 32 x 32 pixels.

It follows the same readings of the paper as the C++ oracle but is written independently:
  * Sec. 3.1, Eq. 1: Sigma = R S S^T R^T; projection Sigma2D = J W Sigma W^T J^T + eps I
    (the Jacobian's x/z, y/z clamped to 1.3 of the half field of view), opacity scaled by
    sqrt(det(raw) / det(dilated)) when anti-aliasing is on (Sec. 3.5.4).
  * A Gaussian reaches a pixel only if the pixel's tile lies in its 3-sigma tile rectangle
    (and, with tile culling on, the tile is not culled: Sec. 3.4.2).
  * Sec. 3.1, Eq. 2: front to back in (float32(z), index) order with alpha = min(0.99, o'G'),
    skip alpha < 1/255, stop before the Gaussian that would take T below 1e-4.
  * The SH basis here is the explicit degree <= 3 polynomial table computed from the
    spherical-harmonic normalisation constants K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!).
"""
from __future__ import annotations

import math

import numpy as np

TILE = 16


def _k(l, m):
    m = abs(m)
    return math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - m) / math.factorial(l + m))


def sh_poly(x, y, z):
    """Real SH with Condon-Shortley phase, as explicit polynomials of a unit vector.
    P_l^m below are the associated Legendre functions without the phase, written in x, y, z."""
    s2 = math.sqrt(2.0)
    out = [0.0] * 16
    out[0] = _k(0, 0)
    # l = 1: P_1^0 = z, P_1^1 = sin(theta)
    out[1] = -s2 * _k(1, 1) * y
    out[2] = _k(1, 0) * z
    out[3] = -s2 * _k(1, 1) * x
    # l = 2: P_2^0 = (3z^2-1)/2, P_2^1 = 3 z sin, P_2^2 = 3 sin^2
    out[4] = s2 * _k(2, 2) * 3.0 * (2.0 * x * y)
    out[5] = -s2 * _k(2, 1) * 3.0 * z * y
    out[6] = _k(2, 0) * 0.5 * (3.0 * z * z - 1.0)
    out[7] = -s2 * _k(2, 1) * 3.0 * z * x
    out[8] = s2 * _k(2, 2) * 3.0 * (x * x - y * y)
    # l = 3: P_3^0 = (5z^3-3z)/2, P_3^1 = 1.5 (5z^2-1) sin, P_3^2 = 15 z sin^2, P_3^3 = 15 sin^3
    out[9] = -s2 * _k(3, 3) * 15.0 * (3.0 * x * x * y - y ** 3)
    out[10] = s2 * _k(3, 2) * 15.0 * z * (2.0 * x * y)
    out[11] = -s2 * _k(3, 1) * 1.5 * (5.0 * z * z - 1.0) * y
    out[12] = _k(3, 0) * 0.5 * (5.0 * z ** 3 - 3.0 * z)
    out[13] = -s2 * _k(3, 1) * 1.5 * (5.0 * z * z - 1.0) * x
    out[14] = s2 * _k(3, 2) * 15.0 * z * (x * x - y * y)
    out[15] = -s2 * _k(3, 3) * 15.0 * (x ** 3 - 3.0 * x * y * y)
    return out


def _rot(q):
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _splat(mean, scale, quat, opac, sh, deg, cam, eps, aa):
    V = np.asarray(cam.viewmat, np.float64)
    W, tc = V[:, :3], V[:, 3]
    t = W @ mean + tc
    if not (cam.near < t[2] < cam.far):
        return None
    if not np.linalg.norm(quat) > 0:
        return None
    R = _rot(quat)
    Sig = R @ np.diag(scale ** 2) @ R.T
    Sc = W @ Sig @ W.T
    limx = 1.3 * 0.5 * cam.width / cam.fx
    limy = 1.3 * 0.5 * cam.height / cam.fy
    u = min(max(t[0] / t[2], -limx), limx)
    v = min(max(t[1] / t[2], -limy), limy)
    J = np.array([[cam.fx / t[2], 0, -cam.fx * u / t[2]], [0, cam.fy / t[2], -cam.fy * v / t[2]]])
    S2r = J @ Sc @ J.T
    S2 = S2r + eps * np.eye(2)
    det = np.linalg.det(S2)
    if not det > 0:
        return None
    o = opac
    if aa:
        ratio = np.linalg.det(S2r) / det
        o = opac * math.sqrt(ratio) if ratio > 0 else 0.0
    conic = np.linalg.inv(S2)
    mid = 0.5 * (S2[0, 0] + S2[1, 1])
    lam = mid + math.sqrt(max(0.1, mid * mid - det))
    r = math.ceil(3.0 * math.sqrt(lam))
    mx = cam.fx * t[0] / t[2] + cam.cx
    my = cam.fy * t[1] / t[2] + cam.cy
    tx = (cam.width + TILE - 1) // TILE
    ty = (cam.height + TILE - 1) // TILE

    def cl(vv, hi):
        f = math.floor(vv)
        return 0 if f <= 0 else min(f, hi)
    rect = (cl((mx - r) / TILE, tx), cl((mx + r + TILE - 1) / TILE, tx),
            cl((my - r) / TILE, ty), cl((my + r + TILE - 1) / TILE, ty))
    if (rect[1] - rect[0]) * (rect[3] - rect[2]) <= 0:
        return None
    centre = -W.T @ tc
    d = mean - centre
    d = d / np.linalg.norm(d)
    Y = sh_poly(*d)
    nb = (deg + 1) ** 2
    rgb = np.array([max(0.0, 0.5 + sum(sh[k, ch] * Y[k] for k in range(nb))) for ch in range(3)])
    return dict(m=np.array([mx, my]), conic=conic, o=o, rgb=rgb, z=t[2], rect=rect)


def _tile_kept(s, cam, tx, ty):
    """StopThePop test by dense search over the tile's pixel centres (max alpha >= 1/255)."""
    best = -1.0
    for y in range(ty * TILE, min((ty + 1) * TILE, cam.height)):
        for x in range(tx * TILE, min((tx + 1) * TILE, cam.width)):
            d = s["m"] - np.array([x + 0.5, y + 0.5])
            best = max(best, s["o"] * math.exp(-0.5 * d @ s["conic"] @ d))
    return best >= 1.0 / 255.0


def render(scene, cam, eps=0.3, aa=True, tile_cull=False, bg=(0.0, 0.0, 0.0), affine=None):
    """Returns a dict with rgb [H,W,3], depth_acc, alpha, T, n_contrib (list positions walked
    in the pixel's own candidate list; only comparable when nothing is tile-culled)."""
    n = scene.means.shape[0]
    sp = []
    for g in range(n):
        s = _splat(np.asarray(scene.means[g], np.float64), np.asarray(scene.scales[g], np.float64),
                   np.asarray(scene.quats[g], np.float64), float(scene.opacities[g]),
                   np.asarray(scene.sh[g], np.float64), scene.sh_degree, cam, eps, aa)
        sp.append(s)
    A = np.eye(3) if affine is None else np.asarray(affine, np.float64).reshape(3, 4)[:, :3]
    b = np.zeros(3) if affine is None else np.asarray(affine, np.float64).reshape(3, 4)[:, 3]
    H, Wd = cam.height, cam.width
    rgb = np.zeros((H, Wd, 3))
    dep = np.zeros((H, Wd))
    alp = np.zeros((H, Wd))
    Tf = np.zeros((H, Wd))
    kept = {}
    for y in range(H):
        for x in range(Wd):
            tx, ty = x // TILE, y // TILE
            cand = []
            for g, s in enumerate(sp):
                if s is not None and tile_cull and (g, tx, ty) not in kept:
                    kept[(g, tx, ty)] = _tile_kept(s, cam, tx, ty)
                if s is None:
                    continue
                x0, x1, y0, y1 = s["rect"]
                if not (x0 <= tx < x1 and y0 <= ty < y1):
                    continue
                if tile_cull and not kept[(g, tx, ty)]:
                    continue
                cand.append((np.float32(s["z"]), g))
            cand.sort()
            T = 1.0
            C = np.zeros(3)
            D = 0.0
            for _, g in cand:
                s = sp[g]
                d = s["m"] - np.array([x + 0.5, y + 0.5])
                sig = 0.5 * (s["conic"][0, 0] * d[0] ** 2 + s["conic"][1, 1] * d[1] ** 2) + s["conic"][0, 1] * d[0] * d[1]
                if sig < 0:
                    continue
                a = min(0.99, s["o"] * math.exp(-sig))
                if a < 1.0 / 255.0:
                    continue
                Tn = T * (1 - a)
                if Tn < 1e-4:
                    break
                C += (A @ s["rgb"] + b) * a * T
                D += s["z"] * a * T
                T = Tn
            rgb[y, x] = C + T * np.asarray(bg)
            dep[y, x] = D
            alp[y, x] = 1 - T
            Tf[y, x] = T
    return dict(rgb=rgb, depth_acc=dep, alpha=alp, T=Tf)
