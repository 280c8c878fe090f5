"""FP64 central finite differences of the oracle for chosen Gaussians of a large scene (the FD
protocol for gradient parity).

For Gaussian gi only the tiles of its own rectangle see it, so L(theta) - L restricted to those
tiles does not depend on gi's parameters: the difference quotient of L equals that of the sum of
<upstream, outputs> over those tiles' pixels. Those pixels are rendered from the sub-scene of the
Gaussians whose rectangles meet gi's (in their original order, so depth ties resolve the same),
which gives them exactly the full render's values there. A parameter whose + or - step changes a
discrete decision (any pixel's contributor set, clamp or termination, gi's rectangle, visibility
or projection clamps) is dropped and counted.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_2507_23006_gb300 import scenes

GROUPS = (("means", 3), ("scales", 3), ("quats", 4), ("opacities", 1), ("sh", 48))


def tile_pixels(tiles, cam):
    ntx = (cam.width + 15) // 16
    pix = []
    for t in tiles:
        ty, tx = divmod(int(t), ntx)
        for y in range(ty * 16, min(ty * 16 + 16, cam.height)):
            pix.extend(range(y * cam.width + tx * 16, y * cam.width + min(tx * 16 + 16, cam.width)))
    return np.array(pix, np.int64)


class SubScene:
    """The Gaussians whose rectangles meet Gaussian gi's, as FP64 arrays gi's row of which can be
    perturbed."""

    def __init__(self, scene, cam, opts, rec, vis, gi, affine=None):
        x0, x1, y0, y1 = (rec[:, k].astype(np.int64) for k in (11, 12, 13, 14))
        ov = vis[(x0[vis] < x1[gi]) & (x1[vis] > x0[gi]) & (y0[vis] < y1[gi]) & (y1[vis] > y0[gi])]
        self.idx = np.sort(ov)
        self.pos = int(np.searchsorted(self.idx, gi))
        assert self.idx[self.pos] == gi
        ntx = (cam.width + 15) // 16
        self.tiles = np.array([ty * ntx + tx for ty in range(y0[gi], y1[gi]) for tx in range(x0[gi], x1[gi])],
                              np.int64)
        self.pix = tile_pixels(self.tiles, cam)
        self.arr = {k: np.array(getattr(scene, k), np.float64)[self.idx].copy()
                    for k in ("means", "scales", "quats", "opacities", "sh")}
        self.deg = scene.sh_degree
        self.cam = cam
        self.opts = opts
        self.affine = affine

    def scene(self):
        a = self.arr
        return scenes.Scene(a["means"], a["scales"], a["quats"], a["opacities"], a["sh"], self.deg)

    def evaluate(self, up):
        """(L over the sub-scene's tiles, per-pixel decision signatures, gi's projection
        decisions)."""
        sc = self.scene()
        r = oracle.render(sc, [self.cam], self.opts, affines=None if self.affine is None else self.affine[None],
                          tile_subset=self.tiles, want_pairs=False, want_sig=True)
        L = float(np.sum(up[self.pix] * r.img[self.pix, :6]))
        rec, fl = oracle.project(sc, self.cam, self.opts)
        proj = (int(fl[self.pos]), tuple(rec[self.pos, 11:15].astype(np.int64)))
        return L, r.sig[self.pix].copy(), proj


def fd_gradients(scene, cam, opts, up, chosen, affine=None, groups=GROUPS):
    """Central differences (h = 1e-6 max(1, |theta|)) of L = sum <up, outputs> for every
    parameter of every Gaussian in `chosen`. Returns (fd dict group -> [len(chosen), width] with
    NaN where dropped, number of parameters dropped, number computed)."""
    rec, fl = oracle.project(scene, cam, opts)
    vis = np.nonzero(fl & 1)[0]
    out = {k: np.full((len(chosen), w), np.nan) for k, w in groups}
    dropped = 0
    total = 0
    for row, gi in enumerate(chosen):
        sub = SubScene(scene, cam, opts, rec, vis, int(gi), affine)
        _, sig0, proj0 = sub.evaluate(up)
        for name, width in groups:
            arr = sub.arr[name].reshape(len(sub.idx), -1)
            for j in range(min(width, arr.shape[1])):
                th = arr[sub.pos, j]
                h = 1e-6 * max(1.0, abs(th))
                L = []
                same = True
                for sgn in (1.0, -1.0):
                    arr[sub.pos, j] = th + sgn * h
                    Lv, sig, proj = sub.evaluate(up)
                    same &= np.array_equal(sig, sig0) and proj == proj0
                    L.append(Lv)
                arr[sub.pos, j] = th
                total += 1
                if not same:
                    dropped += 1
                    continue
                out[name][row, j] = (L[0] - L[1]) / (2.0 * h)
    return out, dropped, total


def fd_affine(raw_C, T, bg, up, affine, h=1e-6):
    """Central differences of L = sum over pixels of <up_rgb, A C + b (1 - T) + T bg> with
    respect to the 12 entries of [A | b], from the raw colour sums C and final transmittances T
    of a render without the transform."""
    out = np.zeros(12)
    for k in range(12):
        vals = []
        for sgn in (1.0, -1.0):
            A = np.array(affine, np.float64).reshape(3, 4).copy()
            A.reshape(-1)[k] += sgn * h
            rgb = raw_C @ A[:, :3].T + np.outer(1.0 - T, A[:, 3]) + np.outer(T, bg)
            vals.append(float(np.sum(up[:, 0:3] * rgb)))
        out[k] = (vals[0] - vals[1]) / (2.0 * h)
    return out


# ---- the street-block case of the protocol, rebuilt from its recipe by pool workers -----------

def build_case(recipe):
    """(scene, camera, 3x4 transform, oracle options, upstream [npix, 6], oracle render) of the FD
    protocol's case: the seeded 500k street block and its 1920x1080 camera, a per-image transform
    I + N(0, 0.01) (seed aff_seed), upstream N(0, 1) (seed up_seed) on rgb, depth_acc, alpha and
    depth_exp (where alpha > 0.05), zero on the oracle's marked pixels."""
    from tests import parity_util as pu
    scene = scenes.street_block(recipe["seed"], recipe["n"])
    cam = scenes.street_block_camera()
    rng = np.random.default_rng(recipe["aff_seed"])
    aff = np.concatenate([np.eye(3), np.zeros((3, 1))], 1) + rng.normal(0, 0.01, (3, 4))
    opts = oracle.Opts(tile_cull=recipe["tile_cull"])
    res = oracle.render(scene, [cam], opts, affines=aff[None], want_pairs=False)
    up = pu.upstream(res, cam.width * cam.height, seed=recipe["up_seed"])
    return scene, cam, aff, opts, up, res


STREET_RECIPE = dict(seed=1, n=500_000, aff_seed=1, up_seed=3, tile_cull=True)

_W = {}


def _init_worker(recipe):
    scene, cam, aff, opts, up, _ = build_case(recipe)
    oracle.set_num_threads(1)
    _W.update(scene=scene, cam=cam, aff=aff, opts=opts, up=up)


def _run_chunk(chunk):
    return fd_gradients(_W["scene"], _W["cam"], _W["opts"], _W["up"], chunk, affine=_W["aff"])


def fd_gradients_parallel(recipe, chosen, workers=8):
    """fd_gradients for `chosen`, split over a pool of spawned processes (each rebuilds the case
    from its recipe). Returns the same triple, rows in the order of `chosen`."""
    import concurrent.futures as cf
    import multiprocessing as mp
    chunks = [c for c in np.array_split(np.asarray(chosen), workers) if len(c)]
    with cf.ProcessPoolExecutor(max_workers=len(chunks), mp_context=mp.get_context("spawn"),
                                initializer=_init_worker, initargs=(recipe,)) as ex:
        parts = list(ex.map(_run_chunk, chunks))
    out = {k: np.concatenate([p[0][k] for p in parts]) for k, _ in GROUPS}
    return out, sum(p[1] for p in parts), sum(p[2] for p in parts)
