"""FP64 CPU oracle of the differentiable tile-based Gaussian rasterizer.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package's smoke check and by the
benchmark's CPU-baseline leg, never by the product path. It shares no code with the CUDA
implementation. The arithmetic lives in ``gsr_oracle.cpp`` (plain C++17, double precision,
OpenMP over Gaussians and tiles); this module compiles it with g++ and marshals numpy arrays.

Every function takes float inputs, converts them to float64 exactly and returns float64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gsr_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)
_I32 = ctypes.POINTER(ctypes.c_int32)
_U8 = ctypes.POINTER(ctypes.c_uint8)
_U64 = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (skipped when up to date)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.oracle_project.restype = ctypes.c_int
            L.oracle_project.argtypes = [ctypes.c_int64, _D, _D, _D, _D, _D, ctypes.c_int, ctypes.c_int,
                                         _D, _D, _D, _I32, _D, _D, _D]
            L.oracle_render.restype = ctypes.c_int64
            L.oracle_render.argtypes = [ctypes.c_int64, _D, _D, _D, _D, _D, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, _D, _D, _D, _I64, ctypes.c_int64, _D, _U8, _U64,
                                        _I64, ctypes.c_int64, _U8, _D, _D, _D, _D]
            L.oracle_backward.restype = ctypes.c_int
            L.oracle_backward.argtypes = [ctypes.c_int64, _D, _D, _D, _D, _D, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D,
                                          _I64, ctypes.c_int64, _D, _D, _D, _D, _D, _D, _D]
            L.oracle_sh_basis.restype = ctypes.c_int
            L.oracle_sh_basis.argtypes = [ctypes.c_int64, _D, ctypes.c_int, _D]
            L.oracle_select_lod.restype = ctypes.c_int
            L.oracle_select_lod.argtypes = [ctypes.c_int, _D, ctypes.c_int, _I64, _D, _D, ctypes.c_int64,
                                            _I32, _I64, _I32, _I64]
            L.oracle_num_threads.restype = ctypes.c_int
            L.oracle_set_mutation.restype = ctypes.c_int
            L.oracle_set_mutation.argtypes = [ctypes.c_int]
            L.oracle_set_num_threads.argtypes = [ctypes.c_int]
            _lib = L
    return _lib


def _p(a, ty):
    return None if a is None else a.ctypes.data_as(ty)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class Opts:
    """Render options: eps2d, antialiased, tile_cull, background."""

    def __init__(self, eps2d=0.3, antialiased=True, tile_cull=False, bg=(0.0, 0.0, 0.0)):
        self.eps2d = eps2d
        self.antialiased = antialiased
        self.tile_cull = tile_cull
        self.bg = tuple(bg)

    def row(self):
        return np.array([self.eps2d, float(self.antialiased), float(self.tile_cull), *self.bg], np.float64)


def _scene_args(scene):
    means = _f64(scene.means)
    scales = _f64(scene.scales)
    quats = _f64(scene.quats)
    opac = _f64(scene.opacities)
    sh = _f64(scene.sh)
    K = int(sh.shape[1]) if sh.ndim == 3 else 1
    return means, scales, quats, opac, sh, K, int(scene.sh_degree)


def _cam_rows(cams):
    return np.ascontiguousarray(np.stack([c.as_row() for c in cams]))


MLP_SIZES = dict(gauss_embed=16, image_embed=32, hidden=32, out=4)


def _mlp_args(mlp, n, C):
    """Appearance transform (Sec. 3.5.1) inputs -> (gemb [n,16], iemb [C,32], params [1700]) or
    Nones. mlp: dict(gemb [n,16], iemb [C,32], w1 [32,48], b1 [32], w2 [4,32], b2 [4])."""
    if mlp is None:
        return None, None, None
    gemb = _f64(mlp["gemb"]).reshape(n, 16)
    iemb = _f64(mlp["iemb"]).reshape(C, 32)
    params = np.ascontiguousarray(np.concatenate([_f64(mlp["w1"]).reshape(-1), _f64(mlp["b1"]).reshape(-1),
                                                  _f64(mlp["w2"]).reshape(-1), _f64(mlp["b2"]).reshape(-1)]))
    assert params.size == 32 * 48 + 32 + 4 * 32 + 4
    return gemb, iemb, params


MUTATIONS = {1: "alpha clamp mask dropped", 2: "degree-2 SH band sign flipped",
             3: "depth term of dL/dalpha left out", 4: "conic a and c gradients swapped"}


class mutation:
    """Context manager for tests: the oracle's gradients carry one known mistake (MUTATIONS)
    inside the block, so a test can show that a parity bar would catch it."""

    def __init__(self, k: int):
        self.k = int(k)

    def __enter__(self):
        self.prev = lib().oracle_set_mutation(self.k)
        return self

    def __exit__(self, *exc):
        lib().oracle_set_mutation(self.prev)
        return False


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def set_num_threads(k: int) -> None:
    lib().oracle_set_num_threads(int(k))


def project(scene, cam, opts: Opts | None = None, mlp=None):
    """Per-Gaussian projection for one camera -> (rec [n,16], flags [n]). With mlp (see
    _mlp_args; its image embedding is the camera's), colour and opacity are transformed."""
    opts = opts or Opts()
    means, scales, quats, opac, sh, K, deg = _scene_args(scene)
    n = means.shape[0]
    rec = np.zeros((n, 16), np.float64)
    flags = np.zeros(n, np.int32)
    gemb, iemb, params = _mlp_args(mlp, n, 1)
    rc = lib().oracle_project(n, _p(means, _D), _p(scales, _D), _p(quats, _D), _p(opac, _D), _p(sh, _D),
                              K, deg, _p(_cam_rows([cam]), _D), _p(opts.row(), _D), _p(rec, _D),
                              _p(flags, _I32), _p(gemb, _D), _p(iemb, _D), _p(params, _D))
    if rc != 0:
        raise ValueError("oracle_project: invalid arguments")
    return rec, flags


# Reasons of a pixel's knife-edge mark (bits of RenderResult.mark). MARK_SOFT: only a near-tie
# in depth order whose swap cannot move the pixel's outputs by 1e-5 (the gradients and the list
# positions of the swapped contributors still depend on it).
MARK_EDGE, MARK_ALPHA_MIN, MARK_ALPHA_MAX, MARK_STOP, MARK_TIE, MARK_TILE, MARK_SOFT = 1, 2, 4, 8, 16, 32, 64


class RenderResult:
    def __init__(self, img, mark, sig, pairs, gmark, cams, bound=None):
        self.img = img          # [sum HW, 8]
        self.bound = bound      # [sum HW, 3] or None: largest change of rgb / depth_acc / alpha the
                                # marked decisions could make (MARK_TILE excepted)
        self.mark = mark        # [sum HW] uint8: reasons (MARK_*) a decision is within FP32 reach, 0 if none
        self.sig = sig          # [sum HW] uint64
        self.pairs = pairs      # [P, 2] int64 (global tile, c*n+g)
        self.gmark = gmark      # [C*n] uint8
        self.cams = cams

    def split(self, c):
        """Per-camera views: dict of rgb [H,W,3], depth_acc, depth_exp, alpha, T, n_contrib, mark."""
        off = 0
        for k, cam in enumerate(self.cams):
            hw = cam.width * cam.height
            if k == c:
                im = self.img[off:off + hw].reshape(cam.height, cam.width, 8)
                return dict(rgb=im[..., 0:3], depth_acc=im[..., 3], depth_exp=im[..., 4], alpha=im[..., 5],
                            T=im[..., 6], n_contrib=im[..., 7],
                            mark=self.mark[off:off + hw].reshape(cam.height, cam.width))
            off += hw
        raise IndexError(c)


def render(scene, cams, opts: Opts | None = None, affines=None, tile_subset=None, want_pairs=True,
           want_sig=False, mlp=None, want_bound=False) -> RenderResult:
    """Forward render of a list of cameras, packed one after another (mlp: the appearance
    transform's inputs, see _mlp_args)."""
    opts = opts or Opts()
    if not isinstance(cams, (list, tuple)):
        cams = [cams]
    means, scales, quats, opac, sh, K, deg = _scene_args(scene)
    n = means.shape[0]
    C = len(cams)
    rows = _cam_rows(cams)
    aff = None if affines is None else _f64(affines).reshape(C, 12)
    npix = sum(c.width * c.height for c in cams)
    img = np.zeros((npix, 8), np.float64)
    mark = np.zeros(npix, np.uint8)
    sig = np.zeros(npix, np.uint64) if want_sig else None
    gmark = np.zeros(C * n, np.uint8)
    bound = np.zeros((npix, 3), np.float64) if want_bound else None
    sub = None if tile_subset is None else np.ascontiguousarray(np.asarray(tile_subset, np.int64))
    nsub = 0 if sub is None else sub.size
    gemb, iemb, params = _mlp_args(mlp, n, C)
    margs = (_p(gemb, _D), _p(iemb, _D), _p(params, _D))
    args = (n, _p(means, _D), _p(scales, _D), _p(quats, _D), _p(opac, _D), _p(sh, _D), K, deg, C,
            _p(rows, _D), _p(aff, _D), _p(opts.row(), _D), _p(sub, _I64), nsub)
    # first call sizes the pair list
    P = lib().oracle_render(*args, _p(img, _D), _p(mark, _U8), _p(sig, _U64), None, 0, _p(gmark, _U8), *margs,
                            _p(bound, _D))
    if P < 0:
        raise ValueError("oracle_render: invalid arguments")
    pairs = None
    if want_pairs:
        pairs = np.zeros((max(P, 1), 2), np.int64)
        P2 = lib().oracle_render(n, _p(means, _D), _p(scales, _D), _p(quats, _D), _p(opac, _D), _p(sh, _D),
                                 K, deg, C, _p(rows, _D), _p(aff, _D), _p(opts.row(), _D),
                                 _p(np.zeros(1, np.int64), _I64), 0, _p(np.zeros((1, 8)), _D), None, None,
                                 _p(pairs, _I64), pairs.shape[0], None, *margs, None)
        assert P2 == P
        pairs = pairs[:P]
    return RenderResult(img, mark, sig, pairs, gmark, list(cams), bound)


def backward(scene, cams, up_grads, opts: Opts | None = None, affines=None, want_g2d=False, tile_subset=None,
             want_mag=False, mlp=None):
    """Analytic gradients of L = <up_grads, outputs>; up_grads is [sum HW, 6]
    (d rgb 3, d depth_acc, d depth_exp, d alpha). Returns a dict of float64 arrays. With
    want_mag, out["mag"] holds, per gradient array, the magnitude of each element's sum (the
    pixels' contributions in absolute value through the absolute Jacobian): |gradient| <= mag."""
    opts = opts or Opts()
    if not isinstance(cams, (list, tuple)):
        cams = [cams]
    means, scales, quats, opac, sh, K, deg = _scene_args(scene)
    n = means.shape[0]
    C = len(cams)
    rows = _cam_rows(cams)
    aff = None if affines is None else _f64(affines).reshape(C, 12)
    up = _f64(up_grads).reshape(-1, 6)
    out = dict(means=np.zeros((n, 3)), scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
               opacities=np.zeros(n), sh=np.zeros((n, K, 3)), affine=np.zeros((C, 12)),
               absgrad=np.zeros((n, 2)))
    g2d = np.zeros((C * n, 12)) if want_g2d else None
    mag = np.zeros((n, 11 + 3 * K)) if want_mag else None
    gemb, iemb, params = _mlp_args(mlp, n, C)
    g_gemb = np.zeros((n, 16)) if mlp is not None else None
    g_iemb = np.zeros((C, 32)) if mlp is not None else None
    g_mlp = np.zeros(params.size) if mlp is not None else None
    sub = None if tile_subset is None else np.ascontiguousarray(np.asarray(tile_subset, np.int64))
    nsub = 0 if sub is None else sub.size
    rc = lib().oracle_backward(n, _p(means, _D), _p(scales, _D), _p(quats, _D), _p(opac, _D), _p(sh, _D), K, deg,
                               C, _p(rows, _D), _p(aff, _D), _p(opts.row(), _D), _p(up, _D),
                               _p(out["means"], _D), _p(out["scales"], _D), _p(out["quats"], _D),
                               _p(out["opacities"], _D), _p(out["sh"], _D), _p(out["affine"], _D),
                               _p(out["absgrad"], _D), _p(g2d, _D), _p(sub, _I64), nsub, _p(mag, _D),
                               _p(gemb, _D), _p(iemb, _D), _p(params, _D), _p(g_gemb, _D), _p(g_iemb, _D),
                               _p(g_mlp, _D))
    if rc != 0:
        raise ValueError("oracle_backward: invalid arguments")
    if want_g2d:
        out["g2d"] = g2d
    if mlp is not None:
        w1n, b1n, w2n = 32 * 48, 32, 4 * 32
        out["mlp"] = dict(gemb=g_gemb, iemb=g_iemb, w1=g_mlp[:w1n].reshape(32, 48), b1=g_mlp[w1n:w1n + b1n],
                          w2=g_mlp[w1n + b1n:w1n + b1n + w2n].reshape(4, 32), b2=g_mlp[w1n + b1n + w2n:])
    if want_mag:
        out["mag"] = dict(means=mag[:, 0:3], scales=mag[:, 3:6], quats=mag[:, 6:10], opacities=mag[:, 10],
                          sh=mag[:, 11:].reshape(n, K, 3))
    return out


def sh_basis(dirs, deg=3):
    dirs = _f64(dirs).reshape(-1, 3)
    out = np.zeros((dirs.shape[0], 16))
    rc = lib().oracle_sh_basis(dirs.shape[0], _p(dirs, _D), int(deg), _p(out, _D))
    if rc != 0:
        raise ValueError("oracle_sh_basis: bad degree")
    return out


def select_lod(aabb, level_offsets, cam, thresholds, budget=0):
    """Partition-level LOD selection -> (status, levels [P], segments [nsegs,2], n_selected)."""
    aabb = _f64(aabb).reshape(-1, 6)
    P = aabb.shape[0]
    lo = np.ascontiguousarray(np.asarray(level_offsets, np.int64))
    L = lo.shape[0]
    assert lo.shape == (L, P + 1)
    thr = _f64(thresholds).reshape(-1)
    assert thr.size == L - 1 or (L == 1)
    if thr.size == 0:
        thr = np.zeros(1)
    levels = np.zeros(P, np.int32)
    segs = np.zeros((max(P, 1), 2), np.int64)
    ns = np.zeros(1, np.int32)
    nsel = np.zeros(1, np.int64)
    st = lib().oracle_select_lod(P, _p(aabb, _D), L, _p(lo, _I64), _p(_cam_rows([cam]), _D), _p(thr, _D),
                                 int(budget), _p(levels, _I32), _p(segs, _I64), _p(ns, _I32), _p(nsel, _I64))
    if st < 0:
        raise ValueError("oracle_select_lod: invalid arguments")
    return st, levels, segs[:ns[0]], int(nsel[0])
