"""Python binding of libgsr (include/gsr.h): argument marshalling only.

Every step of rendering runs in the CUDA library; this module converts torch tensors and
camera descriptions into the C structs, passes device pointers and the current CUDA stream,
and raises on any non-OK status. There is no fallback: if libgsr.so cannot be loaded, every
entry point raises.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading
import weakref
from typing import Optional, Sequence

import numpy as np
import torch

from . import build as _build

_lib = None
_lock = threading.Lock()

GSR_OK = 0
GSR_WARN_OVER_BUDGET = 1
STATUS_NAMES = {0: "ok", 1: "over budget", -1: "invalid argument", -2: "out of device memory",
                -3: "CUDA error", -4: "device wait timed out", -5: "unsupported size"}

DTYPES = {torch.float32: 0, torch.float16: 1, torch.bfloat16: 2}

BUF_RECORDS, BUF_OWNER, BUF_PAIR_VALS, BUF_RANGES, BUF_T_FINAL, BUF_N_CONTRIB, BUF_DEPTH_STATE = range(7)
REC_FLOATS = 16  # one splat record: four float4

EXPORTED = [
    "gsr_create", "gsr_destroy", "gsr_status_string", "gsr_last_error", "gsr_workspace_query",
    "gsr_workspace_bytes", "gsr_render_forward", "gsr_render_backward", "gsr_state_release",
    "gsr_state_get_info", "gsr_state_copy", "gsr_sync_check", "gsr_sort_pairs_u32", "gsr_select_lod",
    "gsr_appearance_cache",
    "gsr_profile_enable", "gsr_profile_collect", "gsr_sort_pairs_u32_noalloc", "gsr_profile_select",
    "gsr_param_grads_zero", "gsr_set_wait_limit", "gsr_set_fill_rate", "gsr_set_fill_split",
]

STAGES = ["preprocess", "tile_count", "tile_scan", "readback", "place", "tile_sort", "blend_fwd", "blend_bwd",
          "preprocess_bwd", "between_stages", "appearance_bwd", "depth_sort", "ranges"]
COUNTERS = ["fwd_evals", "fwd_contribs", "bwd_evals", "bwd_contribs", "bwd_warp_iters", "bwd_warp_iters_contrib"]


class GsrError(RuntimeError):
    def __init__(self, status: int, detail: str = ""):
        super().__init__(f"gsr: {STATUS_NAMES.get(status, status)}" + (f": {detail}" if detail else ""))
        self.status = status


class Segment(ctypes.Structure):
    _fields_ = [("begin", ctypes.c_int64), ("count", ctypes.c_int64)]


class CAppearanceMLP(ctypes.Structure):
    _fields_ = [("gauss_embed", ctypes.c_void_p), ("image_embed", ctypes.c_void_p), ("params", ctypes.c_void_p),
                ("cached", ctypes.c_void_p)]


class CGaussians(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("means", ctypes.c_void_p), ("scales", ctypes.c_void_p),
                ("quats", ctypes.c_void_p), ("opacities", ctypes.c_void_p), ("sh", ctypes.c_void_p),
                ("sh_coeffs", ctypes.c_int32), ("sh_degree", ctypes.c_int32), ("attr_dtype", ctypes.c_int32),
                ("sh_dtype", ctypes.c_int32), ("segs", ctypes.POINTER(Segment)), ("nsegs", ctypes.c_int32),
                ("mlp", ctypes.POINTER(CAppearanceMLP)), ("seg_cams", ctypes.POINTER(ctypes.c_uint32))]


class CCamera(ctypes.Structure):
    _fields_ = [("viewmat", ctypes.c_float * 12), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("near_plane", ctypes.c_float), ("far_plane", ctypes.c_float),
                ("appearance", ctypes.c_void_p)]


class COpts(ctypes.Structure):
    _fields_ = [("eps2d", ctypes.c_float), ("antialiased", ctypes.c_int32), ("tile_cull", ctypes.c_int32),
                ("bg", ctypes.c_float * 3), ("save_state", ctypes.c_int32), ("absgrad", ctypes.c_int32),
                ("global_sort", ctypes.c_int32)]


class COutputs(ctypes.Structure):
    _fields_ = [("rgb", ctypes.c_void_p), ("depth_acc", ctypes.c_void_p), ("depth_exp", ctypes.c_void_p),
                ("alpha", ctypes.c_void_p)]


class COutGrads(ctypes.Structure):
    _fields_ = [("rgb", ctypes.c_void_p), ("depth_acc", ctypes.c_void_p), ("depth_exp", ctypes.c_void_p),
                ("alpha", ctypes.c_void_p)]


class CParamGrads(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("scales", ctypes.c_void_p), ("quats", ctypes.c_void_p),
                ("opacities", ctypes.c_void_p), ("sh", ctypes.c_void_p), ("appearance", ctypes.c_void_p),
                ("absgrad", ctypes.c_void_p), ("gauss_embed", ctypes.c_void_p), ("image_embed", ctypes.c_void_p),
                ("mlp_params", ctypes.c_void_p)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class CAllocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", ctypes.c_void_p)]


class TorchAllocator:
    """Backs a context's workspace with PyTorch's caching allocator (gsr_allocator callbacks):
    the library's scratch then shares torch's memory pool and shows in its statistics.
    alloc(bytes, stream) returns a device address or 0 (the library reports GSR_ERR_OOM)."""

    def __init__(self, device: int = 0):
        self.device = int(device)

    def alloc(self, nbytes: int, stream: int) -> int:
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), self.device, int(stream or 0)))
        except RuntimeError:  # torch's out-of-memory error
            return 0

    def free(self, ptr: int, nbytes: int, stream: int) -> None:
        torch.cuda.caching_allocator_delete(int(ptr))


class CStateInfo(ctypes.Structure):
    _fields_ = [("n_render", ctypes.c_int64), ("n_cams", ctypes.c_int32), ("n_visible", ctypes.c_int64),
                ("n_pairs", ctypes.c_int64), ("n_tiles", ctypes.c_int64), ("n_pixels", ctypes.c_int64),
                ("max_tile_pairs", ctypes.c_int64)]


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libgsr.so (building it first if it is missing and a toolkit is present)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise OSError(f"libgsr.so not built ({path}); run paper_2507_23006_gb300.build.build()")
            _build.build()
        L = ctypes.CDLL(path)
        vp = ctypes.c_void_p
        L.gsr_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, vp]
        L.gsr_destroy.argtypes = [vp]
        L.gsr_destroy.restype = None
        L.gsr_status_string.argtypes = [ctypes.c_int]
        L.gsr_status_string.restype = ctypes.c_char_p
        L.gsr_last_error.argtypes = [vp]
        L.gsr_last_error.restype = ctypes.c_char_p
        L.gsr_workspace_query.argtypes = [vp, ctypes.c_int64, ctypes.POINTER(CCamera), ctypes.c_int32, ctypes.c_int64,
                                          ctypes.POINTER(ctypes.c_size_t)]
        L.gsr_workspace_bytes.argtypes = [vp]
        L.gsr_workspace_bytes.restype = ctypes.c_size_t
        L.gsr_render_forward.argtypes = [vp, ctypes.POINTER(CGaussians), ctypes.POINTER(CCamera), ctypes.c_int32,
                                         ctypes.POINTER(COpts), ctypes.POINTER(COutputs), ctypes.POINTER(vp), vp]
        L.gsr_render_backward.argtypes = [vp, ctypes.POINTER(CGaussians), ctypes.POINTER(CCamera), ctypes.c_int32,
                                          ctypes.POINTER(COpts), vp, ctypes.POINTER(COutGrads),
                                          ctypes.POINTER(CParamGrads), vp]
        L.gsr_state_release.argtypes = [vp, vp]
        L.gsr_state_release.restype = None
        L.gsr_state_get_info.argtypes = [vp, ctypes.POINTER(CStateInfo)]
        L.gsr_state_copy.argtypes = [vp, ctypes.c_int32, vp, ctypes.c_size_t, vp]
        L.gsr_sync_check.argtypes = [vp, vp]
        L.gsr_sort_pairs_u32.argtypes = [vp, vp, vp, vp, vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, vp]
        L.gsr_select_lod.argtypes = [ctypes.c_int32, vp, ctypes.c_int32, vp, ctypes.POINTER(CCamera), vp,
                                     ctypes.c_int64, vp, ctypes.POINTER(Segment), ctypes.POINTER(ctypes.c_int32),
                                     ctypes.POINTER(ctypes.c_int64)]
        L.gsr_sort_pairs_u32_noalloc.argtypes = [vp, vp, vp, vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                                 vp, vp]
        L.gsr_profile_enable.argtypes = [vp, ctypes.c_int32, ctypes.c_int32]
        L.gsr_profile_collect.argtypes = [vp, vp, vp, vp]
        L.gsr_profile_select.argtypes = [vp, ctypes.c_uint32]
        L.gsr_param_grads_zero.argtypes = [vp, vp, vp, vp]
        L.gsr_set_wait_limit.argtypes = [vp, ctypes.c_uint32, ctypes.c_int32]
        L.gsr_set_fill_rate.argtypes = [vp, ctypes.c_float, ctypes.c_int32]
        L.gsr_set_fill_split.argtypes = [vp, ctypes.c_float]
        L.gsr_appearance_cache.argtypes = [vp, ctypes.POINTER(CGaussians), ctypes.c_int32, vp, vp]
        for name in EXPORTED:
            getattr(L, name)
        for name in ("gsr_create", "gsr_workspace_query", "gsr_render_forward", "gsr_render_backward",
                     "gsr_state_get_info", "gsr_state_copy", "gsr_sync_check", "gsr_sort_pairs_u32",
                     "gsr_select_lod", "gsr_profile_enable", "gsr_profile_collect",
                     "gsr_sort_pairs_u32_noalloc", "gsr_profile_select", "gsr_param_grads_zero",
                     "gsr_appearance_cache", "gsr_set_wait_limit", "gsr_set_fill_rate",
                     "gsr_set_fill_split"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
        return L


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


MLP_PARAMS = 32 * 48 + 32 + 4 * 32 + 4


@dataclasses.dataclass
class AppearanceMLP:
    """Per-Gaussian appearance transform (Sec. 3.5.1), FP32 device tensors: Gaussian embeddings,
    one image embedding per camera of a launch (in camera order) and the packed weights
    w1 [32,48] | b1 [32] | w2 [4,32] | b2 [4]. Or, for rendering only, `cached`: the outputs of
    every Gaussian for one image embedding (appearance_cache); the other three are then unused."""
    gauss_embed: Optional[torch.Tensor]  # [n,16]
    image_embed: Optional[torch.Tensor]  # [n_cams,32]
    params: Optional[torch.Tensor]       # [1700]
    cached: Optional[torch.Tensor] = None  # [n,4]

    @staticmethod
    def from_arrays(d: dict, device="cuda") -> "AppearanceMLP":
        """From dict(gemb, iemb, w1, b1, w2, b2) of arrays (the layout scenes.appearance_mlp draws)."""
        def t(a):
            return torch.as_tensor(np.ascontiguousarray(a, np.float32)).to(device).contiguous()
        params = np.concatenate([np.asarray(d[k], np.float32).reshape(-1) for k in ("w1", "b1", "w2", "b2")])
        return AppearanceMLP(t(d["gemb"]), t(d["iemb"]), t(params))

    def c_struct(self, n: int) -> CAppearanceMLP:
        if self.cached is not None:
            if tuple(self.cached.shape) != (n, 4) or self.cached.dtype != torch.float32 or not self.cached.is_contiguous():
                raise ValueError("cached must be a contiguous float32 [n, 4] tensor")
            return CAppearanceMLP(None, None, None, _ptr(self.cached))
        for name, a, shape in (("gauss_embed", self.gauss_embed, (n, 16)), ("params", self.params, (MLP_PARAMS,))):
            if tuple(a.shape) != shape:
                raise ValueError(f"{name} must have shape {shape}")
        if self.image_embed.dim() != 2 or self.image_embed.shape[1] != 32:
            raise ValueError("image_embed must have shape [n_cams, 32]")
        for a in (self.gauss_embed, self.image_embed, self.params):
            if a.dtype != torch.float32 or not a.is_contiguous():
                raise ValueError("appearance-transform tensors must be contiguous float32")
        return CAppearanceMLP(_ptr(self.gauss_embed), _ptr(self.image_embed), _ptr(self.params), None)


@dataclasses.dataclass
class Gaussians:
    """Device-resident Gaussians (structure of arrays)."""
    means: torch.Tensor       # [n,3] float32
    scales: torch.Tensor      # [n,3] attribute dtype, linear
    quats: torch.Tensor       # [n,4] attribute dtype (w,x,y,z)
    opacities: torch.Tensor   # [n] attribute dtype
    sh: torch.Tensor          # [n,K,3] sh dtype
    sh_degree: int = 3
    segments: Optional[Sequence[tuple]] = None
    mlp: Optional[AppearanceMLP] = None
    # per segment, the cameras of a launch that render it (bit c = camera c); None: all of them
    segment_cams: Optional[Sequence[int]] = None

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @staticmethod
    def from_scene(scene, device="cuda", attr_dtype=torch.float32, sh_dtype=torch.float32) -> "Gaussians":
        def t(a, dt):
            return torch.as_tensor(np.ascontiguousarray(a)).to(device=device, dtype=dt).contiguous()
        return Gaussians(t(scene.means, torch.float32), t(scene.scales, attr_dtype), t(scene.quats, attr_dtype),
                         t(scene.opacities, attr_dtype), t(scene.sh, sh_dtype), int(scene.sh_degree))

    def c_struct(self):
        seg_arr = None
        if self.segments is not None:
            seg_arr = (Segment * max(len(self.segments), 1))()
            for k, (b, c) in enumerate(self.segments):
                seg_arr[k].begin = int(b)
                seg_arr[k].count = int(c)
        cam_arr = None
        if self.segment_cams is not None:
            if self.segments is None or len(self.segment_cams) != len(self.segments):
                raise ValueError("segment_cams needs one camera mask per segment")
            cam_arr = (ctypes.c_uint32 * max(len(self.segment_cams), 1))(*[int(m) for m in self.segment_cams])
        n = self.n
        cmlp = self.mlp.c_struct(n) if self.mlp is not None else None
        g = CGaussians(n, _ptr(self.means), _ptr(self.scales), _ptr(self.quats), _ptr(self.opacities),
                       _ptr(self.sh), int(self.sh.shape[1]) if self.sh.dim() == 3 else 1, int(self.sh_degree),
                       DTYPES[self.scales.dtype], DTYPES[self.sh.dtype],
                       ctypes.cast(seg_arr, ctypes.POINTER(Segment)) if seg_arr is not None else None,
                       len(self.segments) if self.segments is not None else 0,
                       ctypes.pointer(cmlp) if cmlp is not None else None,
                       ctypes.cast(cam_arr, ctypes.POINTER(ctypes.c_uint32)) if cam_arr is not None else None)
        if self.means.dtype != torch.float32:
            raise ValueError("means must be float32")
        if not (self.scales.dtype == self.quats.dtype == self.opacities.dtype):
            raise ValueError("scales, quats and opacities must share one dtype")
        return g, (seg_arr, cmlp, cam_arr)

    def check_cameras(self, n_cams: int):
        if self.mlp is not None and self.mlp.cached is None and self.mlp.image_embed.shape[0] != n_cams:
            raise ValueError(f"image_embed has {self.mlp.image_embed.shape[0]} rows for {n_cams} cameras")

    def render_count(self) -> int:
        if self.segments is None:
            return self.n
        return int(sum(c for _, c in self.segments))


def c_camera(cam, appearance: Optional[torch.Tensor] = None) -> CCamera:
    vm = np.asarray(cam.viewmat, np.float64).reshape(12)
    c = CCamera()
    for k in range(12):
        c.viewmat[k] = float(vm[k])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    c.near_plane, c.far_plane = float(cam.near), float(cam.far)
    c.appearance = _ptr(appearance) if appearance is not None else None
    return c


def c_cameras(cams, appearances=None):
    arr = (CCamera * len(cams))()
    for k, cam in enumerate(cams):
        arr[k] = c_camera(cam, None if appearances is None else appearances[k])
    return arr


@dataclasses.dataclass
class Options:
    eps2d: float = 0.3
    antialiased: bool = True
    tile_cull: bool = False
    bg: tuple = (0.0, 0.0, 0.0)
    save_state: bool = True
    absgrad: bool = False
    global_sort: bool = False  # order the pairs with global radix sorts instead of per-tile sorts

    def c_struct(self) -> COpts:
        o = COpts()
        o.eps2d = float(self.eps2d)
        o.antialiased = int(bool(self.antialiased))
        o.tile_cull = int(bool(self.tile_cull))
        for k in range(3):
            o.bg[k] = float(self.bg[k])
        o.save_state = int(bool(self.save_state))
        o.absgrad = int(bool(self.absgrad))
        o.global_sort = int(bool(self.global_sort))
        return o


class State:
    """A forward state: what render_backward needs; released when garbage-collected, or when
    its Context is closed (whichever comes first)."""

    def __init__(self, ctx: "Context", handle: int):
        self.ctx = ctx
        self.handle = handle
        ctx._states.add(self)

    def info(self) -> dict:
        i = CStateInfo()
        _check(self.ctx, load().gsr_state_get_info(self.handle, ctypes.byref(i)))
        return dict(n_render=i.n_render, n_cams=i.n_cams, n_visible=i.n_visible, n_pairs=i.n_pairs,
                    n_tiles=i.n_tiles, n_pixels=i.n_pixels, max_tile_pairs=i.max_tile_pairs)

    def copy(self, which: int, count: int, dtype=torch.int32, width: int = 1) -> torch.Tensor:
        out = torch.empty((count, width) if width > 1 else (count,), dtype=dtype, device=f"cuda:{self.ctx.device}")
        nbytes = out.numel() * out.element_size()
        if nbytes:
            _check(self.ctx, load().gsr_state_copy(self.handle, which, _ptr(out), nbytes, _stream()))
        return out

    def release(self):
        if self.handle:
            # a state must go back to a live context; a closed context already released it
            if self.ctx.handle:
                load().gsr_state_release(self.ctx.handle, self.handle)
            self.handle = None
            self.ctx._states.discard(self)

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


class Context:
    """One library context (workspace) bound to one device; use one per stream.

    allocator: None (the library's own stream-ordered pool) or an object with
    alloc(nbytes, stream) -> address (0 on failure) and free(address, nbytes, stream), e.g.
    TorchAllocator; its callbacks are kept alive as long as the context."""

    def __init__(self, device: int = 0, allocator=None):
        L = load()
        self.device = int(device)
        self.handle = None
        self._states = weakref.WeakSet()
        self._alloc_keep = None
        calloc = None
        if allocator is not None:
            a_fn = ALLOC_FN(lambda nbytes, stream, user: allocator.alloc(nbytes, stream or 0) or None)
            f_fn = FREE_FN(lambda ptr, nbytes, stream, user: allocator.free(ptr, nbytes, stream or 0))
            calloc = CAllocator(a_fn, f_fn, None)
            self._alloc_keep = (allocator, a_fn, f_fn, calloc)
        h = ctypes.c_void_p()
        st = L.gsr_create(ctypes.byref(h), self.device, ctypes.byref(calloc) if calloc is not None else None)
        if st != GSR_OK:
            raise GsrError(st, "gsr_create")
        self.handle = h.value

    def close(self):
        if getattr(self, "handle", None):
            for st in list(self._states):
                st.release()
            load().gsr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return load().gsr_last_error(self.handle).decode()

    def workspace_bytes(self) -> int:
        return int(load().gsr_workspace_bytes(self.handle))

    def workspace_query(self, n_render: int, cams, expected_pairs: int) -> int:
        arr = c_cameras(cams)
        out = ctypes.c_size_t()
        _check(self, load().gsr_workspace_query(self.handle, int(n_render), arr, len(cams), int(expected_pairs),
                                                ctypes.byref(out)))
        return int(out.value)

    def set_wait_limit(self, polls: int = 0, never_ready: bool = False):
        """Bound on the polls of every device wait (0: the default); never_ready makes every wait
        run to it (a test of failure detection). See gsr_set_wait_limit."""
        _check(self, load().gsr_set_wait_limit(self.handle, int(polls), int(bool(never_ready))))

    def set_fill_rate(self, gb_per_s: float = 0.0, blocks: int = 0):
        """Pace of the gradient zero fill in GB/s (0: unpaced) and its block count (0: keep).
        See gsr_set_fill_rate."""
        _check(self, load().gsr_set_fill_rate(self.handle, float(gb_per_s), int(blocks)))

    def set_fill_split(self, early_share: float = 0.0):
        """Share of a requested gradient fill queued by the forward after its preprocess (the
        rest by the backward before its blend). See gsr_set_fill_split."""
        _check(self, load().gsr_set_fill_split(self.handle, float(early_share)))

    def sync_check(self, stream=None):
        _check(self, load().gsr_sync_check(self.handle, _stream(stream)))

    def profile(self, on: bool = True, count_evals: bool = False, stages=None):
        """Stage events on or off; `stages` (names from STAGES) limits them to those stages."""
        mask = 0xFFFFFFFF if stages is None else sum(1 << STAGES.index(k) for k in stages)
        _check(self, load().gsr_profile_select(self.handle, mask))
        _check(self, load().gsr_profile_enable(self.handle, int(on), int(count_evals)))

    def profile_collect(self) -> dict:
        """Per-stage milliseconds and launches, and blend counters, since the last collect."""
        ms = np.zeros(len(STAGES), np.float64)
        launches = np.zeros(len(STAGES), np.int64)
        cnt = np.zeros(len(COUNTERS), np.int64)
        _check(self, load().gsr_profile_collect(self.handle, ms.ctypes.data, launches.ctypes.data, cnt.ctypes.data))
        return dict(ms=dict(zip(STAGES, ms.tolist())), launches=dict(zip(STAGES, launches.tolist())),
                    counters=dict(zip(COUNTERS, cnt.tolist())))


def _check(ctx, st):
    if st != GSR_OK and st != GSR_WARN_OVER_BUDGET:
        raise GsrError(st, ctx.last_error() if ctx is not None else "")
    return st


def pixel_count(cams) -> int:
    return int(sum(int(c.width) * int(c.height) for c in cams))


def render_forward(ctx: Context, g: Gaussians, cams, opts: Options = None, appearances=None, want_state=True,
                   outputs: Optional[dict] = None, stream=None):
    """Renders cameras packed one after another. Returns (dict of outputs, State or None)."""
    opts = opts or Options()
    dev = f"cuda:{ctx.device}"
    npix = pixel_count(cams)
    if outputs is None:
        outputs = dict(rgb=torch.empty((npix, 3), device=dev), depth_acc=torch.empty(npix, device=dev),
                       depth_exp=torch.empty(npix, device=dev), alpha=torch.empty(npix, device=dev))
    g.check_cameras(len(cams))
    cg, seg_keep = g.c_struct()
    carr = c_cameras(cams, appearances)
    co = opts.c_struct()
    out = COutputs(_ptr(outputs["rgb"]), _ptr(outputs.get("depth_acc")), _ptr(outputs.get("depth_exp")),
                   _ptr(outputs.get("alpha")))
    sh = ctypes.c_void_p()
    st = load().gsr_render_forward(ctx.handle, ctypes.byref(cg), carr, len(cams), ctypes.byref(co), ctypes.byref(out),
                                   ctypes.byref(sh) if want_state else None, _stream(stream))
    _check(ctx, st)
    del seg_keep
    return outputs, (State(ctx, sh.value) if want_state else None)


def param_grads(ctx: Context, g: Gaussians, n_cams: int, absgrad: bool = False) -> dict:
    """Uninitialised gradient arrays for render_backward."""
    dev = f"cuda:{ctx.device}"
    n = g.n
    K = int(g.sh.shape[1])
    out = dict(means=torch.empty((n, 3), device=dev), scales=torch.empty((n, 3), device=dev),
               quats=torch.empty((n, 4), device=dev), opacities=torch.empty(n, device=dev),
               sh=torch.empty((n, K, 3), device=dev), appearance=torch.empty((n_cams, 3, 4), device=dev),
               absgrad=torch.empty((n, 2), device=dev) if absgrad else None)
    if g.mlp is not None:
        out.update(gauss_embed=torch.empty((n, 16), device=dev), image_embed=torch.empty((n_cams, 32), device=dev),
                   mlp_params=torch.empty(MLP_PARAMS, device=dev))
    return out


def _c_param_grads(grads: dict):
    return CParamGrads(_ptr(grads["means"]), _ptr(grads["scales"]), _ptr(grads["quats"]), _ptr(grads["opacities"]),
                       _ptr(grads["sh"]), _ptr(grads.get("appearance")), _ptr(grads.get("absgrad")),
                       _ptr(grads.get("gauss_embed")), _ptr(grads.get("image_embed")), _ptr(grads.get("mlp_params")))


def appearance_cache(ctx: Context, g: Gaussians, image: int = 0, out: Optional[torch.Tensor] = None,
                     stream=None) -> torch.Tensor:
    """The appearance transform's outputs [n,4] of every Gaussian for row `image` of
    g.mlp.image_embed (gsr_appearance_cache); AppearanceMLP(None, None, None, cached=...) renders
    with them without evaluating the transform."""
    if g.mlp is None or g.mlp.cached is not None:
        raise ValueError("needs Gaussians with an evaluated appearance transform")
    if not 0 <= image < g.mlp.image_embed.shape[0]:
        raise ValueError("image is not a row of image_embed")
    if out is None:
        out = torch.empty((g.n, 4), device=g.means.device)
    cg, keep = g.c_struct()
    _check(ctx, load().gsr_appearance_cache(ctx.handle, ctypes.byref(cg), int(image), _ptr(out), _stream(stream)))
    del keep
    return out


def zero_param_grads(ctx: Context, g: Gaussians, grads: dict, stream=None):
    """Requests the zero fill of the gradient arrays ahead of the backward (see
    gsr_param_grads_zero): the next backward given these arrays queues the fill right before its
    blend, which it runs beside."""
    cg, seg_keep = g.c_struct()
    pg = _c_param_grads(grads)
    _check(ctx, load().gsr_param_grads_zero(ctx.handle, ctypes.byref(cg), ctypes.byref(pg), _stream(stream)))
    del seg_keep


def render_backward(ctx: Context, g: Gaussians, cams, state: State, d_out: dict, opts: Options = None,
                    appearances=None, grads: Optional[dict] = None, stream=None) -> dict:
    """Gradients of L given dL/d(outputs) (keys rgb, depth_acc, depth_exp, alpha; missing = 0)."""
    opts = opts or Options()
    if grads is None:
        grads = param_grads(ctx, g, len(cams), opts.absgrad)
    g.check_cameras(len(cams))
    cg, seg_keep = g.c_struct()
    carr = c_cameras(cams, appearances)
    co = opts.c_struct()
    dg = COutGrads(_ptr(d_out.get("rgb")), _ptr(d_out.get("depth_acc")), _ptr(d_out.get("depth_exp")),
                   _ptr(d_out.get("alpha")))
    pg = _c_param_grads(grads)
    st = load().gsr_render_backward(ctx.handle, ctypes.byref(cg), carr, len(cams), ctypes.byref(co), state.handle,
                                    ctypes.byref(dg), ctypes.byref(pg), _stream(stream))
    _check(ctx, st)
    del seg_keep
    return grads


def sort_pairs_u32(ctx: Context, keys: torch.Tensor, vals: torch.Tensor, begin_bit=0, end_bit=32, stream=None):
    """Stable radix sort of uint32 (stored as int32) key/value pairs by key bits [begin_bit, end_bit)."""
    assert keys.dtype == torch.int32 and vals.dtype == torch.int32 and keys.shape == vals.shape
    ko = torch.empty_like(keys)
    vo = torch.empty_like(vals)
    _check(ctx, load().gsr_sort_pairs_u32(ctx.handle, _ptr(keys), _ptr(vals), _ptr(ko), _ptr(vo), keys.numel(),
                                          int(begin_bit), int(end_bit), _stream(stream)))
    return ko, vo


def union_segments(selections):
    """Segments and camera masks for one launch of several views with their own detail levels:
    selections[c] lists view c's (partition, level, begin, count) in partition order (one level
    per partition). Returns (segments, masks) for Gaussians.segments / segment_cams: the union,
    ordered by (partition, level), so every view keeps its own relative order (and so the same
    depth-tie order and the same image as rendered alone)."""
    if len(selections) > 32:
        raise ValueError("at most 32 views per launch")
    table = {}
    for c, sel in enumerate(selections):
        for p, lev, begin, count in sel:
            key = (int(p), int(lev))
            if key in table:
                if (table[key][0], table[key][1]) != (int(begin), int(count)):
                    raise ValueError(f"views disagree on the segment of partition {key[0]} level {key[1]}")
                table[key][2] |= 1 << c
            else:
                table[key] = [int(begin), int(count), 1 << c]
    keys = sorted(table)
    return [(table[k][0], table[k][1]) for k in keys], [table[k][2] for k in keys]


def select_lod(aabb: np.ndarray, level_offsets: np.ndarray, cam, thresholds, budget: int = 0):
    """Host-side detail-level selection -> (status, levels [P], segments [(begin, count)], n_selected)."""
    aabb = np.ascontiguousarray(np.asarray(aabb, np.float64).reshape(-1, 6))
    P = aabb.shape[0]
    lo = np.ascontiguousarray(np.asarray(level_offsets, np.int64))
    L = lo.shape[0]
    thr = np.ascontiguousarray(np.asarray(thresholds, np.float64).reshape(-1))
    if thr.size == 0:
        thr = np.zeros(1)
    levels = np.zeros(max(P, 1), np.int32)
    segs = (Segment * max(P, 1))()
    ns = ctypes.c_int32()
    nsel = ctypes.c_int64()
    cc = c_camera(cam)
    st = load().gsr_select_lod(P, aabb.ctypes.data, L, lo.ctypes.data, ctypes.byref(cc), thr.ctypes.data, int(budget),
                               levels.ctypes.data, segs, ctypes.byref(ns), ctypes.byref(nsel))
    if st < 0:
        raise GsrError(st, "gsr_select_lod")
    return st, levels[:P], [(segs[k].begin, segs[k].count) for k in range(ns.value)], int(nsel.value)
