"""Scene and detail-level files for the serving loop: a level set that took a minute to merge
(20M Gaussians to 6M and 1.5M) is written once and loaded at server start.

Format (one file, little-endian): the 8 bytes ``GSRASSET``, a uint64 header length, a UTF-8 JSON
header, then the raw arrays from the first 64-byte boundary after the header, each on a 64-byte
boundary. The header names the kind (``scene`` or ``lod``), the scalar fields, and per array its
dtype (numpy string with an explicit byte order), shape, size and offset from the arrays' base.
Arrays are stored as the Scene / LodScene hold them (float32 attributes and SH, float64 boxes,
int64 offsets), so a load gives back the same bits.
"""
from __future__ import annotations

import json
import struct

import numpy as np

from .lod import LodScene
from .scenes import Scene

MAGIC = b"GSRASSET"
_ALIGN = 64
_SCENE_ARRAYS = ("means", "scales", "quats", "opacities", "sh")


def _data_start(header_len: int) -> int:
    """The arrays' base: the first 64-byte boundary after the magic, the length and the header."""
    return (len(MAGIC) + 8 + header_len + _ALIGN - 1) // _ALIGN * _ALIGN


def _write(path: str, kind: str, fields: dict, arrays: dict) -> None:
    arrays = {k: np.ascontiguousarray(v) for k, v in arrays.items()}
    layout, off = {}, 0
    for k, a in arrays.items():
        le = a.dtype.newbyteorder("<") if a.dtype.byteorder not in ("|", "<") else a.dtype
        layout[k] = dict(dtype=le.str, shape=list(a.shape), offset=off, nbytes=int(a.nbytes))
        off += (a.nbytes + _ALIGN - 1) // _ALIGN * _ALIGN
    blob = json.dumps(dict(format=1, kind=kind, fields=fields, arrays=layout), sort_keys=True).encode()
    start = _data_start(len(blob))
    with open(path, "wb") as f:
        f.write(MAGIC)
        f.write(struct.pack("<Q", len(blob)))
        f.write(blob)
        for k, a in arrays.items():
            f.write(b"\0" * (start + layout[k]["offset"] - f.tell()))
            f.write(a.astype(np.dtype(layout[k]["dtype"]), copy=False).tobytes())


def _read(path: str, kind: str):
    with open(path, "rb") as f:
        if f.read(len(MAGIC)) != MAGIC:
            raise ValueError(f"{path}: not a scene asset file")
        (n,) = struct.unpack("<Q", f.read(8))
        head = json.loads(f.read(n).decode())
        if head.get("format") != 1 or head.get("kind") != kind:
            raise ValueError(f"{path}: holds a {head.get('kind')!r} asset of format {head.get('format')}, "
                             f"not a {kind!r} asset of format 1")
        start = _data_start(n)
        arrays = {}
        for k, d in head["arrays"].items():
            f.seek(start + d["offset"])
            buf = f.read(d["nbytes"])
            if len(buf) != d["nbytes"]:
                raise ValueError(f"{path}: array {k} is truncated")
            dt = np.dtype(d["dtype"])
            arrays[k] = np.frombuffer(buf, dt).reshape(d["shape"]).astype(dt.newbyteorder("="), copy=True)
    return head["fields"], arrays


def save_scene(path: str, scene: Scene) -> None:
    _write(path, "scene", dict(sh_degree=int(scene.sh_degree), n=scene.n),
           {k: getattr(scene, k) for k in _SCENE_ARRAYS})


def load_scene(path: str) -> Scene:
    fields, a = _read(path, "scene")
    return Scene(*(a[k] for k in _SCENE_ARRAYS), int(fields["sh_degree"]))


def save_lod(path: str, lod: LodScene) -> None:
    g = lod.gaussians
    arrays = {k: getattr(g, k) for k in _SCENE_ARRAYS}
    arrays["aabb"] = np.asarray(lod.aabb, np.float64)
    arrays["level_offsets"] = np.asarray(lod.level_offsets, np.int64)
    _write(path, "lod", dict(sh_degree=int(g.sh_degree), level_sizes=[int(x) for x in lod.level_sizes]), arrays)


def load_lod(path: str) -> LodScene:
    fields, a = _read(path, "lod")
    g = Scene(*(a[k] for k in _SCENE_ARRAYS), int(fields["sh_degree"]))
    return LodScene(g, a["aabb"], a["level_offsets"], list(fields["level_sizes"]))
