"""The C ABI without a GPU: the library loads, exports every function include/gsr.h declares,
rejects bad arguments with a status, and its host-side detail-level selection agrees with the
oracle exactly (it is integer work)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2507_23006_gb300 import native, scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gsr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(gsr_[a-z_0-9]+)\s*\(", src, flags=re.M)))


def test_library_exports_every_declared_function():
    L = native.load()
    names = declared_functions()
    assert len(names) >= 14
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(native.EXPORTED)


def test_status_strings_and_null_arguments():
    L = native.load()
    assert L.gsr_status_string(0) == b"ok"
    assert L.gsr_status_string(-4) == b"device wait timed out"
    # null context / out pointers are rejected before any CUDA call
    assert L.gsr_sort_pairs_u32(None, None, None, None, None, 10, 0, 32, None) == -1
    # the allocation-free sort needs a device error word; without one it refuses
    assert L.gsr_sort_pairs_u32_noalloc(None, None, None, None, 10, 0, 32, None, None) == -1
    assert L.gsr_create(None, 0, None) == -1
    assert L.gsr_render_forward(None, None, None, 1, None, None, None, None) == -1
    assert L.gsr_state_get_info(None, None) == -1
    assert L.gsr_workspace_bytes(None) == 0


def test_create_without_gpu_reports_an_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L = native.load()
    h = ctypes.c_void_p()
    assert L.gsr_create(ctypes.byref(h), 0, None) == -3


def _grid_partitions(nx, ny, size, rng):
    aabb = []
    for i in range(nx):
        for j in range(ny):
            aabb.append([i * size - nx * size / 2, j * size - ny * size / 2, 0.0,
                         (i + 1) * size - nx * size / 2, (j + 1) * size - ny * size / 2, rng.uniform(10, 80)])
    return np.array(aabb)


@pytest.mark.parametrize("seed", range(6))
def test_select_lod_matches_oracle(seed):
    rng = np.random.default_rng(seed)
    aabb = _grid_partitions(8, 7, 100.0, rng)
    P = len(aabb)
    counts = np.stack([rng.integers(0, 50, P), rng.integers(50, 500, P), rng.integers(500, 5000, P)])
    lo = np.zeros((3, P + 1), np.int64)
    off = 0
    for l in range(3):
        lo[l, 0] = off
        lo[l, 1:] = off + np.cumsum(counts[l])
        off = lo[l, -1]
    if seed % 2:
        cam = scenes.aerial_camera(1920, 1080, altitude=rng.uniform(50, 300), pitch_deg=rng.uniform(20, 80),
                                   target=(rng.uniform(-300, 300), rng.uniform(-300, 300), 0.0),
                                   azimuth_deg=rng.uniform(0, 360))
    else:
        cam = scenes.street_level_camera(1280, 720, x=rng.uniform(-300, 300), y=rng.uniform(-300, 300), height_m=2.0)
    for budget in (0, 200_000, 20_000, 100):
        a = native.select_lod(aabb, lo, cam, [100.0, 200.0], budget)
        b = oracle.select_lod(aabb, lo, cam, [100.0, 200.0], budget)
        assert a[0] == b[0]
        np.testing.assert_array_equal(a[1], b[1])
        assert [tuple(s) for s in a[2]] == [tuple(s) for s in b[2].tolist()]
        assert a[3] == b[3]
    assert (a[1] == -1).any() or seed % 2 == 1


def test_select_lod_rejects_bad_arguments():
    cam = scenes.box_camera()
    aabb = np.zeros((2, 6))
    lo = np.zeros((3, 3), np.int64)
    with pytest.raises(native.GsrError) as e:
        native.select_lod(aabb, lo, cam, [200.0, 100.0], 0)   # thresholds must ascend
    assert e.value.status == -1
