"""Scene and detail-level files (no GPU): what is saved loads back bit for bit, and files of the
wrong kind, foreign files and truncated files are refused."""
import numpy as np
import pytest

from paper_2507_23006_gb300 import assets, lod, scenes


def _same_scene(a, b):
    assert a.sh_degree == b.sh_degree and a.n == b.n
    for k in ("means", "scales", "quats", "opacities", "sh"):
        x, y = getattr(a, k), getattr(b, k)
        assert x.dtype == y.dtype and x.shape == y.shape and np.array_equal(x.view(np.uint8), y.view(np.uint8)), k


def test_scene_round_trip(tmp_path):
    sc = scenes.city(7, 3_000)
    p = tmp_path / "city.gsr"
    assets.save_scene(str(p), sc)
    back = assets.load_scene(str(p))
    _same_scene(sc, back)
    raw = p.read_bytes()
    assert raw[:8] == assets.MAGIC
    hlen = int.from_bytes(raw[8:16], "little")
    assert assets._data_start(hlen) % 64 == 0


def test_lod_round_trip_renders_the_same_selection(tmp_path):
    fine = scenes.city(8, 6_000)
    mid = lod.merge_to_count(fine, 1_500, device="cpu")
    L = lod.build_lod([mid, fine])
    p = tmp_path / "levels.gsr"
    assets.save_lod(str(p), L)
    back = assets.load_lod(str(p))
    _same_scene(L.gaussians, back.gaussians)
    assert back.level_sizes == L.level_sizes
    assert back.aabb.dtype == np.float64 and np.array_equal(back.aabb, L.aabb)
    assert back.level_offsets.dtype == np.int64 and np.array_equal(back.level_offsets, L.level_offsets)


def test_wrong_kind_foreign_and_truncated_files_are_refused(tmp_path):
    sc = scenes.city(9, 500)
    p = tmp_path / "s.gsr"
    assets.save_scene(str(p), sc)
    with pytest.raises(ValueError, match="not a 'lod' asset"):
        assets.load_lod(str(p))
    q = tmp_path / "other.bin"
    q.write_bytes(b"NOTASSET" + bytes(64))
    with pytest.raises(ValueError, match="not a scene asset file"):
        assets.load_scene(str(q))
    t = tmp_path / "cut.gsr"
    t.write_bytes(p.read_bytes()[:-100])
    with pytest.raises(ValueError, match="truncated"):
        assets.load_scene(str(t))
