"""Host-side logic of the benchmark and of the appearance-transform binding (no GPU): the
per-stage algorithmic-time fractions, the kernel count per step, the stored-counter keying,
the seeded appearance-transform inputs and the parameter packing."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2507_23006_gb300 import scenes  # noqa: E402


def test_stage_rooflines_pick_the_binding_resource():
    # 1 GB through a 1000 GB/s memory is 1 ms; 2e9 FP32 ops at 1 TFLOP/s are 2 ms
    stage_ms = {"preprocess": 2.0, "blend_bwd": 4.0}
    n, V, P, tiles, npix = 1_000_000, 0, 0, 1, 0
    counts = {"fwd_evals": 0, "bwd_evals": int(2e9 / bench.FLOPS_PER_BWD_EVAL)}
    rows, step = bench.stage_rooflines(stage_ms, n, V, P, tiles, npix, counts, 1.0, 1e15, 1000.0, 8.0)
    pre = rows["preprocess"]
    assert pre["bound"] == "hbm"
    assert pre["algorithmic_us"] == pytest.approx(44.0 * n / 1e12 * 1e6, rel=1e-6)
    assert pre["frac"] == pytest.approx(pre["algorithmic_us"] / 2000.0, rel=1e-3)
    bwd = rows["blend_bwd"]
    assert bwd["bound"] == "alu" and bwd["algorithmic_us"] == pytest.approx(2000.0, rel=1e-3)
    assert bwd["frac"] == pytest.approx(0.5, rel=1e-3)
    # stages not measured (the fill beside the others) have no fraction; the fill's zeros (SH rows
    # of Gaussians without a record) are not counted in the step
    assert rows["gradient_fill"]["frac"] is None
    assert rows["gradient_fill"]["algorithmic_us"] == pytest.approx(192.0 * n / 1e12 * 1e6, rel=1e-6)
    assert rows["preprocess_bwd"]["algorithmic_us"] == pytest.approx(128.0 * n / 1e12 * 1e6, rel=1e-6)
    total = sum(r["algorithmic_us"] for k, r in rows.items() if k != "gradient_fill")
    assert step["algorithmic_us"] == pytest.approx(total, abs=0.1)
    assert step["frac"] == pytest.approx(total / 8000.0, abs=1e-3)  # rounded to three places


def test_kernels_per_step():
    # preprocess (cull and record passes, the latter counting the pairs per tile), tile scan,
    # placing, forward blend (which sorts the tiles' lists), gradient fill, backward blend,
    # projection backward
    assert bench.kernels_per_step(True, {"n_tiles": 8160, "n_visible": 10, "n_pairs": 20, "max_tile_pairs": 5}) == 8
    # a list of more than 1024 pairs is sorted by a launch of its own before the blend
    assert bench.kernels_per_step(True, {"n_tiles": 8160, "n_visible": 10, "n_pairs": 2000,
                                         "max_tile_pairs": 1500}) == 9
    # nothing visible: no placing or sorting
    assert bench.kernels_per_step(False, {"n_tiles": 256, "n_visible": 0, "n_pairs": 0}) == 7


def test_stored_counters_are_keyed_to_their_kernel_sources():
    # every stage with a stored counter names sources that exist; distinct stages that share no
    # file have distinct hashes, and the hash is stable
    for k, files in bench.KERNEL_SOURCES.items():
        for f in files + bench.COMMON_SOURCES:
            assert os.path.exists(os.path.join(ROOT, "paper_2507_23006_gb300", "csrc", f)), f
        assert bench.sources_sha256(k) == bench.sources_sha256(k)
    assert bench.sources_sha256("blend_bwd") != bench.sources_sha256("preprocess")
    assert bench.stored_traffic("blend_bwd", "some_other_workload") is None


def test_appearance_inputs_are_seeded_and_shaped():
    a = scenes.appearance_mlp(np.random.default_rng(3), 10, 2)
    b = scenes.appearance_mlp(np.random.default_rng(3), 10, 2)
    shapes = dict(gemb=(10, 16), iemb=(2, 32), w1=(32, 48), b1=(32,), w2=(4, 32), b2=(4,))
    for k, sh in shapes.items():
        assert a[k].shape == sh
        np.testing.assert_array_equal(a[k], b[k])


def test_appearance_parameters_pack_in_the_documented_order():
    torch = pytest.importorskip("torch")
    from paper_2507_23006_gb300 import native
    d = scenes.appearance_mlp(np.random.default_rng(4), 5, 1)
    m = native.AppearanceMLP.from_arrays(d, device="cpu")
    p = m.params.numpy()
    assert p.size == native.MLP_PARAMS == 1700
    np.testing.assert_array_equal(p[:1536], d["w1"].astype(np.float32).reshape(-1))
    np.testing.assert_array_equal(p[1536:1568], d["b1"].astype(np.float32))
    np.testing.assert_array_equal(p[1568:1696], d["w2"].astype(np.float32).reshape(-1))
    np.testing.assert_array_equal(p[1696:], d["b2"].astype(np.float32))
    assert m.gauss_embed.dtype == torch.float32 and tuple(m.gauss_embed.shape) == (5, 16)
