"""Values the paper prints, kept as small text fixtures under tests/golden/ (each cites its
passage), checked against the oracle and the binding."""
import os

import numpy as np

import oracle
from paper_2507_23006_gb300 import native, scenes

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _sizes():
    out = {}
    with open(os.path.join(GOLDEN, "appearance_transform_sizes.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                out[k] = int(v)
    return out


def test_appearance_transform_sizes():
    s = _sizes()
    n_in = s["gaussian_embedding"] + s["image_embedding"]
    n_params = s["hidden"] * n_in + s["hidden"] + s["outputs"] * s["hidden"] + s["outputs"]
    assert native.MLP_PARAMS == n_params
    # the oracle takes inputs of exactly these sizes (one camera, a few Gaussians)
    sc, cam = scenes.tiny_scene(2, 5, 16, 16)
    mlp = scenes.appearance_mlp(np.random.default_rng(0), sc.n, 1)
    assert mlp["gemb"].shape[1] == s["gaussian_embedding"] and mlp["iemb"].shape[1] == s["image_embedding"]
    assert mlp["w1"].shape == (s["hidden"], n_in) and mlp["w2"].shape == (s["outputs"], s["hidden"])
    img = oracle.render(sc, [cam], oracle.Opts(), mlp=mlp, want_pairs=False).img
    assert np.isfinite(img).all()
