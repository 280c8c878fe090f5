"""Gradient parity on the full 500k street block at 1920x1080 (the training-step configuration):
the CUDA path's gradients of L = sum <w, outputs> (w ~ N(0, 1) on rgb, depth_acc, alpha, and on
depth_exp where alpha > 0.05; zero on marked pixels), with a per-image 3x4 transform I + N(0, 0.01),

* against the oracle's analytic gradient for every Gaussian, and
* against FP64 central finite differences of the oracle for 200 Gaussians (seed 2) that have at
  least one contributing pixel, every one of their 59 parameters, each difference re-compositing
  only the tiles of that Gaussian's rectangle (tests/fd_util.py); parameters whose step changes
  a discrete decision are dropped and counted; the transform by FD of the epilogue over the raw
  colour sums and transmittances.

Both at the gradient bar of tests/parity_util.py (the cancellation term with the oracle's
magnitudes of the elements' sums).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2507_23006_gb300 import native
from tests import fd_util
from tests import parity_util as pu
from tests.test_gpu_parity import _gpu_backward

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return native.Context(0)


def test_street_block_gradients_against_oracle_and_fd(ctx):
    scene, cam, aff, oopts, up, res = fd_util.build_case(fd_util.STREET_RECIPE)
    nopts = native.Options(tile_cull=oopts.tile_cull, antialiased=oopts.antialiased, bg=oopts.bg)
    aff_t = torch.tensor(aff, dtype=torch.float32, device="cuda")
    g = native.Gaussians.from_scene(scene)
    out, st = native.render_forward(ctx, g, [cam], nopts, appearances=[aff_t])
    um = res.mark == 0
    np.testing.assert_allclose(out["rgb"].cpu().numpy()[um], res.img[um, 0:3], atol=1e-4)
    gg = _gpu_backward(ctx, g, [cam], st, up, nopts, appearances=[aff_t])
    ref = oracle.backward(scene, [cam], up, oopts, affines=aff[None], want_mag=True, want_g2d=True)
    for k, _ in fd_util.GROUPS:
        pu.grad_close(gg[k], ref[k], f"{k} vs oracle", mag=ref["mag"][k])
    pu.grad_close(gg["appearance"].reshape(-1), ref["affine"].reshape(-1), "appearance vs oracle")

    contributing = np.nonzero(np.abs(ref["g2d"][:, 5]) > 0)[0]
    chosen = np.random.default_rng(2).choice(contributing, 200, replace=False)
    fd, dropped, total = fd_util.fd_gradients_parallel(fd_util.STREET_RECIPE, chosen, workers=12)
    print(f"\nFD protocol: {len(chosen)} Gaussians, {total} parameters, {dropped} dropped "
          f"(a step changed a discrete decision)")
    assert dropped <= 0.1 * total
    n = scene.n
    for k, _ in fd_util.GROUPS:
        a = np.asarray(gg[k], np.float64).reshape(n, -1)[chosen]
        f = fd[k][:, :a.shape[1]]
        m = np.asarray(ref["mag"][k], np.float64).reshape(n, -1)[chosen]
        keep = ~np.isnan(f)
        # the group's RMS is that of the whole gradient array, as in the comparison with the oracle
        rms = float(np.sqrt(np.mean(np.asarray(ref[k], np.float64) ** 2)))
        pu.grad_close(a[keep], f[keep], f"{k} vs FD ({int(keep.sum())} of {keep.size})", mag=m[keep], rms=rms)
    plain = oracle.render(scene, [cam], oopts, want_pairs=False)
    T = plain.img[:, 6]
    raw_C = plain.img[:, 0:3] - np.outer(T, oopts.bg)
    fd_aff = fd_util.fd_affine(raw_C, T, np.array(oopts.bg), up, aff)
    pu.grad_close(gg["appearance"].reshape(-1), fd_aff, "appearance vs FD of the epilogue")
