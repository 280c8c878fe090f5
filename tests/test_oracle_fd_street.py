"""The oracle's analytic gradient against FP64 central finite differences on the 500k street
block at 1920x1080 (CPU): the FD machinery of the GPU protocol (tests/fd_util.py) checked on a
handful of Gaussians, and the per-image 3x4 transform through the epilogue over the raw colour
sums and transmittances."""
import numpy as np
import pytest

import oracle
from paper_2507_23006_gb300 import scenes
from tests import fd_util


@pytest.fixture(scope="module")
def street_case():
    scene, cam, aff, oopts, up, res = fd_util.build_case(fd_util.STREET_RECIPE)
    ref = oracle.backward(scene, [cam], up, oopts, affines=aff[None], want_g2d=True)
    return scene, cam, aff, oopts, res, up, ref


def test_analytic_gradient_matches_fd_on_the_street_block(street_case):
    scene, cam, aff, oopts, res, up, ref = street_case
    contributing = np.nonzero(np.abs(ref["g2d"][:, 5]) > 0)[0]
    chosen = np.random.default_rng(2).choice(contributing, 6, replace=False)
    fd, dropped, total = fd_util.fd_gradients_parallel(fd_util.STREET_RECIPE, chosen, workers=3)
    assert dropped <= 0.2 * total
    checked = 0
    for name, _ in fd_util.GROUPS:
        a = np.asarray(ref[name]).reshape(scene.n, -1)[chosen]
        f = fd[name][:, :a.shape[1]]
        ok = ~np.isnan(f)
        # FD rounding: L sums about 10^4 FP64 terms of order 1, so its ~1e-12 of rounding over 2h =
        # 2e-6 leaves ~1e-6 of noise in the quotient
        assert np.all(np.abs(a[ok] - f[ok]) <= 1e-5 * np.abs(f[ok]) + 1e-6), name
        checked += int(ok.sum())
    assert checked >= 0.8 * total


def test_affine_gradient_matches_fd_of_the_epilogue(street_case):
    scene, cam, aff, oopts, res, up, ref = street_case
    plain = oracle.render(scene, [cam], oopts, want_pairs=False)
    T = plain.img[:, 6]
    raw_C = plain.img[:, 0:3] - np.outer(T, oopts.bg)
    fd = fd_util.fd_affine(raw_C, T, np.array(oopts.bg), up, aff)
    np.testing.assert_allclose(ref["affine"].reshape(-1), fd, rtol=1e-6, atol=1e-6)
