"""The gradient bar of the GPU parity tests discriminates (CPU only).

The oracle's test switch plants one plausible mistake in its gradients at a time (the 0.99 clamp
mask of alpha dropped, the degree-2 SH band's sign flipped, the depth term of dL/dalpha left out,
the gradients of conic a and c swapped). On the scenes, options and upstream gradients of the GPU
backward tests, the bar actually used there (tests/parity_util.py: 1e-3 relative plus 1e-3 of the
group RMS per element, plus CANCEL_REL of the contributions' magnitude only for cancelling sums)
must reject each mutated gradient wherever the mistake changes it at all, and every mistake must
change (and be caught on) at least one of these scenes.
"""
import numpy as np
import pytest

import oracle
from paper_2507_23006_gb300 import scenes
from tests import parity_util as pu

GROUPS = ("means", "scales", "quats", "opacities", "sh")


def _box_case(aa, cull, deg):
    scene, cam = pu.scene_box_backward(4000, seed=3)
    scene.sh_degree = deg
    oopts = oracle.Opts(antialiased=aa, tile_cull=cull, bg=(0.2, 0.1, 0.0))
    res = oracle.render(scene, [cam], oopts, want_pairs=False)
    up = pu.upstream(res, cam.width * cam.height, seed=11)
    return scene, [cam], oopts, up, None


def _street_case():
    scene, cam = scenes.street_block(1, 500_000), scenes.street_block_camera()
    oopts = oracle.Opts(tile_cull=True)
    ntx, nty = (cam.width + 15) // 16, (cam.height + 15) // 16
    full = oracle.render(scene, [cam], oopts)
    counts = np.bincount(full.pairs[:, 0], minlength=ntx * nty)
    rng = np.random.default_rng(4)
    busy = np.nonzero(counts > 0)[0]
    tiles = np.unique(np.concatenate([rng.choice(busy, 40, replace=False), rng.choice(ntx * nty, 8, replace=False)]))
    pix = []
    for t in tiles:
        ty, tx = divmod(int(t), ntx)
        for y in range(ty * 16, min(ty * 16 + 16, cam.height)):
            pix.extend(range(y * cam.width + tx * 16, y * cam.width + min(tx * 16 + 16, cam.width)))
    pix = np.array(pix)
    um = pix[full.mark[pix] == 0]
    up = pu.upstream_on(um, cam.width * cam.height, seed=9, alpha=full.img[:, 5])
    return scene, [cam], oopts, up, tiles


CASES = {
    "box aa": lambda: _box_case(True, False, 3),
    "box cull no-aa": lambda: _box_case(False, True, 3),
    "box aa cull deg1": lambda: _box_case(True, True, 1),
    "street block 1080p": _street_case,
}


@pytest.fixture(scope="module")
def verdicts():
    """(case, mutation) -> 'invisible' (the mistake does not change this gradient), 'caught (n
    elements outside)' or 'missed'."""
    out = {}
    for case, make in CASES.items():
        scene, cams, oopts, up, tiles = make()
        ref = oracle.backward(scene, cams, up, oopts, tile_subset=tiles, want_mag=True)
        for k in oracle.MUTATIONS:
            with oracle.mutation(k):
                bad = oracle.backward(scene, cams, up, oopts, tile_subset=tiles)
            changed = False
            n_out = 0
            for name in GROUPS:
                a, b = np.asarray(bad[name]).reshape(-1), np.asarray(ref[name]).reshape(-1)
                scale = np.abs(b).max() + 1e-300
                if np.abs(a - b).max() > 1e-9 * scale:
                    changed = True
                ok, _ = pu.grad_stats(a, b, mag=ref["mag"][name])
                n_out += int((~ok).sum())
            out[(case, k)] = f"caught ({n_out} elements outside)" if n_out else ("missed" if changed else "invisible")
    return out


@pytest.mark.parametrize("k", sorted(oracle.MUTATIONS))
def test_bar_rejects_every_visible_mistake(verdicts, k):
    rows = {case: verdicts[(case, k)] for case in CASES}
    print(f"\nmutation {k} ({oracle.MUTATIONS[k]}): {rows}")
    assert "missed" not in rows.values(), rows
    assert any(v.startswith("caught") for v in rows.values()), rows


def test_correct_gradients_pass_their_own_bar():
    scene, cams, oopts, up, tiles = _box_case(True, False, 3)
    ref = oracle.backward(scene, cams, up, oopts, want_mag=True)
    for name in GROUPS:
        ok, st = pu.grad_stats(ref[name], ref[name], mag=ref["mag"][name])
        assert ok.all() and st["strict_pass"] == 1.0


def test_clamp_is_active_in_the_backward_scene():
    """The opaque Gaussians of the backward scene do reach the 0.99 clamp somewhere."""
    scene, cam = pu.scene_box_backward(4000, seed=3)
    rec, flags = oracle.project(scene, cam, oracle.Opts(antialiased=False))
    vis = (flags & 1).astype(bool)
    assert (rec[vis, 5] > 0.99).sum() >= 10
