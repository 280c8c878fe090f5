"""Host logic of the serving loop's detail levels (no GPU): the opacity-weighted merge that
stands in for the paper's trained levels (Sec. 3.4.1) and the level layout that the LOD
selection reads (Sec. 3.4.2), checked against the moments they must preserve and the index
invariants of the layout."""
import numpy as np

from paper_2507_23006_gb300 import lod, scenes


def _rot(q):
    q = np.asarray(q, np.float64)
    return lod._quat_to_rot(q[None] / np.linalg.norm(q))[0]


def test_quaternion_rotation_round_trip():
    rng = np.random.default_rng(0)
    q = rng.normal(size=(500, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    R = lod._quat_to_rot(q)
    np.testing.assert_allclose(np.einsum("nij,nkj->nik", R, R), np.broadcast_to(np.eye(3), R.shape), atol=1e-12)
    np.testing.assert_allclose(np.linalg.det(R), 1.0, atol=1e-12)
    back = lod._rot_to_quat(R)
    sign = np.sign(np.sum(back * q, axis=1))[:, None]  # q and -q are the same rotation
    np.testing.assert_allclose(back * sign, q, atol=1e-9)


def test_two_gaussians_merge_to_their_weighted_moments():
    means = np.array([[0.0, 0.0, 0.0], [0.4, -0.2, 0.1]], np.float32)
    scales = np.array([[0.3, 0.1, 0.2], [0.05, 0.25, 0.15]], np.float32)
    quats = np.array([[1.0, 0.0, 0.0, 0.0], [0.9, 0.3, -0.2, 0.1]], np.float32)
    opac = np.array([0.6, 0.3], np.float32)
    sh = np.random.default_rng(1).normal(size=(2, 16, 3)).astype(np.float32)
    merged = lod.merge_to_count(scenes.Scene(means, scales, quats, opac, sh, 3), 1, extent=100.0, device="cpu")
    assert merged.n == 1
    w = opac.astype(np.float64)
    mu = (w[:, None] * means).sum(0) / w.sum()
    cov = np.zeros((3, 3))
    for i in range(2):
        R = _rot(quats[i])
        d = means[i] - mu
        cov += w[i] * (R @ np.diag(scales[i].astype(np.float64) ** 2) @ R.T + np.outer(d, d))
    cov /= w.sum()
    np.testing.assert_allclose(merged.means[0], mu, atol=1e-6)
    R = _rot(merged.quats[0])
    got = R @ np.diag(merged.scales[0].astype(np.float64) ** 2) @ R.T
    np.testing.assert_allclose(got, cov, rtol=1e-4, atol=1e-7)
    np.testing.assert_allclose(merged.opacities[0], 1 - (1 - 0.6) * (1 - 0.3), atol=1e-6)
    np.testing.assert_allclose(merged.sh[0], (w[:, None, None] * sh).sum(0) / w.sum(), atol=1e-5)


def test_merge_reaches_the_target_count_and_clamps_opacity():
    sc = scenes.city(5, 20_000)
    out = lod.merge_to_count(sc, 5_000, device="cpu")
    assert abs(out.n - 5_000) <= 0.02 * 5_000
    assert np.all(out.opacities > 0) and np.all(out.opacities <= 0.99 + 1e-6)
    np.testing.assert_allclose(np.linalg.norm(out.quats, axis=1), 1.0, atol=1e-5)
    assert np.all(out.scales > 0)


def test_level_layout_is_what_the_selection_reads():
    fine = scenes.city(6, 8_000)
    mid = lod.merge_to_count(fine, 2_000, device="cpu")
    coarse = lod.merge_to_count(mid, 500, device="cpu")
    L = lod.build_lod([coarse, mid, fine], part_size=100.0, extent=1000.0)
    P = 100
    assert L.level_sizes == [coarse.n, mid.n, fine.n]
    assert L.gaussians.n == coarse.n + mid.n + fine.n
    assert L.aabb.shape == (P, 6) and L.level_offsets.shape == (3, P + 1)
    base = 0
    for lvl, sc in enumerate([coarse, mid, fine]):
        off = L.level_offsets[lvl]
        assert off[0] == base and off[-1] == base + sc.n and np.all(np.diff(off) >= 0)
        m = np.asarray(L.gaussians.means[base:base + sc.n], np.float64)
        r = 3.0 * np.asarray(L.gaussians.scales[base:base + sc.n], np.float64).max(axis=1)
        ij = np.clip(np.floor((m[:, :2] + 500.0) / 100.0).astype(np.int64), 0, 9)
        part = ij[:, 0] * 10 + ij[:, 1]
        assert np.all(np.diff(part) >= 0)  # each level sorted by partition
        for p in range(P):  # the offsets delimit each partition's run
            assert np.all(part[off[p] - base:off[p + 1] - base] == p)
        box = L.aabb[part]
        assert np.all(m - r[:, None] >= box[:, :3] - 1e-9) and np.all(m + r[:, None] <= box[:, 3:] + 1e-9)
        base += sc.n
