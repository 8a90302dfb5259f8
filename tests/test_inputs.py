"""The seeded synthetic inputs follow their stated recipes (no GPU).

The paper's Replica / MP3D rooms are replaced by generated scenes; these
tests check that the generator produces what the recipes say: value
ranges, distributions (sample statistics within a few standard errors),
the surface / blob split of the room, the orientation of surface Gaussians
(thinnest axis along the face normal), distinct top-k class ids with
descending Dirichlet weights, the perturbed target copy, the candidate pose
sets and the dense comparator's distributions.
"""
import math

import numpy as np
import pytest

from paper_2506_00225_gb300 import scenes


def _rot(q):
    """Rotation matrices of unit quaternions (w, x, y, z), written out."""
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ], 1)


def _check_semantics(sc, k, m):
    assert sc.sem_ids.shape == (sc.n, k) and sc.sem_w.shape == (sc.n, k)
    assert sc.sem_ids.min() >= 0 and sc.sem_ids.max() < m
    srt = np.sort(sc.sem_ids, axis=1)
    assert (np.diff(srt, axis=1) > 0).all(), "top-k ids of a Gaussian must be distinct"
    assert (np.diff(sc.sem_w, axis=1) <= 0).all(), "weights sorted descending"
    np.testing.assert_allclose(sc.sem_w.sum(1), 1.0, atol=1e-5)
    # Dirichlet(1) over k: the largest of k uniform-simplex weights has mean H_k / k
    hk = sum(1.0 / i for i in range(1, k + 1))
    assert abs(sc.sem_w[:, 0].mean() - hk / k) < 0.01


def test_plain_scene_recipe():
    sc = scenes.scene_plain(0, n=20_000, m=16, k=3)
    assert sc.n == 20_000 and sc.m == 16
    lo, hi = sc.means.min(0), sc.means.max(0)
    assert (lo >= [-2, -2, 0]).all() and (hi <= [2, 2, 3]).all()
    ls = np.log(sc.scales.astype(np.float64))
    assert abs(ls.mean() + 3.0) < 0.02 and abs(ls.std() - 0.5) < 0.02
    np.testing.assert_allclose(np.linalg.norm(sc.quats, axis=1), 1.0, atol=1e-6)
    logit = np.log(sc.opacity / (1 - sc.opacity))
    assert abs(logit.mean()) < 0.03 and abs(logit.std() - 1.0) < 0.03
    assert sc.rgb.min() >= 0 and sc.rgb.max() <= 1 and abs(sc.rgb.mean() - 0.5) < 0.01
    _check_semantics(sc, 3, 16)


def test_room_scene_recipe():
    n = 40_000
    sc = scenes.scene_room(1, n, 102, 3)
    assert sc.n == n and sc.m == 102
    p = sc.means.astype(np.float64)
    # distance to the nearest of the six faces of the 6 x 6 x 3 m room
    dist = np.min(np.stack([np.abs(p[:, 0]), np.abs(p[:, 0] - 6), np.abs(p[:, 1]), np.abs(p[:, 1] - 6),
                            np.abs(p[:, 2]), np.abs(p[:, 2] - 3)], 1), axis=1)
    on_face = dist < 0.05        # five standard deviations of the 1 cm normal jitter
    frac = on_face.mean()
    assert 0.70 <= frac < 0.72, frac  # 70 % on faces, a few blob Gaussians near a face
    # surface Gaussians: the thinnest axis (log-scale ~ -6) lies along the face normal
    ls = np.log(sc.scales.astype(np.float64))
    thin = ls[:, 2] < -5.0
    surf = on_face & thin
    assert surf.mean() > 0.68
    axis_z = _rot(sc.quats.astype(np.float64))[:, :, 2]
    nearest = np.argmin(np.stack([np.abs(p[:, 0]), np.abs(p[:, 0] - 6), np.abs(p[:, 1]), np.abs(p[:, 1] - 6),
                                  np.abs(p[:, 2]), np.abs(p[:, 2] - 3)], 1), axis=1)
    normal_axis = np.array([0, 0, 1, 1, 2, 2])[nearest]
    comp = np.abs(axis_z[surf, normal_axis[surf]])
    assert np.median(comp) > 0.999
    assert abs(ls[surf, 0].mean() + 3.5) < 0.02 and abs(ls[surf, 0].std() - 0.3) < 0.02
    assert abs(ls[surf, 2].mean() + 6.0) < 0.02
    # blobs: the other 30 %, centred in [0.5, 5.5]^2 x [0, 1.5] with 0.25 m spread
    blob = ~thin
    assert 0.29 < blob.mean() < 0.31
    assert abs(ls[blob].mean() + 3.5) < 0.02 and abs(ls[blob].std() - 0.5) < 0.02
    logit = np.log(sc.opacity.astype(np.float64) / (1 - sc.opacity))
    assert abs(logit.mean() - 1.0) < 0.03 and abs(logit.std() - 1.0) < 0.03
    assert sc.rgb.min() >= 0 and sc.rgb.max() <= 1
    _check_semantics(sc, 3, 102)
    # the Gaussian index carries no spatial order (shuffled)
    assert abs(np.corrcoef(np.arange(n), p[:, 0])[0, 1]) < 0.03


def test_rooms_layout_and_top8():
    sc = scenes.scene_rooms(3, 8_000, 256, 8, (2, 2))
    p = sc.means
    # blob centres lie 0.5 m inside the walls with a 0.25 m spread, so a few
    # blob Gaussians reach a little past a wall
    assert p[:, 0].min() > -0.75 and p[:, 0].max() < 12.75 and p[:, 1].min() > -0.75 and p[:, 1].max() < 12.75
    quad = (p[:, 0] > 6).astype(int) + 2 * (p[:, 1] > 6).astype(int)
    counts = np.bincount(quad, minlength=4)
    assert counts.min() > 0.2 * sc.n, counts  # one room per quadrant
    _check_semantics(sc, 8, 256)


def test_perturbed_target_copy():
    sc = scenes.scene_room(1, 20_000, 102, 3)
    tg = scenes.perturbed_copy(sc, 101)
    dm = (tg.means - sc.means).astype(np.float64)
    assert abs(dm.std() - 0.01) < 5e-4
    np.testing.assert_array_equal(tg.scales, sc.scales)
    np.testing.assert_array_equal(tg.quats, sc.quats)
    np.testing.assert_array_equal(tg.sem_ids, sc.sem_ids)
    assert tg.rgb.min() >= 0 and tg.rgb.max() <= 1
    lo = np.log(sc.opacity.astype(np.float64) / (1 - sc.opacity))
    lt = np.log(tg.opacity.astype(np.float64) / (1 - tg.opacity))
    assert abs((lt - lo).std() - 0.3) < 0.01
    assert tg.sem_w.min() >= 0
    dw = (tg.sem_w - sc.sem_w)[tg.sem_w > 0]
    assert abs(dw.std() - 0.05) < 0.005


def test_candidate_pose_sets():
    g = [2.25, 2.75, 3.25, 3.75]
    cams = scenes.candidate_cameras_grid(g, g)
    assert len(cams) == 96
    sizes = [(c.height, c.width, c.fx) for c in cams]
    for v, s in enumerate(sizes):
        assert s == [(170, 300, 150.0), (340, 600, 300.0), (680, 1200, 600.0)][v % 3]
    pos = np.array([c.position() for c in cams])
    assert set(np.round(pos[:, 0], 6)) == set(g) and set(np.round(pos[:, 1], 6)) == set(g)
    np.testing.assert_allclose(pos[:, 2], 1.5, atol=1e-5)
    # six yaws 60 degrees apart at each position: camera z axes (rows of R)
    fwd = np.array([c.w2c[2, :3] for c in cams[:6]], np.float64)
    yaw = np.degrees(np.arctan2(fwd[:, 1], fwd[:, 0])) % 360
    np.testing.assert_allclose(np.sort(yaw), [0, 60, 120, 180, 240, 300], atol=1e-4)
    np.testing.assert_allclose(fwd[:, 2], 0.0, atol=1e-6)


def test_dense_comparator_distributions():
    sc = scenes.scene_room(6, 5_000, 102, 3)
    d = scenes.dense_distributions(sc, 7).astype(np.float64)
    assert d.shape == (sc.n, 102) and (d > 0).all()
    np.testing.assert_allclose(d.sum(1), 1.0, atol=1e-5)
    w = sc.sem_w.astype(np.float64)
    w /= w.sum(1, keepdims=True)
    top = np.take_along_axis(d, sc.sem_ids.astype(np.int64), 1)
    assert (top >= 0.9 * w - 1e-6).all()
    sparse = scenes.sparse_to_dense(sc)
    np.testing.assert_array_equal(np.take_along_axis(sparse, sc.sem_ids.astype(np.int64), 1), sc.sem_w)
    assert (sparse > 0).sum() == (sc.sem_w > 0).sum()


@pytest.mark.parametrize("yaw", [0.0, 45.0, 200.0])
def test_look_camera_principal_axis(yaw):
    cam = scenes.look_camera((1.0, 2.0, 1.5), yaw, 600, 340, 300.0)
    assert (cam.cx, cam.cy) == (300.0, 170.0)
    R = cam.w2c[:, :3].astype(np.float64)
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-6)
    assert np.linalg.det(R) > 0
    ahead = np.array([1.0 + math.cos(math.radians(yaw)), 2.0 + math.sin(math.radians(yaw)), 1.5])
    pc = R @ ahead + cam.w2c[:, 3]
    np.testing.assert_allclose(pc, [0.0, 0.0, 1.0], atol=1e-5)
    # image y points down: a point above the camera projects above the centre
    above = R @ np.array([1.0 + math.cos(math.radians(yaw)), 2.0 + math.sin(math.radians(yaw)), 2.0]) + cam.w2c[:, 3]
    assert above[1] < 0
