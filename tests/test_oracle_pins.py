"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed
forms, a numerically differentiated projection, the literal product form of
Eq. 1, invariants of Eq. 1 / Eq. 3, central finite differences, and brute
force on tiny inputs.  None of these needs a GPU.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2506_00225_gb300.scenes import Camera, Scene, scene_plain, look_camera

ALPHA_MIN = np.float32(1.0) / np.float32(255.0)


def ident_cam(W, H, f, near=0.2):
    w2c = np.zeros((3, 4), np.float32)
    w2c[:, :3] = np.eye(3, dtype=np.float32)
    return Camera(W, H, float(f), float(f), W / 2.0, H / 2.0, near, w2c)


def mk_scene(means, scales, quats, opacity, rgb=None, ids=None, w=None, m=4, unc=None):
    n = len(means)
    rgb = np.full((n, 3), 0.5) if rgb is None else rgb
    ids = np.zeros((n, 1), np.int32) if ids is None else ids
    w = np.ones((n, ids.shape[1])) if w is None else w
    f = lambda a: np.ascontiguousarray(np.asarray(a, np.float64).astype(np.float32))
    return Scene(f(means), f(scales), f(quats), f(opacity), f(rgb), np.ascontiguousarray(ids, np.int32), f(w), m,
                 None if unc is None else f(unc))


def rand_quat(rng, n):
    q = rng.normal(size=(n, 4))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def quat_to_rot(q):
    """Rotation matrix of a unit quaternion (w, x, y, z) via the axis-angle
    (Rodrigues) formula -- an independent route from the oracle's."""
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q)
    w, v = q[0], q[1:]
    s = np.linalg.norm(v)
    if s < 1e-15:
        return np.eye(3)
    axis = v / s
    ang = 2.0 * math.atan2(s, w)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * (K @ K)


# --------------------------------------------------------------------------
# projection
# --------------------------------------------------------------------------

def test_isotropic_on_axis_closed_form():
    """A single isotropic Gaussian on the optical axis renders
    alpha(p) = o exp(-rho^2 / (2 ((f s / z)^2 + 0.3))) (Eq. 1 with one term,
    pinhole projection of an isotropic 3D Gaussian), for any rotation."""
    rng = np.random.default_rng(7)
    W = H = 41
    f, z, s, o = 40.0, 2.0, 0.15, 0.8
    cam = ident_cam(W, H, f)
    for q in [np.array([1.0, 0, 0, 0]), rand_quat(rng, 1)[0], rand_quat(rng, 1)[0]]:
        sc = mk_scene([[0.0, 0.0, z]], [[s, s, s]], [q], [o], rgb=[[1.0, 0.25, 0.5]])
        r = oracle.render(sc, cam, prec="f64")
        # the scene stores float32 values; the closed form uses those
        s32, z32, o32 = float(np.float32(s)), float(np.float32(z)), float(np.float32(o))
        var = (f * s32 / z32) ** 2 + 0.3
        lam = var + math.sqrt(0.1)  # eigenvalue floor of the radius rule
        rad = math.ceil(3 * math.sqrt(lam))
        ys, xs = np.mgrid[0:H, 0:W]
        dx = xs + 0.5 - W / 2.0
        dy = ys + 0.5 - H / 2.0
        a = np.minimum(0.99, o32 * np.exp(-0.5 * (dx ** 2 + dy ** 2) / var))
        inside = (np.abs(dx) <= rad) & (np.abs(dy) <= rad) & (a >= 1 / 255)
        expect = np.where(inside, a, 0.0)
        np.testing.assert_allclose(r["sil"], expect, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(r["rgb"][..., 1], 0.25 * expect, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(r["depth"], z32 * expect, rtol=1e-12, atol=1e-14)


def test_isotropic_on_axis_anisotropic_focal_lengths():
    """The same Gaussian seen through fx != fy renders the axis-aligned
    ellipse alpha(p) = o exp(-(dx^2 / var_x + dy^2 / var_y) / 2), var_x =
    (fx s / z)^2 + 0.3, var_y = (fy s / z)^2 + 0.3, inside the square of half
    size ceil(3 sqrt(lambda_max)) (lambda_max = var_x: the eigenvalue gap
    exceeds the floor)."""
    W = H = 41
    fx, fy, z, s, o = 40.0, 24.0, 2.0, 0.15, 0.8
    w2c = np.zeros((3, 4), np.float32)
    w2c[:, :3] = np.eye(3, dtype=np.float32)
    cam = Camera(W, H, fx, fy, W / 2.0, H / 2.0, 0.2, w2c)
    sc = mk_scene([[0.0, 0.0, z]], [[s, s, s]], [[1.0, 0, 0, 0]], [o])
    r = oracle.render(sc, cam, prec="f64")
    s32, z32, o32 = float(np.float32(s)), float(np.float32(z)), float(np.float32(o))
    vx, vy = (fx * s32 / z32) ** 2 + 0.3, (fy * s32 / z32) ** 2 + 0.3
    assert ((vx - vy) / 2) ** 2 > 0.1
    rad = math.ceil(3 * math.sqrt(vx))
    ys, xs = np.mgrid[0:H, 0:W]
    dx = xs + 0.5 - W / 2.0
    dy = ys + 0.5 - H / 2.0
    a = np.minimum(0.99, o32 * np.exp(-0.5 * (dx ** 2 / vx + dy ** 2 / vy)))
    inside = (np.abs(dx) <= rad) & (np.abs(dy) <= rad) & (a >= 1 / 255)
    np.testing.assert_allclose(r["sil"], np.where(inside, a, 0.0), rtol=1e-12, atol=1e-14)


def test_row_sample_renders_exactly_its_rows():
    """rows = (begin, end, step) renders rows begin, begin + step, ... below
    end, each equal to the full render's row, and leaves every other row
    (including those past end on the same stride) at zero."""
    rng = np.random.default_rng(12)
    cam = ident_cam(24, 20, 18.0)
    n = 60
    z = rng.uniform(1.0, 3.0, n)
    means = np.stack([rng.uniform(-0.5, 0.5, n) * z, rng.uniform(-0.5, 0.5, n) * z, z], 1)
    sc = mk_scene(means, np.exp(rng.normal(-1.8, 0.3, (n, 3))), rand_quat(rng, n), rng.uniform(0.3, 0.9, n))
    full = oracle.render(sc, cam, prec="f32")
    part = oracle.render(sc, cam, prec="f32", rows=(2, 10, 3))
    sel = np.zeros(cam.height, bool)
    sel[[2, 5, 8]] = True
    for key in ("rgb", "depth", "sil", "sem"):
        np.testing.assert_array_equal(part[key][sel], full[key][sel], err_msg=key)
        assert not part[key][~sel].any(), key
    assert full["sil"][[11, 14, 17]].any()  # rows the sample must leave out are not empty


def test_near_threshold_flags():
    """A pixel is flagged when a threshold decision lies within a relative
    1e-5 of its threshold: bit 1 for alpha at the 1/255 skip or the
    transmittance at the 1e-4 stop, bit 2 for alpha at the 0.99 cap.  On a
    1 x 1 view a Gaussian centred on the pixel has G = 1, so alpha is its
    opacity."""
    w2c = np.zeros((3, 4), np.float32)
    w2c[:, :3] = np.eye(3, dtype=np.float32)
    cam = Camera(1, 1, 10.0, 10.0, 0.5, 0.5, 0.2, w2c)

    def flag(opacities, depths):
        n = len(opacities)
        sc = mk_scene([[0.0, 0.0, d] for d in depths], [[0.2, 0.2, 0.2]] * n, [[1.0, 0, 0, 0]] * n, opacities)
        return int(oracle.render(sc, cam, prec="f32")["flag"][0, 0])

    assert flag([0.5], [2.0]) == 0
    assert flag([(1 / 255) * (1 + 1e-7)], [2.0]) & 1
    assert flag([(1 / 255) * (1 - 1e-7)], [2.0]) & 1
    assert flag([(1 / 255) * 1.01], [2.0]) == 0
    assert flag([(1 / 255) * 1.001], [2.0]) == 0  # the margin is relative: 1e-5 of 1/255
    assert flag([(1 / 255) * 1.0005], [2.0]) == 0
    assert flag([0.99 * (1 + 1e-6)], [2.0]) == 2
    assert flag([0.99 * (1 - 1e-6)], [2.0]) == 2
    assert flag([0.98], [2.0]) == 0
    # two capped Gaussians: T = 0.01, then 1e-4 within rounding of the stop
    assert flag([0.995, 0.995], [2.0, 3.0]) & 1
    assert flag([0.9, 0.9], [2.0, 3.0]) == 0


def _proj_numeric(mean, scale, q, cam):
    """EWA linearisation by numerical differentiation of the pinhole map
    (world point -> pixel) at the mean, in float64."""
    w2c = cam.w2c.astype(np.float64)

    def pix(X):
        t = w2c[:, :3] @ X + w2c[:, 3]
        return np.array([cam.fx * t[0] / t[2] + cam.cx, cam.fy * t[1] / t[2] + cam.cy])

    h = 1e-6
    J = np.zeros((2, 3))
    for i in range(3):
        e = np.zeros(3); e[i] = h
        J[:, i] = (pix(mean + e) - pix(mean - e)) / (2 * h)
    R = quat_to_rot(q)
    S3 = R @ np.diag(np.asarray(scale, np.float64) ** 2) @ R.T
    S2 = J @ S3 @ J.T + 0.3 * np.eye(2)
    return pix(mean), S2


def test_projection_matches_numeric_jacobian():
    rng = np.random.default_rng(11)
    cam = look_camera((0.3, -0.2, 1.4), 25.0, 96, 64, 70.0, pitch_deg=-10.0)
    n = 200
    c2w_r = cam.w2c[:, :3].astype(np.float64).T
    pos = cam.position()
    # points in front of the camera, inside the frustum clamp
    tc = np.stack([rng.uniform(-0.5, 0.5, n), rng.uniform(-0.35, 0.35, n), rng.uniform(1.0, 4.0, n)], 1)
    tc[:, 0] *= tc[:, 2]
    tc[:, 1] *= tc[:, 2]
    means = tc @ c2w_r.T + pos
    scales = np.exp(rng.normal(-2.5, 0.6, size=(n, 3)))
    quats = rand_quat(rng, n) * rng.uniform(0.5, 2.0, size=(n, 1))  # not unit
    sc = mk_scene(means, scales, quats, np.full(n, 0.5))
    p = oracle.project(sc, cam, prec="f64")
    checked = 0
    for i in range(n):
        if not p["visible"][i]:
            continue
        uv, S2 = _proj_numeric(sc.means[i].astype(np.float64), sc.scales[i], sc.quats[i], cam)
        np.testing.assert_allclose(p["uv"][i], uv, rtol=0, atol=1e-6)
        conic = np.linalg.inv(S2)
        np.testing.assert_allclose(p["conic"][i], [conic[0, 0], conic[0, 1], conic[1, 1]], rtol=2e-6, atol=1e-9)
        ev = np.linalg.eigvalsh(S2)
        mid = 0.5 * (ev[0] + ev[1])
        lam = mid + math.sqrt(max(0.1, (0.5 * (ev[1] - ev[0])) ** 2))
        assert p["radius"][i] == math.ceil(3 * math.sqrt(lam)) or abs(3 * math.sqrt(lam) - round(3 * math.sqrt(lam))) < 1e-6
        t = cam.w2c[:, :3].astype(np.float64) @ sc.means[i] + cam.w2c[:, 3]
        assert abs(p["depth"][i] - t[2]) < 1e-12
        checked += 1
    assert checked > 150


def test_frustum_clamp_of_the_jacobian():
    """A Gaussian beyond 1.3 tan(half field of view) of the optical axis is
    linearised at the clamped point (x/z clamped to +-1.3 (W/2)/f, y/z to
    +-1.3 (H/2)/f): its conic equals the EWA form with a numerically
    differentiated pinhole map at that point, and differs from the one at its
    own mean; one within the limit is linearised at its mean.  A square and
    a wide view, offsets along x and along y, inside and beyond each axis's
    limit."""
    f, z, s = 40.0, 2.0, 0.5
    for W, H in ((41, 41), (61, 31)):
        cam = ident_cam(W, H, f)
        lims = (1.3 * (W / 2.0) / f, 1.3 * (H / 2.0) / f)
        for axis in (0, 1):
            for off in (0.3, 0.8, 1.2):
                for sign in (1.0, -1.0):
                    mean = np.array([0.1, 0.1, z])
                    mean[axis] = sign * off * z
                    sc = mk_scene([mean], [[s, s, s]], [[1, 0, 0, 0]], [0.9])
                    p = oracle.project(sc, cam, prec="f64")
                    assert p["visible"][0], (W, H, axis, off, sign)
                    m32 = np.asarray(sc.means[0], np.float64)
                    s32 = float(sc.scales[0, 0])

                    def pix(X):
                        return np.array([f * X[0] / X[2] + W / 2.0, f * X[1] / X[2] + H / 2.0])

                    def ewa_conic(X):
                        J = np.zeros((2, 3))
                        for i in range(3):
                            e = np.zeros(3); e[i] = 1e-6
                            J[:, i] = (pix(X + e) - pix(X - e)) / 2e-6
                        S2 = J @ (s32 ** 2 * np.eye(3)) @ J.T + 0.3 * np.eye(2)
                        inv = np.linalg.inv(S2)
                        return np.array([inv[0, 0], inv[0, 1], inv[1, 1]])

                    clamped = np.array([np.clip(m32[0] / m32[2], -lims[0], lims[0]) * m32[2],
                                        np.clip(m32[1] / m32[2], -lims[1], lims[1]) * m32[2], m32[2]])
                    np.testing.assert_allclose(p["conic"][0], ewa_conic(clamped), rtol=1e-6)
                    if abs(m32[axis] / m32[2]) > lims[axis]:
                        assert np.abs(p["conic"][0] - ewa_conic(m32)).max() > 1e-3 * np.abs(p["conic"][0]).max()


def test_near_plane_culls_at_and_before_it():
    """t_z <= near (0.2 m) is culled, just beyond it is kept."""
    cam = ident_cam(9, 9, 8.0, near=0.2)
    zs = [0.19, 0.2, 0.21, 0.25]
    sc = mk_scene([[0.0, 0.0, z] for z in zs], [[0.01, 0.01, 0.01]] * 4, [[1, 0, 0, 0]] * 4, [0.5] * 4)
    p = oracle.project(sc, cam, prec="f64")
    assert list(p["visible"]) == [False, False, True, True]


def test_opacity_cap_and_equal_depth_order():
    """alpha is capped at 0.99 (a Gaussian of opacity 0.999 leaves S = 0.99
    at its centre); Gaussians at exactly equal depth composite in ascending
    index order."""
    cam = ident_cam(1, 1, 10.0)
    sc = mk_scene([[0.0, 0.0, 1.0]], [[1.0, 1.0, 1.0]], [[1, 0, 0, 0]], [0.999])
    r = oracle.render(sc, cam, prec="f64")
    assert abs(r["sil"][0, 0] - 0.99) < 1e-15
    sc = mk_scene([[0.0, 0.0, 1.0]] * 2, [[1.0, 1.0, 1.0]] * 2, [[1, 0, 0, 0]] * 2, [0.5, 0.5],
                  rgb=[[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    r = oracle.render(sc, cam, prec="f64")
    np.testing.assert_allclose(r["rgb"][0, 0], [0.5, 0.25, 0.0], atol=1e-15)


def test_uncertainty_composited_like_colour_and_hole_count():
    """Per-Gaussian uncertainty is composited by Eq. 1 (U = u1 a1 + u2 a2 (1 - a1)
    for two stacked Gaussians at the pixel centre); N_S counts only pixels
    with S exactly 0, not faint ones (S = 0.005)."""
    cam = ident_cam(1, 1, 10.0)
    sc = mk_scene([[0.0, 0.0, 1.0], [0.0, 0.0, 1.5]], [[1.0, 1.0, 1.0]] * 2, [[1, 0, 0, 0]] * 2, [0.5, 0.6],
                  unc=[2.0, 3.0])
    r = oracle.render(sc, cam, prec="f64", unc=True)
    a1, a2 = 0.5, float(np.float32(0.6))
    assert abs(r["unc"][0, 0] - (2.0 * a1 + 3.0 * a2 * (1 - a1))) < 1e-12
    su, sh, ns, nf = oracle.candidate(sc, cam, prec="f64")
    assert abs(su - (2.0 * a1 + 3.0 * a2 * (1 - a1))) < 1e-12 and ns == 0
    faint = mk_scene([[0.0, 0.0, 1.0]], [[1.0, 1.0, 1.0]], [[1, 0, 0, 0]], [0.005], unc=[1.0])
    assert abs(oracle.render(faint, cam, prec="f64")["sil"][0, 0] - float(np.float32(0.005))) < 1e-12
    assert oracle.candidate(faint, cam, prec="f64")[2] == 0
    behind = mk_scene([[0.0, 0.0, -1.0]], [[1.0, 1.0, 1.0]], [[1, 0, 0, 0]], [0.5], unc=[1.0])
    assert oracle.candidate(behind, cam, prec="f64")[2] == 1


def test_rect_rule_bruteforce_and_tiles():
    """Pixel rectangle = bounding set of pixels whose centre lies within the
    radius of the 2D mean (per axis); tile rectangle = tiles it touches."""
    sc = scene_plain(0, n=3000)
    cam = look_camera((0.0, 0.0, 1.5), 0.0, 100, 70, 80.0)
    for tile in [(16, 16), (8, 8), (32, 8)]:
        p = oracle.project(sc, cam, tile=tile, prec="f32")
        for i in np.nonzero(p["visible"])[0][:400]:
            u, v = p["uv"][i].astype(np.float64)
            r = float(p["radius"][i])
            xs = np.arange(cam.width)
            ys = np.arange(cam.height)
            okx = xs[np.abs(xs + 0.5 - u) <= r]
            oky = ys[np.abs(ys + 0.5 - v) <= r]
            x0, x1, y0, y1 = p["rect"][i]
            assert (okx.min(), okx.max(), oky.min(), oky.max()) == (x0, x1, y0, y1)
            tx0, tx1, ty0, ty1 = p["trect"][i]
            assert (tx0, tx1, ty0, ty1) == (x0 // tile[0], x1 // tile[0], y0 // tile[1], y1 // tile[1])
            assert p["ntiles"][i] == (tx1 - tx0 + 1) * (ty1 - ty0 + 1)
        assert not p["visible"][p["depth"] <= cam.near].any()


def test_tile_lists_bruteforce_and_tiebreak():
    """Each tile's list = Gaussians whose tile rectangle holds the tile,
    front to back by depth, ties by gid (Sec. 3.1 front-to-back sort)."""
    rng = np.random.default_rng(3)
    n = 300
    cam = ident_cam(64, 48, 50.0)
    z = rng.choice([1.5, 2.0, 2.5], size=n)  # many exactly equal depths
    means = np.stack([rng.uniform(-0.6, 0.6, n) * z, rng.uniform(-0.45, 0.45, n) * z, z], 1)
    sc = mk_scene(means, np.exp(rng.normal(-3, 0.4, (n, 3))), rand_quat(rng, n), np.full(n, 0.5))
    p = oracle.project(sc, cam, prec="f32")
    ranges, gids, offs = oracle.tile_lists([p], [cam])
    gx, gy = oracle.tiles_of(cam)
    for t in range(gx * gy):
        tx, ty = t % gx, t // gx
        members = [g for g in range(n) if p["visible"][g] and p["trect"][g][0] <= tx <= p["trect"][g][1]
                   and p["trect"][g][2] <= ty <= p["trect"][g][3]]
        members.sort(key=lambda g: (float(p["depth"][g]), g))
        s, e = ranges[t]
        assert list(gids[s:e]) == members


def test_tile_lists_several_ragged_views():
    """Two views, one of them ragged (57 x 41 with 16 x 16 tiles: the last
    column and row of tiles are partial): view v's tiles follow all tiles
    of the views before it, each view has ceil(W / 16) x ceil(H / 16) tiles
    numbered row-major, and each tile holds its view's Gaussians whose tile
    rectangle contains it, front to back, ties by gid."""
    rng = np.random.default_rng(4)
    n = 200
    cams = [ident_cam(64, 48, 50.0), ident_cam(57, 41, 45.0)]
    z = rng.choice([1.5, 2.0, 2.5], size=n)
    means = np.stack([rng.uniform(-0.7, 0.7, n) * z, rng.uniform(-0.55, 0.55, n) * z, z], 1)
    sc = mk_scene(means, np.exp(rng.normal(-3, 0.4, (n, 3))), rand_quat(rng, n), np.full(n, 0.5))
    projs = [oracle.project(sc, cam, prec="f32") for cam in cams]
    ranges, gids, offs = oracle.tile_lists(projs, cams)
    counts = [((c.width + 15) // 16) * ((c.height + 15) // 16) for c in cams]
    assert counts == [12, 12] and offs.tolist() == [0, 12, 24] and len(ranges) == 24
    for v, (p, cam) in enumerate(zip(projs, cams)):
        gx = (cam.width + 15) // 16
        for t in range(counts[v]):
            tx, ty = t % gx, t // gx
            members = [g for g in range(n) if p["visible"][g] and p["trect"][g][0] <= tx <= p["trect"][g][1]
                       and p["trect"][g][2] <= ty <= p["trect"][g][3]]
            members.sort(key=lambda g: (float(p["depth"][g]), g))
            s_, e = ranges[offs[v] + t]
            assert list(gids[s_:e]) == members, (v, t)
    # the ragged view's partial tiles are reached
    assert any(projs[1]["trect"][g][1] == 3 for g in range(n) if projs[1]["visible"][g])


# --------------------------------------------------------------------------
# compositing (Eq. 1, Eq. 3)
# --------------------------------------------------------------------------

def _tiny_scene(rng, n, m=6, k=2, omax=0.8):
    cam = ident_cam(16, 16, 14.0)
    z = rng.uniform(1.0, 3.0, n)
    means = np.stack([rng.uniform(-0.4, 0.4, n) * z, rng.uniform(-0.4, 0.4, n) * z, z], 1)
    scales = np.exp(rng.normal(-1.6, 0.4, (n, 3)))
    ids = np.stack([rng.choice(m, k, replace=False) for _ in range(n)]).astype(np.int32)
    w = rng.dirichlet(np.ones(k), n)
    sc = mk_scene(means, scales, rand_quat(rng, n), rng.uniform(0.2, omax, n), rgb=rng.uniform(0, 1, (n, 3)),
                  ids=ids, w=w, m=m)
    return sc, cam


def test_product_form_tiny_scenes():
    """Eq. 1 and Eq. 3 evaluated literally -- sum_i z_i f_i prod_{j<i}(1-f_j)
    over the depth-sorted candidates -- match the oracle on tiny scenes."""
    rng = np.random.default_rng(5)
    for trial in range(6):
        sc, cam = _tiny_scene(rng, 5)
        p = oracle.project(sc, cam, prec="f64")
        r = oracle.render(sc, cam, prec="f64")
        order = sorted(np.nonzero(p["visible"])[0], key=lambda g: (p["depth"][g], g))
        for y in range(cam.height):
            for x in range(cam.width):
                fs, zs = [], []
                for g in order:
                    x0, x1, y0, y1 = p["rect"][g]
                    if not (x0 <= x <= x1 and y0 <= y <= y1):
                        continue
                    dx, dy = p["uv"][g][0] - (x + 0.5), p["uv"][g][1] - (y + 0.5)
                    a, b, c = p["conic"][g]
                    pw = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
                    al = min(0.99, float(sc.opacity[g]) * math.exp(pw))
                    if pw > 0 or al < 1 / 255:
                        continue
                    fs.append(al)
                    zs.append(g)
                wts = [fs[i] * np.prod([1 - fs[j] for j in range(i)]) for i in range(len(fs))]
                assert np.prod([1 - f for f in fs]) >= 1e-4  # no early stop in these scenes
                sil = sum(wts)
                col = sum(wi * sc.rgb[g].astype(np.float64) for wi, g in zip(wts, zs)) if zs else np.zeros(3)
                dep = sum(wi * p["depth"][g] for wi, g in zip(wts, zs))
                sem = np.zeros(sc.m)
                for wi, g in zip(wts, zs):
                    for j in range(sc.k):
                        sem[sc.sem_ids[g, j]] += wi * float(sc.sem_w[g, j])
                assert abs(r["sil"][y, x] - sil) < 1e-12
                np.testing.assert_allclose(r["rgb"][y, x], col, atol=1e-12)
                assert abs(r["depth"][y, x] - dep) < 1e-12
                np.testing.assert_allclose(r["sem"][y, x], sem, atol=1e-12)


def test_transmittance_stop_rule():
    """Stacked Gaussians with alpha = 0.95 each: T after 3 is 1.25e-4, the
    4th would take it below 1e-4, so exactly 3 contribute and
    S = 1 - 0.05^3 at the centre pixel."""
    cam = ident_cam(3, 3, 10.0)
    n = 6
    means = [[0.0, 0.0, 1.0 + 0.1 * i] for i in range(n)]
    sc = mk_scene(means, [[1.0, 1.0, 1.0]] * n, [[1, 0, 0, 0]] * n, [0.95] * n)
    r = oracle.render(sc, cam, prec="f64")
    # centre pixel: dx = dy = 0 -> alpha = opacity exactly
    assert r["n_contrib"][1, 1] == 3
    o32 = float(np.float32(0.95))
    assert abs(r["sil"][1, 1] - (1 - (1 - o32) ** 3)) < 1e-12


def test_white_gaussians_colour_equals_silhouette():
    """With c_i = 1, Eq. 1 for colour equals Eq. 1 for silhouette, which the
    oracle computes separately as 1 - prod(1 - alpha_i)."""
    sc = scene_plain(0, n=4000)
    sc.rgb[:] = 1.0
    cam = look_camera((0.0, 0.0, 1.5), 0.0, 64, 64, 55.0)
    r = oracle.render(sc, cam, prec="f32")
    for c in range(3):
        np.testing.assert_allclose(r["rgb"][..., c], r["sil"], atol=2e-6)
    r64 = oracle.render(sc, cam, prec="f64")
    np.testing.assert_allclose(r64["rgb"][..., 0], r64["sil"], atol=1e-12)


def test_semantics_sum_and_per_class_channel():
    """Eq. 3: weights summing to 1 give sum_m P_m = S; and P_m equals Eq. 1
    with z_i = p_{i,m} rendered through the colour channel."""
    sc = scene_plain(0, n=4000, m=16, k=3)
    cam = look_camera((0.0, 0.0, 1.5), 0.0, 64, 64, 55.0)
    r = oracle.render(sc, cam, prec="f32")
    np.testing.assert_allclose(r["sem"].sum(-1), r["sil"], atol=5e-6)
    for classes in [(0, 5, 9), (15, 3, 7)]:
        dense = np.zeros((sc.n, 3), np.float32)
        for c, m_ in enumerate(classes):
            hit = sc.sem_ids == m_
            dense[:, c] = (sc.sem_w * hit).sum(1)
        sc2 = Scene(sc.means, sc.scales, sc.quats, sc.opacity, dense, sc.sem_ids, sc.sem_w, sc.m)
        r2 = oracle.render(sc2, cam, prec="f32", sem=False)
        for c, m_ in enumerate(classes):
            np.testing.assert_allclose(r2["rgb"][..., c], r["sem"][..., m_], atol=1e-6)


def test_isotropic_independent_of_rotation():
    rng = np.random.default_rng(2)
    sc = scene_plain(1, n=800)
    sc.scales[:] = sc.scales[:, :1]
    cam = look_camera((0.0, 0.0, 1.5), 0.0, 48, 48, 40.0)
    r0 = oracle.render(sc, cam, prec="f64")
    sc.quats[:] = rand_quat(rng, sc.n).astype(np.float32)
    r1 = oracle.render(sc, cam, prec="f64")
    np.testing.assert_allclose(r0["rgb"], r1["rgb"], atol=1e-9)
    np.testing.assert_allclose(r0["sem"], r1["sem"], atol=1e-9)


def test_pixel_list_equals_full_image():
    sc = scene_plain(0, n=3000)
    cam = look_camera((0.0, 0.0, 1.5), 0.0, 40, 30, 35.0)
    r = oracle.render(sc, cam, prec="f32")
    rng = np.random.default_rng(0)
    xs = rng.integers(0, 40, 50)
    ys = rng.integers(0, 30, 50)
    rp = oracle.render_pixels(sc, cam, xs, ys, prec="f32")
    for key in ("rgb", "sem", "sil", "depth", "T", "n_contrib", "flag"):
        np.testing.assert_array_equal(rp[key], r[key][ys, xs], err_msg=key)
    # a flagged pixel: alpha at the skip threshold on a 1 x 1 view
    w2c = np.zeros((3, 4), np.float32)
    w2c[:, :3] = np.eye(3, dtype=np.float32)
    cam1 = Camera(1, 1, 10.0, 10.0, 0.5, 0.5, 0.2, w2c)
    sc1 = mk_scene([[0.0, 0.0, 2.0]], [[0.2, 0.2, 0.2]], [[1.0, 0, 0, 0]], [(1 / 255) * (1 + 1e-7)])
    rp1 = oracle.render_pixels(sc1, cam1, np.array([0]), np.array([0]), prec="f32")
    assert rp1["flag"][0] & 1 and rp1["flag"][0] == oracle.render(sc1, cam1, prec="f32")["flag"][0, 0]


# --------------------------------------------------------------------------
# adjoint
# --------------------------------------------------------------------------

def _fd_scene(seed):
    rng = np.random.default_rng(seed)
    n, m, k = 5, 5, 2
    cam = look_camera((0.0, 0.0, 0.0), 0.0, 20, 18, 24.0, pitch_deg=5.0)
    cam.near = 0.2
    c2w = cam.w2c[:, :3].astype(np.float64).T
    z = rng.uniform(1.5, 3.0, n)
    tc = np.stack([rng.uniform(-0.25, 0.25, n) * z, rng.uniform(-0.25, 0.25, n) * z, z], 1)
    means = tc @ c2w.T + cam.position()
    scales = np.exp(rng.normal(-1.9, 0.3, (n, 3)))
    ids = np.stack([rng.choice(m, k, replace=False) for _ in range(n)]).astype(np.int32)
    sc = mk_scene(means, scales, rand_quat(rng, n) * 1.3, rng.uniform(0.3, 0.85, n),
                  rgb=rng.uniform(0, 1, (n, 3)), ids=ids, w=rng.uniform(0.1, 0.9, (n, k)), m=m)
    W, H = cam.width, cam.height
    up = dict(d_rgb=rng.normal(size=(H, W, 3)), d_depth=rng.normal(size=(H, W)), d_sil=rng.normal(size=(H, W)),
              d_sem=rng.normal(size=(H, W, m)))
    return sc, cam, up


def _loss(sc, cam, up, with_sem=True):
    r = oracle.render(sc, cam, prec="f64")
    L = (r["rgb"] * up["d_rgb"]).sum() + (r["depth"] * up["d_depth"]).sum() + (r["sil"] * up["d_sil"]).sum()
    if with_sem:
        L += (r["sem"] * up["d_sem"]).sum()
    return L, r["n_contrib"].copy(), r["flag"].copy()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_adjoint_matches_central_differences(seed):
    sc, cam, up = _fd_scene(seed)
    g = oracle.render_bwd(sc, cam, **up, sem_detach=False, prec="f64")
    fields = ["means", "scales", "quats", "opacity", "rgb", "sem_w"]
    skipped = 0
    total = 0
    for fld in fields:
        arr = getattr(sc, fld)
        flat = arr.reshape(-1)
        ga = g[fld].reshape(-1)
        scale = np.abs(ga).max() + 1e-12
        for j in range(flat.size):
            x0 = float(flat[j])
            # the scene is float32; perturb in double by editing a float64 copy
            h = 1e-6 * max(1.0, abs(x0))
            vals = []
            sigs = []
            for sgn in (1, -1):
                sc2 = Scene(*[np.array(getattr(sc, a), dtype=np.float64) for a in ["means", "scales", "quats",
                                                                                      "opacity", "rgb"]],
                            sc.sem_ids, np.array(sc.sem_w, np.float64), sc.m)
                getattr(sc2, fld).reshape(-1)[j] = x0 + sgn * h
                L, nc, fl = _loss(sc2, cam, up)
                vals.append(L)
                sigs.append(nc)
            total += 1
            if not np.array_equal(sigs[0], sigs[1]):
                skipped += 1
                continue
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - ga[j]) <= 1e-5 * abs(ga[j]) + 1e-6 * scale, (fld, j, fd, ga[j])
    assert skipped <= total // 20


def _fd_compare(sc, cam, up, fields, rel=1e-5, abs_frac=1e-6):
    """Central differences of the double-precision render against the
    oracle's adjoint, coordinate by coordinate; coordinates whose two
    perturbed renders differ in their contributor counts are skipped."""
    g = oracle.render_bwd(sc, cam, **up, sem_detach=False, prec="f64")
    skipped = total = 0
    for fld in fields:
        flat = getattr(sc, fld).reshape(-1)
        ga = g[fld].reshape(-1)
        scale = np.abs(ga).max() + 1e-12
        for j in range(flat.size):
            x0 = float(flat[j])
            h = 1e-6 * max(1.0, abs(x0))
            vals, sigs = [], []
            for sgn in (1, -1):
                sc2 = Scene(*[np.array(getattr(sc, a), dtype=np.float64) for a in ["means", "scales", "quats",
                                                                                      "opacity", "rgb"]],
                            sc.sem_ids, np.array(sc.sem_w, np.float64), sc.m)
                getattr(sc2, fld).reshape(-1)[j] = x0 + sgn * h
                L, nc, _ = _loss(sc2, cam, up)
                vals.append(L)
                sigs.append(nc)
            total += 1
            if not np.array_equal(sigs[0], sigs[1]):
                skipped += 1
                continue
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - ga[j]) <= rel * abs(ga[j]) + abs_frac * scale, (fld, j, fd, ga[j])
    return skipped, total


def test_adjoint_beyond_frustum_clamp_and_at_opacity_cap():
    """Gaussians whose means lie beyond the 1.3 tan(half-FOV) clamp on each
    side (their Jacobian is taken at the clamped point, so the chain to the
    mean differs) and one whose alpha is capped at 0.99 on its centre pixel
    (no gradient through alpha there): the adjoint still matches central
    differences."""
    rng = np.random.default_rng(11)
    cam = ident_cam(20, 18, 24.0)
    limx, limy = 1.3 * 10.0 / 24.0, 1.3 * 9.0 / 24.0
    z = np.array([2.0, 2.2, 2.4, 2.6, 1.9])  # distinct depths: no order flips under perturbation
    rx = np.array([1.2 * limx, -1.25 * limx, 0.1, -0.05, 0.0])
    ry = np.array([0.05, -0.1, 1.2 * limy, -1.25 * limy, 0.0])
    means = np.stack([rx * z, ry * z, z], 1)
    # the last Gaussian sits on the centre of pixel (10, 9): alpha capped there
    means[4, :2] = [(10.5 - 10.0) / 24.0 * 1.9, (9.5 - 9.0) / 24.0 * 1.9]
    scales = np.array([[0.3, 0.25, 0.2], [0.28, 0.3, 0.22], [0.26, 0.3, 0.2], [0.3, 0.24, 0.25], [0.15, 0.15, 0.15]])
    sc = mk_scene(means, scales, rand_quat(rng, 5), [0.8, 0.7, 0.75, 0.85, 0.9995], rgb=rng.uniform(0, 1, (5, 3)),
                  ids=np.stack([rng.choice(4, 2, replace=False) for _ in range(5)]).astype(np.int32),
                  w=rng.uniform(0.1, 0.9, (5, 2)), m=4)
    p = oracle.project(sc, cam, prec="f64")
    assert p["visible"].all()
    H, W = cam.height, cam.width
    up = dict(d_rgb=rng.normal(size=(H, W, 3)), d_depth=rng.normal(size=(H, W)), d_sil=rng.normal(size=(H, W)),
              d_sem=rng.normal(size=(H, W, 4)))
    r = oracle.render(sc, cam, prec="f64")
    assert r["sil"][9, 10] >= 0.99  # the capped pixel
    skipped, total = _fd_compare(sc, cam, up, ["means", "scales", "quats", "opacity"])
    assert skipped <= total // 20


def _deep_stack_scene(seed):
    """Tens of large, half-transparent Gaussians stacked along the optical
    axis: every pixel composites many layers, so the adjoint's transmittance
    recovery runs through long products and the 1e-4 stop rule cuts some
    pixels' lists."""
    rng = np.random.default_rng(seed)
    n, m, k = 40, 6, 3
    cam = look_camera((0.0, 0.0, 0.0), 0.0, 24, 20, 24.0)
    c2w = cam.w2c[:, :3].astype(np.float64).T
    z = rng.uniform(1.5, 4.0, n)
    tc = np.stack([rng.uniform(-0.15, 0.15, n) * z, rng.uniform(-0.15, 0.15, n) * z, z], 1)
    means = tc @ c2w.T + cam.position()
    scales = np.exp(rng.normal(-0.6, 0.2, (n, 3))) * z[:, None] / 3.0
    ids = np.stack([rng.choice(m, k, replace=False) for _ in range(n)]).astype(np.int32)
    sc = mk_scene(means, scales, rand_quat(rng, n), rng.uniform(0.2, 0.6, n), rgb=rng.uniform(0, 1, (n, 3)),
                  ids=ids, w=rng.uniform(0.1, 0.9, (n, k)), m=m)
    W, H = cam.width, cam.height
    up = dict(d_rgb=rng.normal(size=(H, W, 3)), d_depth=rng.normal(size=(H, W)), d_sil=rng.normal(size=(H, W)),
              d_sem=rng.normal(size=(H, W, m)))
    return sc, cam, up


@pytest.mark.parametrize("seed", [0, 1])
def test_adjoint_directional_derivatives_deep_stacks(seed):
    """v . grad L equals the central difference of L along v (double
    precision), for random directions v through all parameters at once, on
    scenes where each pixel composites many layers."""
    sc, cam, up = _deep_stack_scene(seed)
    r0 = oracle.render(sc, cam, prec="f64")
    assert np.median(r0["n_contrib"]) >= 20  # deep per-pixel lists
    assert (r0["T"] < 0.01).mean() > 0.3  # most light absorbed on many pixels
    assert r0["T"].min() < 2e-4  # the 1e-4 stop rule is reached
    g = oracle.render_bwd(sc, cam, **up, sem_detach=False, prec="f64")
    fields = ["means", "scales", "quats", "opacity", "rgb", "sem_w"]
    rng = np.random.default_rng(100 + seed)
    h = 1e-6
    checked = 0
    for _ in range(6):
        v = {f: rng.normal(size=getattr(sc, f).shape) for f in fields}
        v["scales"] *= sc.scales  # relative steps for the scales
        dirn = sum(float((g[f] * v[f]).sum()) for f in fields)
        mag = sum(float(np.abs(g[f] * v[f]).sum()) for f in fields)
        vals, sigs = [], []
        for sgn in (1, -1):
            arrs = {f: np.array(getattr(sc, f), np.float64) + sgn * h * v[f] for f in fields}
            sc2 = Scene(arrs["means"], arrs["scales"], arrs["quats"], arrs["opacity"], arrs["rgb"], sc.sem_ids,
                        arrs["sem_w"], sc.m)
            L, nc, fl = _loss(sc2, cam, up)
            vals.append(L)
            sigs.append(nc)
        if not np.array_equal(sigs[0], sigs[1]):
            continue  # a skip or stop decision flipped between the two sides
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - dirn) <= 1e-6 * abs(dirn) + 1e-8 * mag, (fd, dirn, mag)
        checked += 1
    assert checked >= 4


def test_semantic_gradient_block():
    """With the block on, geometric gradients do not depend on the semantic
    upstream gradient, and semantic-weight gradients do not change."""
    sc, cam, up = _fd_scene(4)
    g1 = oracle.render_bwd(sc, cam, **up, sem_detach=True, prec="f64")
    up0 = dict(up)
    up0["d_sem"] = np.zeros_like(up["d_sem"])
    g0 = oracle.render_bwd(sc, cam, **up0, sem_detach=True, prec="f64")
    for fld in ["means", "scales", "quats", "opacity", "rgb"]:
        np.testing.assert_array_equal(g1[fld], g0[fld])
    g2 = oracle.render_bwd(sc, cam, **up, sem_detach=False, prec="f64")
    np.testing.assert_array_equal(g1["sem_w"], g2["sem_w"])
    assert np.abs(g1["opacity"] - g2["opacity"]).max() > 0


# --------------------------------------------------------------------------
# candidate-view reductions (Eq. 6, Eq. 7 with Eq. 4)
# --------------------------------------------------------------------------

def test_candidate_empty_view():
    sc = scene_plain(0, n=500, m=16)
    sc.geo_unc = np.ones(sc.n, np.float32)
    cam = look_camera((0.0, 0.0, 1.5), 0.0, 30, 20, 25.0)
    cam.w2c[:, 3] += np.float32(100.0) * cam.w2c[:, 2]  # push everything behind the camera
    cam.w2c[2, 3] = np.float32(-100.0)
    su, sh, ns, nf = oracle.candidate(sc, cam)
    assert ns == 30 * 20
    assert su == 0.0
    assert abs(sh - 30 * 20 * math.log(16)) < 1e-9


def test_candidate_single_class_closed_form():
    """One Gaussian, one class with weight 1: P_0 = S, other classes 0, so
    after clipping to [0.001, 1] and renormalising the entropy per pixel has
    a closed form in S; u_i = 1 gives U = S."""
    cam = ident_cam(24, 20, 18.0)
    m = 10
    sc = mk_scene([[0.1, -0.05, 2.0]], [[0.4, 0.25, 0.3]], [[0.9, 0.1, 0.2, 0.3]], [0.9], ids=np.array([[3]]),
                  w=np.array([[1.0]]), m=m, unc=[1.0])
    su, sh, ns, nf = oracle.candidate(sc, cam, prec="f64")
    r = oracle.render(sc, cam, prec="f64")
    s = r["sil"].reshape(-1)
    p0 = np.clip(s, 0.001, 1.0)
    z = p0 + 0.001 * (m - 1)
    h = -(p0 / z) * np.log(p0 / z) - (m - 1) * (0.001 / z) * np.log(0.001 / z)
    assert abs(sh - h.sum()) < 1e-9 * h.sum()
    assert abs(su - s.sum()) < 1e-9
    assert ns == int((s == 0).sum()) and 0 < ns < s.size


def test_entropy_uniform_k_is_log_k():
    """Sec. 3.1: tau = log k is the entropy of a uniform distribution over k
    classes.  A pixel whose semantic map is uniform over k classes with mass
    well above the clip floor has entropy close to log k."""
    cam = ident_cam(1, 1, 10.0)
    for k in (2, 3, 8):
        m = k
        sc = mk_scene([[0.0, 0.0, 1.0]], [[1.0, 1.0, 1.0]], [[1, 0, 0, 0]], [0.99], ids=np.arange(k)[None, :],
                      w=np.full((1, k), 1.0 / k), m=m)
        su, sh, ns, nf = oracle.candidate(sc, cam, prec="f64")
        assert abs(sh - math.log(k)) < 1e-12


def test_golden_closed_forms():
    import json
    import os
    d = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))
    cam = ident_cam(1, 1, 10.0)
    for k, v in zip(d["entropy_uniform_k"]["k"], d["entropy_uniform_k"]["value"]):
        sc = mk_scene([[0.0, 0.0, 1.0]], [[1.0, 1.0, 1.0]], [[1, 0, 0, 0]], [0.99], ids=np.arange(k)[None, :],
                      w=np.full((1, k), 1.0 / k), m=k)
        assert abs(oracle.candidate(sc, cam, prec="f64")[1] - v) < 1e-12
    for m, v in zip(d["entropy_empty_pixel"]["m"], d["entropy_empty_pixel"]["value"]):
        sc = mk_scene([[0.0, 0.0, -1.0]], [[1.0, 1.0, 1.0]], [[1, 0, 0, 0]], [0.5], m=m)
        assert abs(oracle.candidate(sc, cam, prec="f64")[1] - v) < 1e-12
    # one capped Gaussian (alpha = 0.99) at the pixel centre: P = 0.99 w
    e = d["entropy_clip_then_normalise"]
    p = np.asarray(e["p"])
    nz = np.nonzero(p)[0]
    sc = mk_scene([[0.0, 0.0, 1.0]], [[1.0, 1.0, 1.0]], [[1, 0, 0, 0]], [0.99], ids=nz[None, :].astype(np.int32),
                  w=(p[nz] / 0.99)[None, :], m=p.size)
    assert abs(oracle.candidate(sc, cam, prec="f64")[1] - e["value"]) < 1e-6
    # the stop rule: stacked alpha = 0.95 Gaussians at the centre pixel
    st = d["stop_rule_alpha_0p95"]
    cam3 = ident_cam(3, 3, 10.0)
    sc = mk_scene([[0.0, 0.0, 1.0 + 0.1 * i] for i in range(5)], [[1.0, 1.0, 1.0]] * 5, [[1, 0, 0, 0]] * 5,
                  [0.95] * 5)
    r = oracle.render(sc, cam3, prec="f64")
    assert r["n_contrib"][1, 1] == st["n_contrib"]
    assert abs(r["sil"][1, 1] - st["silhouette_exact_alpha"]) < 1e-9  # 0.95 stored as float32


# ---------------------------------------------------------------------------
# mapping objective (Sec. 3.1): geometric L1 under the silhouette mask,
# entropy-masked Hellinger + cosine semantic term
# ---------------------------------------------------------------------------

def test_mapping_loss_semantic_closed_forms():
    from oracle import mapping_loss as ml
    k = 3
    # identical sharp distributions: Hellinger 0, cosine 1 -> term 0 and a
    # zero gradient
    q = np.array([0.9, 0.05, 0.05, 0.0])
    t, g = ml.semantic_terms(q[None], q[None], k)
    assert abs(t[0]) < 1e-12 and np.abs(g).max() < 1e-12
    # disjoint one-hots: Hellinger sqrt(0.5 * 2) = 1, cosine 0 -> 0.8 + 0.2
    t, _ = ml.semantic_terms(np.array([[1.0, 0, 0]]), np.array([[0, 1.0, 0]]), k)
    assert abs(t[0] - 1.0) < 1e-5
    # scaled prediction: cosine unchanged (1), Hellinger of (Q, c Q) = sqrt(0.5) |1 - sqrt(c)|
    c = 0.49
    t, _ = ml.semantic_terms(q[None], c * q[None], k)
    assert abs(t[0] - 0.8 * math.sqrt(0.5) * (1 - math.sqrt(c)) * math.sqrt((q).sum())) < 1e-5
    # entropy mask: uniform over k + 1 classes has H = ln(k + 1) > ln k -> masked
    # out (exactly uniform over k sits on the threshold: a rounding tie)
    qu = np.array([[0.25, 0.25, 0.25, 0.25]])
    t, g = ml.semantic_terms(qu, np.array([[0.0, 0.0, 0.0, 1.0]]), k)
    assert t[0] == 0.0 and not g.any()
    # just below ln k -> kept
    qs = np.array([[0.36, 0.33, 0.31, 0.0]])
    assert -(qs[qs > 0] * np.log(qs[qs > 0])).sum() < math.log(k)
    t, _ = ml.semantic_terms(qs, np.array([[0.0, 0.0, 0.0, 1.0]]), k)
    assert t[0] > 0.5
    # a negative rendered entry counts as 0 under the square roots (the
    # module's reading): P = (1, -0.5) against Q = (1, 0) is at Hellinger
    # distance 0, and the cosine sees the raw P: 1 / sqrt(1.25)
    t, _ = ml.semantic_terms(np.array([[1.0, 0.0]]), np.array([[1.0, -0.5]]), k)
    assert abs(t[0] - 0.2 * (1.0 - 1.0 / math.sqrt(1.25))) < 1e-9


def test_mapping_loss_semantic_degenerate_cases():
    """The module's readings at its degenerate points, in closed form:
    an uncovered pixel (P = 0) against a one-hot Q has cosine 0 and a zero
    cosine gradient, so its term is 0.8 D + 0.2 and its gradient the
    Hellinger one alone; distributions within 1e-12 in Hellinger distance
    have a zero Hellinger gradient."""
    from oracle import mapping_loss as ml
    k = 3
    eps = 1e-12
    q = np.array([[1.0, 0.0, 0.0]])
    t, g = ml.semantic_terms(q, np.zeros((1, 3)), k)
    sq0, s0 = math.sqrt(1.0 + eps), math.sqrt(eps)
    d = math.sqrt(0.5 * (sq0 - s0) ** 2)
    assert abs(t[0] - (0.8 * d + 0.2)) < 1e-12
    expect = np.array([[0.8 * (s0 - sq0) / (2.0 * s0) / (2.0 * d), 0.0, 0.0]])
    np.testing.assert_allclose(g, expect, rtol=1e-9, atol=0)
    # P within 1e-13 of Q: Hellinger distance below 1e-12, so only the
    # cosine part (of the order of the difference) is left in the gradient
    qh = np.array([[0.5, 0.5, 0.0]])
    ph = np.array([[0.5 + 1e-13, 0.5 - 1e-13, 0.0]])
    t, g = ml.semantic_terms(qh, ph, k)
    assert abs(t[0]) < 1e-12 and np.abs(g).max() < 1e-11


def test_mapping_loss_geometric_closed_form_and_mask():
    from oracle import mapping_loss as ml
    rgb = np.array([[[0.6, 0.3, 0.55]], [[0.2, 0.2, 0.2]]])
    t_rgb = np.array([[[0.5, 0.5, 0.5]], [[0.9, 0.9, 0.9]]])
    depth = np.array([[2.3], [1.0]])
    t_depth = np.array([[2.0], [5.0]])
    sil = np.array([[1.0], [0.99]])  # the second pixel sits on the threshold: excluded
    sem = np.zeros((2, 1, 2))
    t_sem = np.full((2, 1, 2), 0.5)  # uniform over k = 2: masked semantic term
    loss, d_rgb, d_depth, d_sem = ml.mapping_loss(rgb, depth, sil, sem, t_rgb, t_depth, t_sem, k=2)
    assert abs(loss - (0.3 + 0.5 * (0.1 + 0.2 + 0.05))) < 1e-12
    np.testing.assert_array_equal(d_depth, [[1.0], [0.0]])
    np.testing.assert_array_equal(d_rgb[0, 0], [0.5, -0.5, 0.5])
    assert not d_rgb[1].any() and not d_sem.any()


def test_mapping_loss_gradient_matches_central_differences():
    from oracle import mapping_loss as ml
    rng = np.random.default_rng(11)
    H, W, M, k = 3, 4, 7, 2
    t_sem = rng.dirichlet(np.full(M, 0.15), size=(H, W))   # mostly sharp: H < ln 2 for many pixels
    sem = rng.dirichlet(np.full(M, 1.0), size=(H, W)) * 0.9 + 0.01
    rgb, t_rgb = rng.uniform(size=(H, W, 3)), rng.uniform(size=(H, W, 3))
    depth, t_depth = rng.uniform(1, 3, size=(H, W)), rng.uniform(1, 3, size=(H, W))
    sil = rng.uniform(0.95, 1.0, size=(H, W))
    keep = np.abs(rgb - t_rgb).min() > 1e-3 and np.abs(depth - t_depth).min() > 1e-3
    assert keep
    f = lambda **kw: ml.mapping_loss(**{**dict(rgb=rgb, depth=depth, sil=sil, sem=sem, t_rgb=t_rgb,
                                                t_depth=t_depth, t_sem=t_sem, k=k), **kw})[0]
    _, d_rgb, d_depth, d_sem = ml.mapping_loss(rgb, depth, sil, sem, t_rgb, t_depth, t_sem, k)
    masked = sum(1 for y in range(H) for x in range(W)
                 if -(t_sem[y, x] * np.log(t_sem[y, x])).sum() < math.log(k))
    assert 0 < masked < H * W
    h = 1e-6
    for name, arr, grad in (("sem", sem, d_sem), ("depth", depth, d_depth), ("rgb", rgb, d_rgb)):
        num = np.zeros_like(arr)
        for idx in np.ndindex(arr.shape):
            a, b = arr.copy(), arr.copy()
            a[idx] += h
            b[idx] -= h
            num[idx] = (f(**{name: a}) - f(**{name: b})) / (2 * h)
        np.testing.assert_allclose(grad, num, rtol=1e-5, atol=1e-8, err_msg=name)


# ---------------------------------------------------------------------------
# candidate scoring and generation (Sec. 3.2, Eq. 6-8, "Exploration Strategy")
# ---------------------------------------------------------------------------

def test_scoring_closed_forms():
    from oracle import explore as ex
    # Eq. 6: the softmax of log N is the normalisation N / sum N (0 for N = 0)
    ns = np.array([0.0, 5.0, 15.0, 30.0])
    sums = np.stack([np.zeros(4), np.full(4, 7.0), ns], axis=1)
    pos = np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0], [-1.0, 0, 0]])  # all at distance 1
    sc, keep, best = ex.score(sums, np.full(4, 1000), pos, np.zeros(3))
    np.testing.assert_allclose(sc[:, 1], ns / ns.sum(), rtol=1e-15)
    # equal entropy sums and equal distances: uniform 1/V factors
    np.testing.assert_allclose(sc[:, 2], 0.25, rtol=1e-15)
    np.testing.assert_allclose(sc[:, 3], 0.75, rtol=1e-15)
    np.testing.assert_allclose(sc[:, 0], 0.75 * 0.25 * ns / ns.sum(), rtol=1e-14)
    # pruning: N_S < 0.5 % of 1000 pixels = 5 -> only the first is dropped
    assert keep.tolist() == [False, True, True, True] and best == 3
    # a hand-evaluated three-candidate case: N_S = (10, 30, 60), sum H =
    # (2, 3, 2), distances (0, 1, 2) from the current position
    sums = np.array([[0, 2.0, 10], [0, 3.0, 30], [0, 2.0, 60]])
    pos = np.array([[0.0, 0, 0], [0, 1.0, 0], [0, 0, 2.0]])
    sc, keep, best = ex.score(sums, np.full(3, 100), pos, np.zeros(3))
    e = math.e
    igeo = np.array([0.1, 0.3, 0.6])
    isem = np.array([1.0, e, 1.0]) / (2.0 + e)
    mov = 1.0 - np.array([1.0, e, e * e]) / (1.0 + e + e * e)
    np.testing.assert_allclose(sc[:, 0], mov * igeo * isem, rtol=1e-14)
    assert keep.all() and best == int(np.argmax(mov * igeo * isem)) == 1
    # no candidate reveals anything: the geometric factor is 0 for all
    sc, keep, best = ex.score(np.zeros((2, 3)), np.full(2, 10), np.zeros((2, 3)), np.zeros(3))
    assert not sc[:, 1].any() and not sc[:, 0].any() and best == -1


def test_fibonacci_lattice_properties():
    from oracle import explore as ex
    for n in (5, 15, 200):
        d = ex.fibonacci_directions(n)
        np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-15)
        # heights equally spaced in (-1, 1), symmetric about 0
        np.testing.assert_allclose(np.diff(d[:, 2]), -2.0 / n, atol=1e-15)
        assert abs(d[:, 2].sum()) < 1e-12
        # azimuth steps of the golden angle (mod 2 pi)
        az = np.arctan2(d[:, 1], d[:, 0])
        step = np.mod(np.diff(az), 2 * math.pi)
        np.testing.assert_allclose(step, math.pi * (3 - math.sqrt(5)), atol=1e-12)
    # near-uniform coverage (area per point 4 pi / n): every direction of a
    # dense random sample lies within 2.9 / sqrt(n) rad of a lattice point
    # (the lattice reaches 2.61; an azimuth step of 2 rad instead of the
    # golden angle leaves holes of 3.36), and no two points are closer than
    # 2.8 / sqrt(n) (the lattice: 3.10)
    n = 200
    d = ex.fibonacci_directions(n)
    rng = np.random.default_rng(0)
    u = rng.normal(size=(20000, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    cover = np.arccos(np.clip((u @ d.T).max(1), -1, 1)).max()
    assert cover < 2.9 / math.sqrt(n)
    g = np.clip(d @ d.T, -1, 1) - 2 * np.eye(n)
    assert np.arccos(g.max()) > 2.8 / math.sqrt(n)


def test_look_along_pose():
    from oracle import explore as ex
    rng = np.random.default_rng(1)
    for d in ex.fibonacci_directions(15):
        p = rng.uniform(-3, 3, size=3)
        w = ex.look_along(p, d)
        r, t = w[:, :3], w[:, 3]
        np.testing.assert_allclose(r @ r.T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(r) - 1.0) < 1e-12
        np.testing.assert_allclose(r @ p + t, 0.0, atol=1e-12)            # the centre maps to the origin
        np.testing.assert_allclose(r @ (p + d) + t, [0, 0, 1], atol=1e-12)  # one metre ahead on the axis
        assert (r[1] @ np.array([0, 0, 1.0])) <= 1e-12                      # image "down" never points up
    # a horizontal direction reproduces the scenes' horizontal look-at camera
    from paper_2506_00225_gb300 import scenes
    cam = scenes.look_camera((1.0, 2.0, 1.5), 30.0, 64, 48, 50.0)
    d = np.array([math.cos(math.radians(30)), math.sin(math.radians(30)), 0.0])
    np.testing.assert_allclose(ex.look_along((1.0, 2.0, 1.5), d), cam.w2c, atol=1e-6)
    # straight up and straight down (d parallel to z): still a proper pose,
    # right = d x y normalised (the module's reading), forward = d
    for dz in (1.0, -1.0):
        d = np.array([0.0, 0.0, dz])
        w = ex.look_along((0.5, -0.5, 1.0), d)
        r = w[:, :3]
        assert np.isfinite(w).all()
        np.testing.assert_allclose(r @ r.T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(r) - 1.0) < 1e-12
        np.testing.assert_allclose(r[2], d, atol=1e-15)
        np.testing.assert_allclose(r[0], np.cross(d, [0.0, 1.0, 0.0]), atol=1e-15)


def test_candidate_positions_closed_form():
    from oracle import explore as ex
    centres = np.array([[0.1, 0.2, 1.50], [0.4, -0.3, 1.45], [0.6, 0.0, 1.5], [2.9, 1.1, 0.8], [3.1, 0.9, 1.52]])
    p = ex.candidate_positions(centres, 1.0, [1.5], 0.1)
    # rounding to the 1 m lattice: (0, 0), (0, 0), (1, 0), -, (3, 1)
    np.testing.assert_allclose(p, [[0, 0, 1.5], [1, 0, 1.5], [3, 1, 1.5]], atol=1e-7)
    p2 = ex.candidate_positions(centres, 0.5, [0.8, 1.5], 0.1)
    assert len(p2) == 5 and set(np.round(p2[:, 2], 5)) == {0.8, 1.5}
    # a centre within the band of two heights gives a position at each
    p3 = ex.candidate_positions(np.array([[0.1, 0.1, 1.1]]), 1.0, [1.0, 1.2], 0.15)
    np.testing.assert_allclose(p3, [[0, 0, 1.0], [0, 0, 1.2]], atol=1e-7)


# ---------------------------------------------------------------------------
# sparse top-k initialisation / update (Sec. 3.1) and the Exploration Map
# (Sec. 3.2)
# ---------------------------------------------------------------------------

def test_topk_hand_examples():
    from oracle import sparse as sp
    probs = np.array([[0.1, 0.5, 0.2, 0.2, 0.0],      # tie 0.2 / 0.2: lower id first
                      [np.nan, 0.3, 0.3, 0.3, 0.1],   # NaN last; three-way tie by id
                      [0.0, 0.0, 0.0, 0.0, 1.0]], np.float32)
    ids, w = sp.topk_init(probs, 3)
    assert ids.tolist() == [[1, 2, 3], [1, 2, 3], [4, 0, 1]]
    np.testing.assert_array_equal(w, np.float32([[0.5, 0.2, 0.2], [0.3, 0.3, 0.3], [1.0, 0.0, 0.0]]))
    # NaN ranks below every number, zero included
    ids, _ = sp.topk_init(np.array([[np.nan, 0.0, 0.2]], np.float32), 3)
    assert ids.tolist() == [[2, 1, 0]]
    # rows select observations; k = m returns a full descending order
    ids, w = sp.topk_init(probs, 5, rows=[2, 0])
    assert ids.tolist() == [[4, 0, 1, 2, 3], [1, 2, 3, 0, 4]]
    # gather with fixed ids; an invalid id keeps its value
    g = sp.topk_gather(probs, np.array([[4, 0, -1]], np.int32), np.array([[9.0, 9.0, 9.0]], np.float32), rows=[0])
    np.testing.assert_array_equal(g, np.float32([[0.0, 0.1, 9.0]]))
    # Gaussian i reads its own observation row rows[i], not row i
    g = sp.topk_gather(probs, np.array([[4, 0, 1], [3, 4, 7]], np.int32), np.full((2, 3), 9.0, np.float32),
                       rows=[2, 1])
    np.testing.assert_array_equal(g, np.float32([[1.0, 0.0, 0.0], [0.3, 0.1, 9.0]]))


def test_topk_matches_python_selection():
    from oracle import sparse as sp
    rng = np.random.default_rng(0)
    probs = rng.integers(0, 6, size=(50, 13)).astype(np.float32) / 5.0  # many ties
    ids, w = sp.topk_init(probs, 4)
    for i in range(50):
        ref = sorted(range(13), key=lambda c: (-float(probs[i, c]), c))[:4]
        assert ids[i].tolist() == ref
        assert w[i].tolist() == [float(probs[i, c]) for c in ref]


def _axis_cam(pos, yaw, w, h, f):
    from paper_2506_00225_gb300 import scenes
    return scenes.look_camera(pos, yaw, w, h, f)


def test_voxel_axis_aligned_ray_closed_form():
    """A 1x1 camera at the centre of voxel (0, 2, 2) looking along +x with
    depth 5 voxels: voxels x = 0..4 free, x = 5 occupied (its centre holds the
    point); cut at max_depth 3.2 voxels: x = 0..3 free, nothing occupied."""
    from oracle import voxel as vx
    vs = 0.25
    cam = _axis_cam(((0.5) * vs, 2.5 * vs, 2.5 * vs), 0.0, 1, 1, 10.0)
    depth = np.array([[5.0 * vs]], np.float32)
    sure, maybe = vx.integrate((0, 0, 0), vs, (8, 5, 5), depth, cam)
    st = vx.state_of(sure)
    assert [int(st[2, 2, x]) for x in range(8)] == [1, 1, 1, 1, 1, 2, 0, 0]
    assert st.sum() == 5 * 1 + 2 and (maybe == sure).all()
    sure, _ = vx.integrate((0, 0, 0), vs, (8, 5, 5), depth, cam, max_depth=3.2 * vs)
    assert [int(vx.state_of(sure)[2, 2, x]) for x in range(8)] == [1, 1, 1, 1, 0, 0, 0, 0]
    # invalid depths mark nothing
    for bad in (0.0, -1.0, np.nan, np.inf):
        s_, m_ = vx.integrate((0, 0, 0), vs, (8, 5, 5), np.array([[bad]], np.float32), cam)
        assert not s_.any() and not m_.any()


def test_voxel_ray_on_a_face_is_undecided():
    """The same ray moved onto the face between voxel rows y = 1 and y = 2
    (y = 2.0 voxels, exact in float): it touches both rows' cubes on their
    shared face only, so those voxels are near ties, in `maybe` but not in
    `sure`; the rows beside them are untouched."""
    from oracle import voxel as vx
    vs = 0.25
    cam = _axis_cam((0.5 * vs, 2.0 * vs, 2.5 * vs), 0.0, 1, 1, 10.0)
    depth = np.array([[5.0 * vs]], np.float32)
    sure, maybe = vx.integrate((0, 0, 0), vs, (8, 5, 5), depth, cam)
    for x in range(4):  # away from the end point's cells (x = 4..6)
        for y in (1, 2):
            assert sure[2, y, x] & 1 == 0 and maybe[2, y, x] & 1 == 1, (x, y)
    assert not sure[:, (0, 3, 4), :].any() and not maybe[:, (0, 3, 4), :].any()


def test_voxel_ray_entering_from_outside_and_sampling():
    """A camera outside the grid: only the voxels inside count.  The decided
    voxels agree with a dense sampling of the segment (a voxel sampled by the
    segment is met; a voxel met by the segment beyond a margin is sampled)."""
    from oracle import voxel as vx
    vs = 0.2
    cam = _axis_cam((-1.0, 0.53, 0.61), 17.0, 9, 7, 6.0)
    rng = np.random.default_rng(3)
    depth = rng.uniform(1.0, 4.0, size=(7, 9)).astype(np.float32)
    sure, maybe = vx.integrate((0, 0, 0), vs, (12, 9, 6), depth, cam)
    assert (sure & ~maybe).sum() == 0
    # dense sampling of every segment (points strictly inside, away from p)
    sampled = np.zeros_like(sure)
    n = np.array([12, 9, 6])
    for o, p, hit in vx.ray_points(depth, cam, 1, 10.0):
        a, b = o / vs, p / vs
        t = np.linspace(0.0, 1.0, 20001)[:-1]
        pts = a[None] + t[:, None] * (b - a)[None]
        c = np.floor(pts).astype(np.int64)
        ok = np.all((c >= 0) & (c < n), axis=1)
        end = np.floor(b).astype(np.int64)
        c = c[ok & ~np.all(c == end, axis=1)]
        sampled[c[:, 2], c[:, 1], c[:, 0]] |= 1
    free_sure = (sure & 1).astype(bool)
    assert free_sure.any()
    assert (sampled.astype(bool) <= (maybe & 1).astype(bool)).all()  # every sampled voxel may be free
    assert ((sure & 1).astype(bool) <= sampled.astype(bool) | (maybe & 2).astype(bool)).all()


def test_scoring_tie_and_band_boundary():
    """Equal scores among kept candidates pick the lowest index; a voxel
    centre exactly one band away from a height yields a candidate position,
    one just beyond does not."""
    from oracle import explore as ex
    sums = np.array([[0, 1.0, 50], [0, 1.0, 50], [0, 1.0, 10]])
    pos = np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]])
    sc, keep, best = ex.score(sums, np.full(3, 100), pos, np.zeros(3))
    assert sc[0, 0] == sc[1, 0] > sc[2, 0] and keep.all() and best == 0
    centres = np.array([[0.0, 0.0, 1.75], [2.0, 0.0, 1.7501]])
    p = ex.candidate_positions(centres, 1.0, [1.5], 0.25)
    np.testing.assert_allclose(p, [[0.0, 0.0, 1.5]])


def test_voxel_off_centre_pixel_depth_limit_and_states():
    """Pixel centres (u + 0.5, v + 0.5) set the ray: in a 2x1 image (f = 2)
    the left pixel's ray leans 0.25 m per metre to its side, so a depth of
    1 m ends in voxel (4, 3, 2); a depth equal to max_depth still marks its
    voxel occupied; occupied wins over free; newly freed voxels are free now
    and unknown before (not occupied before)."""
    from oracle import voxel as vx
    vs = 0.25
    cam = _axis_cam((0.5 * vs, 2.5 * vs, 2.5 * vs), 0.0, 2, 1, 2.0)
    depth = np.array([[1.0, 0.0]], np.float32)  # the right pixel is invalid
    sure, maybe = vx.integrate((0, 0, 0), vs, (8, 6, 5), depth, cam)
    st = vx.state_of(sure)
    assert st[2, 3, 4] == 2 and (st == 2).sum() == 1 and (maybe == sure).all()
    ax = _axis_cam((0.5 * vs, 2.5 * vs, 2.5 * vs), 0.0, 1, 1, 10.0)
    d5 = np.array([[5.0 * vs]], np.float32)
    sure, _ = vx.integrate((0, 0, 0), vs, (8, 5, 5), d5, ax, max_depth=5.0 * vs)
    assert vx.state_of(sure)[2, 2, 5] == 2
    assert vx.state_of(np.array([0, 1, 2, 3], np.uint8)).tolist() == [0, 1, 2, 2]
    prev = np.array([[[2, 0, 1, 3]]], np.uint8)
    cur = np.array([[[1, 1, 1, 1]]], np.uint8)
    np.testing.assert_allclose(vx.new_free(prev, cur, (0.0, 0.0, 0.0), vs), [[1.5 * vs, 0.5 * vs, 0.5 * vs]])


def test_evaluation_count_per_pixel():
    """N_eval of the per-pixel definition (the work count of the forward
    blend's roofline): a pixel whose final transmittance is at least 0.01
    cannot have stopped (alpha <= 0.99 keeps T (1 - alpha) >= 1e-4), so it
    tested every visible Gaussian whose pixel rectangle holds it -- a count
    that the rectangles alone fix.  The stopped pixels tested a prefix of
    that set, including the stopping pair; the per-pixel counts add up to
    the oracle's total, and in the stack of the stop-rule example exactly
    the 3 contributors and the stopping 4th Gaussian are tested."""
    sc = scene_plain(5, n=10000, m=8, k=2)
    cam = look_camera((0.0, 0.0, 1.5), 15.0, 61, 47, 40.0)
    r = oracle.render(sc, cam, prec="f32")
    p = oracle.project(sc, cam, prec="f32")
    vis = np.nonzero(p["visible"])[0]
    x0, x1, y0, y1 = (p["rect"][vis, i][:, None, None] for i in range(4))
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    cover = ((xs[None] >= x0) & (xs[None] <= x1) & (ys[None] >= y0) & (ys[None] <= y1)).sum(axis=0)
    open_px = r["T"] >= 0.01
    assert open_px.sum() > 100 and (~open_px).sum() > 100
    np.testing.assert_array_equal(r["n_eval_px"][open_px], cover[open_px])
    assert (r["n_eval_px"][~open_px] <= cover[~open_px]).all()
    assert (r["n_eval_px"] >= r["n_contrib"]).all()
    assert int(r["n_eval_px"].sum()) == r["n_eval"]
    # stop-rule stack: 3 contributors + the stopping Gaussian at the centre
    cam3 = ident_cam(3, 3, 10.0)
    means = [[0.0, 0.0, 1.0 + 0.1 * i] for i in range(6)]
    st = mk_scene(means, [[1.0, 1.0, 1.0]] * 6, [[1, 0, 0, 0]] * 6, [0.95] * 6)
    r3 = oracle.render(st, cam3, prec="f64")
    assert r3["n_contrib"][1, 1] == 3 and r3["n_eval_px"][1, 1] == 4
