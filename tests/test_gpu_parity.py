"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances (spec bar): tile lists and sort order bit-exact; projected
records bit-exact; rendered images and semantic maps within 1e-5 max abs
(pixels where the oracle saw a threshold decision within a relative 1e-5 of
its threshold are excluded and counted -- the two sides may round exp()
differently by an ulp or two); gradients within 1e-3 relative of the oracle's
float32 adjoint (floored at 1e-4 of the tensor's largest entry, see
gradtol); per-view candidate sums
within 1e-5 relative, N_S within the number of flagged pixels.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_00225_gb300 import raster, scenes
from gradtol import FLOOR, WIDE, grad_close

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_00225_gb300 import build
    build.build()


def small_case(n=6000, w=80, h=60, seed=0, m=16, k=3):
    sc = scenes.scene_plain(seed, n=n, m=m, k=k)
    cam = scenes.look_camera((0.0, 0.0, 1.5), 10.0, w, h, 60.0, pitch_deg=-5.0)
    return sc, cam


# ---------------------------------------------------------------------------
# projection + binning: bit-exact
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 8)])
def test_projection_records_bitexact(tile):
    sc, cam = small_case(w=123, h=77)
    g = raster.Gaussians.from_scene(sc)
    rast = raster.Rasterizer(tile=tile)
    rast._project_bin(g, [cam], check=True)
    wv = rast.workspace_views()
    p = oracle.project(sc, cam, tile=tile, prec="f32")
    vis = np.nonzero(p["visible"])[0]
    assert wv["n_records"] == vis.size
    gid = wv["gid"].cpu().numpy()
    np.testing.assert_array_equal(gid, vis)  # compacted in gid order
    np.testing.assert_array_equal(wv["uv"].cpu().numpy().view(np.uint32), p["uv"][vis].view(np.uint32))
    np.testing.assert_array_equal(wv["conic"][:, :3].cpu().numpy().view(np.uint32), p["conic"][vis].view(np.uint32))
    np.testing.assert_array_equal(wv["depth"].cpu().numpy().view(np.uint32), p["depth"][vis].view(np.uint32))
    np.testing.assert_array_equal(wv["rect"].cpu().numpy().astype(np.int32), p["rect"][vis])


def _skewed_case(w=123, h=77, seed=0):
    """small_case seen through unequal focal lengths and an off-centre
    principal point (the other cases use fx = fy and the image centre)."""
    sc, cam = small_case(w=w, h=h, seed=seed)
    cam = scenes.Camera(cam.width, cam.height, 1.25 * cam.fx, 0.8 * cam.fy, 0.43 * w, 0.58 * h, cam.near,
                        cam.w2c.copy())
    return sc, cam


def test_unequal_focal_lengths_and_offset_principal_point():
    """Records bit-exact, tile lists bit-exact, forward images within 1e-5
    and gradients within 1e-3 of the oracle on a camera with fx != fy and
    cx, cy away from the image centre (a swapped focal length or principal
    point coordinate anywhere on the path fails here)."""
    sc, cam = _skewed_case()
    g = raster.Gaussians.from_scene(sc)
    rast = raster.Rasterizer()
    rast._project_bin(g, [cam], check=True)
    wv = rast.workspace_views()
    p = oracle.project(sc, cam, prec="f32")
    vis = np.nonzero(p["visible"])[0]
    np.testing.assert_array_equal(wv["gid"].cpu().numpy(), vis)
    np.testing.assert_array_equal(wv["uv"].cpu().numpy().view(np.uint32), p["uv"][vis].view(np.uint32))
    np.testing.assert_array_equal(wv["conic"][:, :3].cpu().numpy().view(np.uint32), p["conic"][vis].view(np.uint32))
    np.testing.assert_array_equal(wv["rect"].cpu().numpy().astype(np.int32), p["rect"][vis])
    _check_lists(wv, [p], [cam], (16, 16))
    rgb, depth, sil, sem = _fwd(sc, cam)
    r = oracle.render(sc, cam, prec="f32")
    ok = r["flag"] & 1 == 0
    assert (~ok).sum() <= max(2, ok.size // 1000)
    for x, name in ((rgb, "rgb"), (depth, "depth"), (sil, "sil"), (sem, "sem")):
        _img_close(x, r[name], ok)
    rng = np.random.default_rng(3)
    H, W = cam.height, cam.width
    up = dict(d_rgb=rng.normal(size=(H, W, 3)).astype(np.float32), d_depth=rng.normal(size=(H, W)).astype(np.float32),
              d_sil=rng.normal(size=(H, W)).astype(np.float32), d_sem=rng.normal(size=(H, W, sc.m)).astype(np.float32))
    _mask_flagged(up, r["flag"])
    rast.forward(g, cam)
    t = {key: torch.from_numpy(v).cuda() for key, v in up.items()}
    grads = rast.backward(g, cam, t["d_rgb"], t["d_depth"], t["d_sil"], t["d_sem"])
    ref = oracle.render_bwd(sc, cam, **up, prec="f32")
    for name in ["means", "scales", "quats", "opacity", "rgb", "sem_w"]:
        _grad_close(grads[name].cpu().numpy(), ref[name], name=name)


def _check_lists(wv, projs, cams, tile):
    ranges, gids, offs = oracle.tile_lists(projs, cams, tile)
    assert wv["n_pairs"] == gids.size
    np.testing.assert_array_equal(wv["tile_offset"].cpu().numpy(), offs)
    np.testing.assert_array_equal(wv["ranges"].cpu().numpy(), ranges)
    rec = wv["pair_rec"].cpu().numpy()
    rec_gid = wv["gid"].cpu().numpy()
    np.testing.assert_array_equal(rec_gid[rec], gids)
    tiles = np.repeat(np.arange(ranges.shape[0]), ranges[:, 1] - ranges[:, 0])
    np.testing.assert_array_equal(wv["pair_tile"].cpu().numpy(), tiles)


@pytest.mark.parametrize("tile", [(16, 16), (16, 8)])
def test_binning_bitexact_single_view(tile):
    sc, cam = small_case(w=150, h=90)
    rast = raster.Rasterizer(tile=tile)
    rast._project_bin(raster.Gaussians.from_scene(sc), [cam], check=True)
    _check_lists(rast.workspace_views(), [oracle.project(sc, cam, tile=tile)], [cam], tile)


def test_binning_bitexact_multi_view_equal_depths():
    """Mixed resolutions in one sort; many exactly equal depths to exercise
    the gid tie-break."""
    sc, _ = small_case(n=4000)
    sc.means[:, 0] = np.round(sc.means[:, 0] * 4) / 4  # quantised x -> equal depths for yaw-0 views
    cams = [scenes.look_camera((0.0, 0.0, 1.5), 0.0, 64, 48, 50.0),
            scenes.look_camera((0.1, 0.0, 1.4), 0.0, 130, 70, 90.0),
            scenes.look_camera((0.0, 0.2, 1.5), 35.0, 33, 17, 20.0)]
    rast = raster.Rasterizer()
    rast._project_bin(raster.Gaussians.from_scene(sc), cams, check=True)
    wv = rast.workspace_views()
    projs = [oracle.project(sc, c) for c in cams]
    assert wv["n_records"] == sum(int(p["visible"].sum()) for p in projs)
    _check_lists(wv, projs, cams, (16, 16))


def test_non_finite_gaussians_culled_like_the_oracle():
    """NaN / Inf means and scales, zero and NaN quaternions: such Gaussians
    get no record (as in the oracle), the rest render as usual, outputs stay
    finite and the adjoint leaves their gradients at zero."""
    sc, cam = small_case(n=3000, w=80, h=60)
    rng = np.random.default_rng(3)
    bad = rng.choice(sc.n, 120, replace=False)
    sc.means[bad[:30], 0] = np.nan
    sc.scales[bad[30:60], 1] = np.inf
    sc.quats[bad[60:90], :] = 0.0
    sc.quats[bad[90:], 2] = np.nan
    g = raster.Gaussians.from_scene(sc)
    rast = raster.Rasterizer()
    rast._project_bin(g, [cam], check=True)
    wv = rast.workspace_views()
    p = oracle.project(sc, cam, prec="f32")
    np.testing.assert_array_equal(wv["gid"].cpu().numpy(), np.nonzero(p["visible"])[0])
    assert not np.isin(bad, wv["gid"].cpu().numpy()).any()
    rgb, depth, sil, sem = _fwd(sc, cam)
    r = oracle.render(sc, cam, prec="f32")
    ok = r["flag"] & 1 == 0
    for x, name in ((rgb, "rgb"), (depth, "depth"), (sil, "sil"), (sem, "sem")):
        assert np.isfinite(x).all(), name
        _img_close(x, r[name], ok)
    up = torch.ones(cam.height, cam.width, 3, device="cuda")
    rast.forward(g, cam)
    grads = rast.backward(g, cam, up, None, None, None)
    for name in ("means", "scales", "quats", "opacity", "rgb"):
        v = grads[name].cpu().numpy()
        assert np.isfinite(v).all(), name
        assert (v[bad] == 0).all(), name


# ---------------------------------------------------------------------------
# forward render
# ---------------------------------------------------------------------------

def _fwd(sc, cam, tile=(16, 16), ppt=0):
    g = raster.Gaussians.from_scene(sc)
    rast = raster.Rasterizer(tile=tile, px_per_thread=ppt)
    with torch.no_grad():
        out = rast.forward(g, cam)
    return [t.cpu().numpy() if t is not None else None for t in out]


def _img_close(a, b, ok, tol=IMG_TOL):
    err = np.abs(a - b)
    if err.ndim > ok.ndim:
        err = err.reshape(ok.shape + (-1,)).max(-1)
    assert err[ok].max(initial=0.0) <= tol, err[ok].max()


@pytest.mark.parametrize("w,h", [(128, 128), (123, 77), (16, 16), (17, 1)])
def test_forward_parity(w, h):
    sc, cam = small_case(w=w, h=h)
    rgb, depth, sil, sem = _fwd(sc, cam)
    r = oracle.render(sc, cam, prec="f32")
    ok = r["flag"] & 1 == 0
    assert (~ok).sum() <= max(2, ok.size // 1000)
    _img_close(rgb, r["rgb"], ok)
    _img_close(depth, r["depth"], ok)
    _img_close(sil, r["sil"], ok)
    _img_close(sem, r["sem"], ok)


def test_forward_plain10k_workload():
    w = scenes.workload("plain10k")
    sc, cam = w["scene"], w["cams"][0]
    rgb, depth, sil, sem = _fwd(sc, cam)
    r = oracle.render(sc, cam, prec="f32")
    ok = r["flag"] & 1 == 0
    _img_close(rgb, r["rgb"], ok)
    _img_close(depth, r["depth"], ok)
    _img_close(sil, r["sil"], ok)
    _img_close(sem, r["sem"], ok)


def test_forward_independent_of_tile_shape_and_mapping():
    sc, cam = small_case(w=100, h=70)
    base = _fwd(sc, cam, (16, 16), 1)
    for tile in [(16, 16), (16, 8), (8, 8), (32, 8)]:
        for ppt in (1, 2):
            other = _fwd(sc, cam, tile, ppt)
            for a, b in zip(base, other):
                np.testing.assert_array_equal(a, b)


def test_backward_independent_of_mapping():
    """Pixels per thread changes only the order of the float atomics."""
    sc, cam = small_case(n=2500, w=45, h=37, seed=2)
    g = raster.Gaussians.from_scene(sc)
    H, W = cam.height, cam.width
    torch.manual_seed(0)
    ups = [torch.randn(H, W, 3, device="cuda"), torch.randn(H, W, device="cuda"), torch.randn(H, W, device="cuda"),
           torch.randn(H, W, sc.m, device="cuda")]
    res = []
    for tile, ppt in [((16, 16), 1), ((16, 16), 2), ((16, 16), 4), ((32, 8), 2)]:
        rast = raster.Rasterizer(tile=tile, px_per_thread=ppt, sem_detach_geometry=False)
        rast.forward(g, cam)
        res.append({k: v.cpu().numpy() for k, v in rast.backward(g, cam, *ups).items()})
    for other in res[1:]:
        for name in res[0]:
            _grad_close(other[name], res[0][name], rtol=1e-4, name=name, floor=WIDE)


def test_autotune_picks_a_compiled_config():
    from paper_2506_00225_gb300 import autotune
    sc, cam, t, _ = _l1_case(seed=7)
    g = raster.Gaussians.from_scene(sc)
    tt = [torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda() for x in (t["rgb"], t["depth"], t["sem"])]
    best, table = autotune.tune_mapping(g, cam, *tt, reps=2)
    valid = [(t, p) for t in autotune.SHAPES for p in autotune.PPTS if autotune._valid(t, p)]
    assert len(table) == len(valid)
    assert best["ms"] == min(r["ms"] for r in table) and best["px_per_thread"] in (1, 2, 4)


def test_forward_class_chunking_large_m():
    """M = 300 does not fit one shared-memory chunk at 16x16: chunked passes
    must give the same map."""
    sc, cam = small_case(n=3000, w=64, h=40, m=300, k=8)
    rgb, depth, sil, sem = _fwd(sc, cam)
    r = oracle.render(sc, cam, prec="f32")
    ok = r["flag"] & 1 == 0
    _img_close(sem, r["sem"], ok)
    _img_close(rgb, r["rgb"], ok)


def test_forward_empty_and_culled():
    sc, cam = small_case(n=50, w=40, h=30)
    sc.means[:, 0] = -5.0  # all behind the camera
    rgb, depth, sil, sem = _fwd(sc, cam)
    assert not rgb.any() and not depth.any() and not sil.any() and not sem.any()
    empty = sc.subset(np.zeros(0, dtype=np.int64))
    rgb, depth, sil, sem = _fwd(empty, cam)
    assert rgb.shape == (30, 40, 3) and not sil.any()


def test_forward_deterministic():
    sc, cam = small_case()
    a = _fwd(sc, cam)
    b = _fwd(sc, cam)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


# ---------------------------------------------------------------------------
# backward
# ---------------------------------------------------------------------------

def _grad_close(a, b, rtol=1e-3, name="", floor=FLOOR):
    """|a - b| <= rtol * (|b| + floor * max|b|) (gradtol.grad_close)."""
    grad_close(a, b, rtol, name, floor)


def _mask_flagged(up, flag):
    """Zero the upstream gradient at pixels whose skip / stop / cap decision
    lies within a relative 1e-5 of its threshold: there the two sides may
    decide differently (exp rounding), and a zero upstream keeps such a pixel
    out of every gradient."""
    bad = flag != 0
    for key, v in up.items():
        v[bad] = 0.0
    return int(bad.sum())


def _bwd_case(sem_detach, seed=0, w=48, h=40, m=16, k=3, ppt=0, recompute=False):
    sc, cam = small_case(n=2500, w=w, h=h, seed=seed, m=m, k=k)
    rng = np.random.default_rng(seed + 10)
    H, W, m = cam.height, cam.width, sc.m
    up = dict(d_rgb=rng.normal(size=(H, W, 3)).astype(np.float32), d_depth=rng.normal(size=(H, W)).astype(np.float32),
              d_sil=rng.normal(size=(H, W)).astype(np.float32), d_sem=rng.normal(size=(H, W, m)).astype(np.float32))
    nbad = _mask_flagged(up, oracle.render(sc, cam, prec="f32")["flag"])
    assert nbad <= max(2, H * W // 1000)
    g = raster.Gaussians.from_scene(sc)
    rast = raster.Rasterizer(sem_detach_geometry=sem_detach, px_per_thread=ppt, recompute_bwd=recompute)
    rast.forward(g, cam)
    t = {key: torch.from_numpy(v).cuda() for key, v in up.items()}
    grads = rast.backward(g, cam, t["d_rgb"], t["d_depth"], t["d_sil"], t["d_sem"])
    ref = oracle.render_bwd(sc, cam, **up, sem_detach=sem_detach, prec="f32")
    return {k: v.cpu().numpy() for k, v in grads.items()}, ref, sc, cam


@pytest.mark.parametrize("sem_detach", [True, False])
def test_backward_parity(sem_detach):
    grads, ref, sc, cam = _bwd_case(sem_detach)
    for name in ["means", "scales", "quats", "opacity", "rgb", "sem_w"]:
        _grad_close(grads[name], ref[name], name=name)


def test_backward_parity_ragged_edges():
    """Width and height not multiples of the tile: warps straddle the image
    edge (lanes outside the image still take part in the reductions)."""
    for sem_detach in (True, False):
        grads, ref, sc, cam = _bwd_case(sem_detach, seed=1, w=45, h=37)
        for name in ["means", "scales", "quats", "opacity", "rgb", "sem_w"]:
            _grad_close(grads[name], ref[name], name=name)


@pytest.mark.parametrize("ppt,m,k", [(1, 16, 3), (2, 16, 3), (4, 40, 8)])
def test_recompute_mode_ragged(ppt, m, k):
    """recompute_bwd re-derives each pixel's contributors (pairs whose box
    meets the warp's pixel block, then the pixel's box and alpha tests).  On
    a ragged 45 x 37 view, where warps straddle the image edge: its forward
    maps equal the stored-bits forward bit for bit (same contributors, same
    order), and its adjoint equals the oracle's, for 1, 2 and 4 pixels per
    thread and k = 3 and 8."""
    sc, cam = small_case(n=2500, w=45, h=37, seed=7, m=m, k=k)
    g = raster.Gaussians.from_scene(sc)
    outs = []
    for rec in (False, True):
        rast = raster.Rasterizer(px_per_thread=ppt, recompute_bwd=rec)
        with torch.no_grad():
            outs.append([t.cpu().numpy() for t in rast.forward(g, cam)])
    for a, b, name in zip(*outs, ("rgb", "depth", "sil", "sem")):
        np.testing.assert_array_equal(a, b, err_msg=name)
    for sem_detach in (True, False):
        grads, ref, _, _ = _bwd_case(sem_detach, seed=7, w=45, h=37, m=m, k=k, ppt=ppt, recompute=True)
        for name in ["means", "scales", "quats", "opacity", "rgb", "sem_w"]:
            _grad_close(grads[name], ref[name], name=(name, sem_detach))


def test_backward_semantic_block():
    sc, cam = small_case(n=2000, w=40, h=32, seed=3)
    g = raster.Gaussians.from_scene(sc)
    rast = raster.Rasterizer(sem_detach_geometry=True)
    H, W = cam.height, cam.width
    d_rgb = torch.randn(H, W, 3, device="cuda")
    d_sem = torch.randn(H, W, sc.m, device="cuda")
    rast.forward(g, cam)
    g1 = rast.backward(g, cam, d_rgb=d_rgb, d_sem=d_sem)
    rast.forward(g, cam)
    g0 = rast.backward(g, cam, d_rgb=d_rgb, d_sem=torch.zeros_like(d_sem))
    # equal up to the order of float atomics (run-to-run reordering ~1e-5)
    for name in ["means", "scales", "quats", "opacity", "rgb"]:
        _grad_close(g1[name].cpu().numpy(), g0[name].cpu().numpy(), rtol=1e-4, name=name, floor=WIDE)
    assert g1["sem_w"].abs().max() > 0 and g0["sem_w"].abs().max() == 0
    # contrast: without the block the semantic term changes geometric gradients
    rast2 = raster.Rasterizer(sem_detach_geometry=False)
    rast2.forward(g, cam)
    g2 = rast2.backward(g, cam, d_rgb=d_rgb, d_sem=d_sem)
    a, b = g2["opacity"].cpu().numpy(), g0["opacity"].cpu().numpy()
    assert np.abs(a - b).max() > 1e-2 * np.abs(b).max()


def test_autograd_function_end_to_end():
    sc, cam = small_case(n=2000, w=40, h=32, seed=4)
    g = raster.Gaussians.from_scene(sc)
    rast = raster.Rasterizer()
    params = [t.clone().requires_grad_(True) for t in (g.means, g.scales, g.quats, g.opacity, g.rgb, g.sem_w)]
    rgb, depth, sil, sem = raster.rasterize(rast, g, cam, *params)
    up = dict(d_rgb=np.random.default_rng(4).normal(size=(cam.height, cam.width, 3)).astype(np.float32),
              d_depth=np.ones((cam.height, cam.width), np.float32))
    _mask_flagged(up, oracle.render(sc, cam, prec="f32")["flag"])
    loss = (rgb * torch.from_numpy(up["d_rgb"]).cuda()).sum() + (depth * torch.from_numpy(up["d_depth"]).cuda()).sum()
    loss.backward()
    ref = oracle.render_bwd(sc, cam, **up, prec="f32")
    for p, name in zip(params, ["means", "scales", "quats", "opacity", "rgb", "sem_w"]):
        _grad_close(p.grad.cpu().numpy(), ref[name], name=name)


# ---------------------------------------------------------------------------
# candidates
# ---------------------------------------------------------------------------

def test_candidates_parity_mixed_resolutions():
    sc, _ = small_case(n=5000, m=16)
    rng = np.random.default_rng(5)
    sc.geo_unc = rng.gamma(2.0, 0.5, size=sc.n).astype(np.float32)
    cams = [scenes.look_camera((0.0, 0.0, 1.5), yaw, w, h, f)
            for yaw, (w, h, f) in zip([0, 30, -40, 90, 180],
                                      [(60, 34, 30.0), (120, 68, 60.0), (240, 136, 120.0), (60, 34, 30.0),
                                       (33, 21, 20.0)])]
    out = raster.Rasterizer().candidates(raster.Gaussians.from_scene(sc), cams).cpu().numpy()
    for v, cam in enumerate(cams):
        su, sh, ns, nf = oracle.candidate(sc, cam)
        assert abs(out[v, 0] - su) <= 1e-5 * abs(su) + 1e-3, (v, out[v, 0], su)
        assert abs(out[v, 1] - sh) <= 1e-5 * abs(sh), (v, out[v, 1], sh)
        assert abs(out[v, 2] - ns) <= nf, (v, out[v, 2], ns, nf)


def test_candidates_single_and_two_pass_agree():
    """Without room for contributor bits (recompute_bwd) the single-pass
    kernel runs; otherwise blend + class passes.  Same sums, and both match
    the oracle, with M = 300 (class chunks) and k = 8."""
    sc, _ = small_case(n=4000, m=300, k=8)
    rng = np.random.default_rng(6)
    sc.geo_unc = rng.gamma(2.0, 0.5, size=sc.n).astype(np.float32)
    cams = [scenes.look_camera((0.0, 0.0, 1.5), yaw, w, h, f)
            for yaw, (w, h, f) in zip([0, 25, -35], [(64, 40, 40.0), (96, 56, 60.0), (37, 29, 25.0)])]
    g = raster.Gaussians.from_scene(sc)
    a = raster.Rasterizer(recompute_bwd=True).candidates(g, cams).cpu().numpy()
    b = raster.Rasterizer().candidates(g, cams).cpu().numpy()
    np.testing.assert_allclose(a, b, rtol=1e-9, atol=1e-6)
    for v, cam in enumerate(cams):
        su, sh, ns, nf = oracle.candidate(sc, cam)
        assert abs(b[v, 0] - su) <= 1e-5 * abs(su) + 1e-3, (v, b[v, 0], su)
        assert abs(b[v, 1] - sh) <= 1e-5 * abs(sh), (v, b[v, 1], sh)
        assert abs(b[v, 2] - ns) <= nf, (v, b[v, 2], ns, nf)


def test_candidates_empty_views():
    sc, _ = small_case(n=300, m=20)
    cam = scenes.look_camera((0.0, 0.0, 1.5), 180.0, 50, 30, 40.0)
    sc.means[:, 0] = np.abs(sc.means[:, 0]) + 0.5  # everything behind this camera
    out = raster.Rasterizer().candidates(raster.Gaussians.from_scene(sc), [cam]).cpu().numpy()
    assert out[0, 2] == 50 * 30 and out[0, 0] == 0.0
    assert abs(out[0, 1] - 50 * 30 * np.log(20)) < 1e-3


# ---------------------------------------------------------------------------
# fused render + mean-L1
# ---------------------------------------------------------------------------

def _l1_case(seed=5, w=53, h=41, m=16, k=3, n=2500):
    """Scene, camera and a target frame (the oracle's render of a perturbed
    copy).  Target values within rounding of the rendered value (a sign that
    float32 rounding could flip) are nudged away, so the sign of
    (rendered - target) is the same on both sides."""
    sc, cam = small_case(n=n, w=w, h=h, seed=seed, m=m, k=k)
    rng = np.random.default_rng(seed)
    tgt = sc.subset(np.arange(sc.n))
    tgt.means = (tgt.means + rng.normal(0, 0.01, tgt.means.shape)).astype(np.float32)
    tgt.rgb = np.clip(tgt.rgb + rng.normal(0, 0.05, tgt.rgb.shape), 0, 1).astype(np.float32)
    tgt.sem_w = np.maximum(tgt.sem_w + rng.normal(0, 0.05, tgt.sem_w.shape), 0).astype(np.float32)
    t = oracle.render(tgt, cam, prec="f32")
    r = oracle.render(sc, cam, prec="f32")
    for key in ("rgb", "depth", "sem"):
        a, b = r[key], t[key]
        d = a.astype(np.float64) - b
        near = (np.abs(d) <= 1e-4 * (np.abs(a) + np.abs(b))) & (d != 0)
        b[near] = (b[near] - np.sign(d[near]) * 1e-3 * np.abs(b[near])).astype(np.float32)
    return sc, cam, t, r


@pytest.mark.parametrize("m,k", [(16, 3), (300, 8)])
def test_fused_l1_loss_and_gradients(m, k):
    """Loss equals mean-L1 of the oracle's render against the targets; the
    gradients equal the oracle adjoint for upstream 2 sign(x - t) / count
    (the loss is scaled by 2 before backward), and the unfused adjoint fed
    the same signs."""
    sc, cam, t, r = _l1_case(m=m, k=k, n=2000 if m > 100 else 2500)
    H, W = cam.height, cam.width
    assert (r["flag"] != 0).sum() == 0
    g = raster.Gaussians.from_scene(sc)
    rast = raster.Rasterizer()
    tt = [torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda() for x in (t["rgb"], t["depth"], t["sem"])]
    params = [p.clone().requires_grad_(True) for p in (g.means, g.scales, g.quats, g.opacity, g.rgb, g.sem_w)]
    loss = raster.render_l1(rast, g, cam, *tt, *params)
    (2.0 * loss).backward()
    ref_loss = (np.abs(r["rgb"].astype(np.float64) - t["rgb"]).mean() + np.abs(r["depth"] - t["depth"]).mean() +
                np.abs(r["sem"].astype(np.float64) - t["sem"]).mean())
    assert abs(loss.item() - ref_loss) <= 1e-5 * ref_loss
    up = dict(d_rgb=2.0 * np.sign(r["rgb"] - t["rgb"]).astype(np.float32) / (3 * H * W),
              d_depth=2.0 * np.sign(r["depth"] - t["depth"]).astype(np.float32) / (H * W),
              d_sem=2.0 * np.sign(r["sem"] - t["sem"]).astype(np.float32) / (H * W * m))
    ref = oracle.render_bwd(sc, cam, **up, prec="f32")
    for p, name in zip(params, ["means", "scales", "quats", "opacity", "rgb", "sem_w"]):
        _grad_close(p.grad.cpu().numpy(), ref[name], name=name)
    # fused adjoint vs the unfused adjoint fed the fused loss's own signs
    rast3 = raster.Rasterizer()
    rgb3, d3, s3, sem3 = rast3.forward(g, cam)
    _, d_rgb, d_depth, d_sem = raster.l1_loss_and_grads(rgb3, d3, sem3, *tt)
    unf = rast3.backward(g, cam, 2.0 * d_rgb, 2.0 * d_depth, None, 2.0 * d_sem)
    for p, name in zip(params, ["means", "scales", "quats", "opacity", "rgb", "sem_w"]):
        a, b = p.grad.cpu().numpy(), unf[name].cpu().numpy()
        _grad_close(a, b, rtol=1e-4, name=name, floor=WIDE)


def test_fused_l1_without_semantic_term():
    sc, cam, t, _ = _l1_case(seed=6)
    g = raster.Gaussians.from_scene(sc)
    rast = raster.Rasterizer()
    tr, td = (torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda() for x in (t["rgb"], t["depth"]))
    loss, (rgb, depth, sil, sem) = rast.forward_l1(g, cam, tr, td, None, outputs=True)
    ref = (rgb - tr).abs().mean() + (depth - td).abs().mean()
    assert abs(loss.item() - ref.item()) <= 1e-6 * ref.item()
    grads = rast.backward_l1(g, cam, torch.ones((), device="cuda"))
    assert grads["sem_w"].abs().max().item() == 0.0 and grads["means"].abs().max().item() > 0


# ---------------------------------------------------------------------------
# loss, capacity, graphs
# ---------------------------------------------------------------------------

def test_l1_loss_matches_torch():
    torch.manual_seed(0)
    H, W, m = 37, 53, 11
    x = [torch.rand(H, W, 3, device="cuda"), torch.rand(H, W, device="cuda"), torch.rand(H, W, m, device="cuda")]
    t = [torch.rand_like(a) for a in x]
    t[2][0, 0, 0] = x[2][0, 0, 0]  # an exact tie -> zero gradient
    loss, d_rgb, d_depth, d_sem = raster.l1_loss_and_grads(*x, *t)
    ref = sum((a - b).abs().mean() for a, b in zip(x, t))
    assert abs(loss.item() - ref.item()) <= 1e-6 * ref.item()
    for d, a, b in zip([d_rgb, d_depth, d_sem], x, t):
        np.testing.assert_array_equal(d.cpu().numpy(), (torch.sign(a - b) / a.numel()).cpu().numpy())
    assert d_sem[0, 0, 0].item() == 0.0


def test_capacity_overflow_reported_then_grown():
    sc, cam = small_case()
    g = raster.Gaussians.from_scene(sc)
    rast = raster.Rasterizer(pair_capacity=1000)
    rast._project_bin(g, [cam], check=False)
    cnt = rast.counters()
    assert cnt.status & (1 << 2) and cnt.n_pairs > 1000
    rgb, depth, sil, sem = rast.forward(g, cam, check=True)  # grows and reruns
    assert rast.counters().status == 0
    r = oracle.render(sc, cam, prec="f32")
    ok = r["flag"] & 1 == 0
    _img_close(sil.cpu().numpy(), r["sil"], ok)


def test_cuda_graph_capture_replay():
    sc, cam = small_case()
    g = raster.Gaussians.from_scene(sc)
    rast = raster.Rasterizer()
    ref = [t.clone() for t in rast.forward(g, cam, check=True)]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        rast.forward(g, cam, check=False)  # warm-up on the side stream
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        outs = rast.forward(g, cam, check=False)
    graph.replay()
    torch.cuda.synchronize()
    for a, b in zip(outs, ref):
        np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())
