"""Candidate renders with every staged batch size and tile shape, and with
the contributor bits bounded so that the views run in several waves (and
some tiles re-test their pairs): the per-view sums equal the oracle's and
do not depend on the configuration."""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_00225_gb300 import raster, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_00225_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def case():
    sc = scenes.scene_plain(11, n=6000, m=20, k=3)
    rng = np.random.default_rng(12)
    sc.geo_unc = rng.gamma(2.0, 0.5, size=sc.n).astype(np.float32)
    cams = [scenes.look_camera((0.0, 0.0, 1.5), yaw, w, h, f, pitch_deg=-3.0)
            for yaw, (w, h, f) in zip([0, 35, -50, 120, 200, 260],
                                      [(75, 42, 37.5), (150, 85, 75.0), (300, 170, 150.0), (75, 42, 37.5),
                                       (150, 85, 75.0), (47, 33, 30.0)])]
    refs = [oracle.candidate(sc, c) for c in cams]
    return sc, cams, refs


def _check(out, refs):
    for v, (su, sh, ns, nf) in enumerate(refs):
        assert abs(out[v, 0] - su) <= 1e-5 * abs(su) + 1e-3, (v, out[v, 0], su)
        assert abs(out[v, 1] - sh) <= 1e-5 * abs(sh), (v, out[v, 1], sh)
        assert abs(out[v, 2] - ns) <= nf, (v, out[v, 2], ns, nf)


@pytest.mark.parametrize("batch", [32, 64, 128])
@pytest.mark.parametrize("tile", [(16, 16), (16, 8), (32, 8), (8, 8)])
def test_batch_sizes_and_tiles_match_the_oracle(case, batch, tile):
    sc, cams, refs = case
    out = raster.Rasterizer(tile=tile, cand_batch=batch).candidates(raster.Gaussians.from_scene(sc), cams)
    _check(out.cpu().numpy(), refs)


@pytest.mark.parametrize("budget", [1 << 16, 3 << 20, 8 << 20])
def test_bounded_bits_run_in_waves(case, budget):
    """A bit budget far below what the views need: several waves of views,
    and tiles of views larger than the budget re-test their pairs.  Same
    sums as the unbounded call (up to the order of the per-view double
    additions) and as the oracle."""
    sc, cams, refs = case
    g = raster.Gaussians.from_scene(sc)
    free = raster.Rasterizer().candidates(g, cams).cpu().numpy()
    rast = raster.Rasterizer(cand_bits_bytes=budget)
    out = rast.candidates(g, cams).cpu().numpy()
    np.testing.assert_allclose(out, free, rtol=1e-9, atol=1e-6)
    _check(out, refs)


def test_bits_stay_within_the_budget_at_the_128_view_workload():
    """The 2M-Gaussian 128-view set: its contributor bits would need about
    9 GB (287M pairs); the workspace keeps at most the default 4 GiB of them
    (its size minus the same layout without bits), the rest being the 66M
    records and the pairs themselves, and the sampled views still match the
    oracle."""
    import ctypes
    from paper_2506_00225_gb300 import _native as N
    wl = scenes.workload("mixed2m")
    sc, cams = wl["scene"], wl["cand_cams"]
    g = raster.Gaussians.from_scene(sc)
    rast = raster.Rasterizer()
    out = rast.candidates(g, cams).cpu().numpy()
    out2 = rast.candidates(g, cams).cpu().numpy()  # fitted capacities, same result
    np.testing.assert_allclose(out, out2, rtol=1e-9, atol=1e-6)
    cnt = rast.counters()
    cfg = rast.config(g.n, len(cams))
    s_ = raster.scene_struct(g.means, g.scales, g.quats, g.opacity, g.rgb, g.sem_ids, g.sem_w, g.m, g.geo_unc)
    cams_arr = raster.cameras_array(cams)
    lib = N.load()
    with_bits = lib.gs_workspace_size(ctypes.byref(s_), cams_arr, len(cams), ctypes.byref(cfg))
    cfg.cand_bits_bytes = 1  # below one unit: no bits
    without = lib.gs_workspace_size(ctypes.byref(s_), cams_arr, len(cams), ctypes.byref(cfg))
    tiles = sum(((c.width + 15) // 16) * ((c.height + 15) // 16) for c in cams)
    need = (cnt.n_pairs // 64 + tiles) * 8 * 256
    assert need > (8 << 30)  # what unbounded bits would take
    assert with_bits - without <= (4 << 30) + 4 * 256 * tiles + (1 << 20), (with_bits, without)
    assert rast.ws.numel() >= with_bits
    for v in [v for v, c in enumerate(cams) if c.width == 300][:2]:
        su, sh, ns, nf = oracle.candidate(sc, cams[v])
        assert abs(out[v, 1] - sh) <= 1e-5 * abs(sh), (v, out[v, 1], sh)
        assert abs(out[v, 2] - ns) <= nf, (v, out[v, 2], ns, nf)


# (pixel budget, groups of views it makes); the views have 3150, 12750,
# 51000, 3150, 12750 and 1551 pixels
GROUPINGS = [(1, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (5, 6)]),
             (16_000, [(0, 2), (2, 3), (3, 5), (5, 6)]),
             (60_000, [(0, 2), (2, 4), (4, 6)])]


@pytest.mark.parametrize("budget,groups", GROUPINGS)
def test_grouped_views_match_the_whole_call(case, budget, groups):
    """Views projected, binned and rendered in pixel-bounded groups within
    one workspace: the same sums as the call over all views at once and as
    the oracle; the counters report the largest group's records and pairs
    (each group's own counts taken from separate calls), so the capacities
    fitted from them hold every group and the refitted call agrees."""
    sc, cams, refs = case
    g = raster.Gaussians.from_scene(sc)
    free = raster.Rasterizer().candidates(g, cams).cpu().numpy()
    rast = raster.Rasterizer(cand_group_pixels=budget)
    out = rast.candidates(g, cams).cpu().numpy()
    np.testing.assert_allclose(out, free, rtol=1e-9, atol=1e-6)
    _check(out, refs)
    cnt = rast.counters()
    recs, pairs = [], []
    for a, b in groups:
        r1 = raster.Rasterizer()
        r1.candidates(g, cams[a:b])
        c1 = r1.counters()
        recs.append(c1.n_records)
        pairs.append(c1.n_pairs)
    assert (cnt.n_records, cnt.n_pairs) == (max(recs), max(pairs)), (cnt.n_records, cnt.n_pairs, recs, pairs)
    out2 = rast.candidates(g, cams).cpu().numpy()
    np.testing.assert_allclose(out2, free, rtol=1e-9, atol=1e-6)


def test_grouped_128_view_workload_fits_8_gib():
    """The 2M-Gaussian 128-view set (66M records, 717M pairs at once): the
    largest pixel budget whose fitted workspace fits 8 GiB renders the same
    per-view sums as the call over all views at once, within 8 GiB."""
    from paper_2506_00225_gb300 import autotune
    wl = scenes.workload("mixed2m")
    sc, cams = wl["scene"], wl["cand_cams"]
    g = raster.Gaussians.from_scene(sc)
    whole = raster.Rasterizer().candidates(g, cams).cpu().numpy()
    rast, budget, ws = autotune.fit_candidate_budget(g, cams, 8 << 30)
    assert 0 < budget and ws <= (8 << 30), (budget, ws)
    out = rast.candidates(g, cams).cpu().numpy()
    np.testing.assert_allclose(out, whole, rtol=1e-9, atol=1e-6)
    assert rast.counters().status == 0
