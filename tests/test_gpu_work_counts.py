"""The GPU work counters (gs_count_work) against the oracle's own counts:
per pixel, the evaluations of the per-pixel definition (pixel-rectangle
pairs up to and including the stopping pair) and the contributions, bit for
bit on every pixel the oracle does not flag as near a threshold; the
contributions also equal the forward blend's own counter; the classes above
the 0.001 clip floor of Eq. 7 within the entries near that floor.  These
counts are the work figures of the forward and candidate rooflines."""
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


def _case(w, h, n=8000, seed=3, m=16, k=3):
    sc = scenes.scene_plain(seed, n=n, m=m, k=k)
    cam = scenes.look_camera((0.0, 0.0, 1.5), 20.0, w, h, 55.0, pitch_deg=-4.0)
    return sc, cam


@pytest.mark.parametrize("tile,size", [((16, 16), (80, 60)), ((8, 8), (123, 77)), ((32, 8), (97, 41))])
def test_per_pixel_counts_match_the_oracle(tile, size):
    sc, cam = _case(*size)
    g = raster.Gaussians.from_scene(sc)
    rast = raster.Rasterizer(tile=tile)
    rast.forward(g, cam)
    n_blend = int(rast.counters().n_contrib)
    wc = rast.work_counts(g, [cam], per_pixel=True)
    ref = oracle.render(sc, cam, prec="f32")
    ok = ref["flag"] == 0
    assert ok.mean() > 0.99
    pp = wc["per_pixel"]
    np.testing.assert_array_equal(pp[..., 0][ok], ref["n_eval_px"][ok])
    np.testing.assert_array_equal(pp[..., 1][ok], ref["n_contrib"][ok])
    assert wc["n_eval"] == int(pp[..., 0].sum()) and wc["n_contrib"] == int(pp[..., 1].sum())
    assert wc["n_contrib"] == n_blend  # the blend kernel's own count of the same contributions
    if ok.all():
        assert wc["n_eval"] == ref["n_eval"] and wc["n_contrib"] == ref["n_contrib_total"]
    assert wc["n_contrib"] <= wc["n_eval_box"] <= wc["n_eval"]
    assert wc["n_pixels"] == cam.width * cam.height
    # classes above the clip floor: the oracle's map, up to entries within
    # float rounding of the floor and the flagged pixels' classes
    sem = ref["sem"]
    touched = int((sem > np.float32(0.001)).sum())
    near = int((np.abs(sem - np.float32(0.001)) < 1e-6).sum()) + int((~ok).sum()) * sc.m
    assert abs(wc["n_touched"] - touched) <= near


def test_multi_view_totals_are_the_sum_of_the_views():
    """Candidate sets: one call over views of mixed resolutions counts what
    the views count one by one (the oracle's totals per view)."""
    sc, _ = _case(64, 48)
    cams = [scenes.look_camera((0.0, 0.0, 1.5), yaw, w, h, f, pitch_deg=-4.0)
            for yaw, (w, h, f) in zip((0.0, 60.0, 140.0), ((48, 36, 30.0), (96, 72, 60.0), (64, 48, 40.0)))]
    g = raster.Gaussians.from_scene(sc)
    wc = raster.Rasterizer().work_counts(g, cams)
    ne = nc = flagged = 0
    for cam in cams:
        ref = oracle.render(sc, cam, prec="f32")
        ne += ref["n_eval"]
        nc += ref["n_contrib_total"]
        flagged += int((ref["flag"] != 0).sum())
    assert wc["n_pixels"] == sum(c.width * c.height for c in cams)
    if flagged == 0:
        assert wc["n_eval"] == ne and wc["n_contrib"] == nc
    else:
        assert abs(wc["n_contrib"] - nc) <= 64 * flagged
    assert wc["n_contrib"] <= wc["n_eval_box"] <= wc["n_eval"]


def test_counts_of_an_empty_view():
    """A view with nothing in front of the camera: no evaluations, no
    contributions, no class above the floor."""
    sc, _ = _case(32, 24)
    cam = scenes.look_camera((0.0, 0.0, 50.0), 0.0, 32, 24, 30.0, pitch_deg=80.0)
    wc = raster.Rasterizer().work_counts(raster.Gaussians.from_scene(sc), [cam])
    assert wc["n_eval"] == wc["n_eval_box"] == wc["n_contrib"] == wc["n_touched"] == 0
    assert wc["n_pixels"] == 32 * 24
