"""gs_render_fwd_noalloc: the forward render for callers that cannot
allocate device memory (graph capture, real-time loops, hosts that own all
device memory).  Its workspace is a fixed device array inside the library;
these checks compare it, through the C ABI, with the CPU oracle and with the
regular entry points (gs_project + gs_bin_sort + gs_render_fwd on a
caller-allocated workspace) on two calls in a row, with the image tolerance
of the parity tests."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2506_00225_gb300 import _native as N
from paper_2506_00225_gb300 import raster, scenes

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_00225_gb300 import build
    build.build()


def _noalloc(g, cam, cfg):
    lib = N.load()
    H, W = cam.height, cam.width
    out = [torch.full((H, W, 3), -7.0, device="cuda"), torch.full((H, W), -7.0, device="cuda"),
           torch.full((H, W), -7.0, device="cuda"), torch.full((H, W, g.m), -7.0, device="cuda")]
    cnt = torch.zeros(4, dtype=torch.int32, device="cuda")
    sc = raster.scene_struct(g.means, g.scales, g.quats, g.opacity, g.rgb, g.sem_ids, g.sem_w, g.m)
    cams = raster.cameras_array([cam])
    st = lib.gs_render_fwd_noalloc(ctypes.byref(sc), cams, ctypes.byref(cfg), *[ctypes.c_void_p(t.data_ptr())
                                                                                 for t in out],
                                   ctypes.c_void_p(cnt.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream()
                                                                                    .cuda_stream))
    assert st == N.GS_OK, lib.gs_status_string(st)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in out], cnt.cpu().numpy().view(np.uint32)


def _regular(g, cam, cfg):
    rast = raster.Rasterizer(tile=(cfg.tile_w, cfg.tile_h), record_capacity=cfg.record_capacity,
                             pair_capacity=cfg.pair_capacity)
    with torch.no_grad():
        out = rast.forward(g, cam, check=False)
    c = rast.counters()
    return [t.cpu().numpy() for t in out], c


def _cfg(n, pairs):
    cfg = N.GsConfig()
    cfg.tile_w, cfg.tile_h = 16, 16
    cfg.sem_detach_geometry = 1
    cfg.record_capacity = n
    cfg.pair_capacity = pairs
    return cfg


def test_noalloc_matches_regular_entry_points_twice():
    cases = [(scenes.scene_plain(0, n=6000, m=16, k=3), scenes.look_camera((0.0, 0.0, 1.5), 10.0, 123, 77, 60.0)),
             (scenes.scene_plain(1, n=3000, m=40, k=5), scenes.look_camera((0.1, 0.0, 1.4), -20.0, 64, 48, 45.0))]
    for sc, cam in cases:  # two calls in a row, different sizes: no state leaks between calls
        g = raster.Gaussians.from_scene(sc)
        cfg = _cfg(sc.n, 1 << 19)
        got, cnt = _noalloc(g, cam, cfg)
        ref, rc = _regular(g, cam, cfg)
        assert cnt[0] == 0 and rc.status == 0
        assert (cnt[1], cnt[2]) == (rc.n_records, rc.n_pairs)
        for a, b in zip(got, ref):
            assert a.shape == b.shape
            assert np.abs(a - b).max() <= IMG_TOL


def test_noalloc_matches_oracle():
    """Eq. 1 colour, depth, silhouette and Eq. 3 class map against the
    oracle, element by element, on a ragged 123 x 77 view (pixels whose
    threshold decision the oracle flags as within rounding are excluded and
    counted, as in the parity tests)."""
    sc = scenes.scene_plain(2, n=6000, m=16, k=3)
    cam = scenes.look_camera((0.0, 0.0, 1.5), 10.0, 123, 77, 60.0, pitch_deg=-5.0)
    g = raster.Gaussians.from_scene(sc)
    got, cnt = _noalloc(g, cam, _cfg(sc.n, 1 << 19))
    assert cnt[0] == 0
    r = oracle.render(sc, cam, prec="f32")
    ok = r["flag"] & 1 == 0
    assert (~ok).sum() <= max(2, ok.size // 1000)
    for x, name in zip(got, ("rgb", "depth", "sil", "sem")):
        err = np.abs(x - r[name])
        if err.ndim > ok.ndim:
            err = err.reshape(ok.shape + (-1,)).max(-1)
        assert err[ok].max(initial=0.0) <= IMG_TOL, (name, err[ok].max())


def test_noalloc_rejects_sizes_beyond_its_scratch():
    sc = scenes.scene_plain(0, n=6000, m=16, k=3)
    g = raster.Gaussians.from_scene(sc)
    cam = scenes.look_camera((0.0, 0.0, 1.5), 10.0, 123, 77, 60.0)
    cfg = _cfg(sc.n, N.GS_NOALLOC_SCRATCH_BYTES // 8)  # pair buffers alone exceed the array
    lib = N.load()
    scs = raster.scene_struct(g.means, g.scales, g.quats, g.opacity, g.rgb, g.sem_ids, g.sem_w, g.m)
    assert lib.gs_workspace_size(ctypes.byref(scs), raster.cameras_array([cam]), 1, ctypes.byref(cfg)) > \
        N.GS_NOALLOC_SCRATCH_BYTES
    st = lib.gs_render_fwd_noalloc(ctypes.byref(scs), raster.cameras_array([cam]), ctypes.byref(cfg), None, None,
                                   None, None, None, None)
    assert st == N.GS_ERR_TOO_LARGE
    assert b"scratch" in lib.gs_status_string(st)
