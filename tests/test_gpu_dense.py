"""The dense-semantic comparator (gs_render_fwd_dense: every Gaussian
carries all M class probabilities, Eq. 3 blends all of them) against the
oracle, and the identity that ties it to the sparse path: a dense array
holding each Gaussian's top-k weights at their ids (zeros elsewhere) renders
the sparse path's maps bit for bit (a zero class adds exactly 0).

Tolerance against the oracle: 1e-5 max abs on pixels without a near-tie
threshold decision (as for the sparse forward)."""
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


def _close(a, b, ok):
    err = np.abs(a - b)
    if err.ndim > ok.ndim:
        err = err.reshape(ok.shape + (-1,)).max(-1)
    assert err[ok].max(initial=0.0) <= IMG_TOL, err[ok].max()


@pytest.mark.parametrize("m,w,h", [(40, 123, 77), (16, 64, 48), (102, 37, 29)])
def test_dense_matches_oracle(m, w, h):
    """Full distributions (one, two and four 32-class chunks, ragged last
    chunk and image edges) against the oracle rendering the same Gaussians
    with k = M (id c, weight p_c)."""
    sc = scenes.scene_plain(4, n=3000, m=m, k=3)
    cam = scenes.look_camera((0.0, 0.0, 1.5), 10.0, w, h, 60.0, pitch_deg=-5.0)
    dense = scenes.dense_distributions(sc, 5)
    r = oracle.render(scenes.dense_as_sparse(sc, dense), cam, prec="f32")
    ok = r["flag"] & 1 == 0
    assert (~ok).sum() <= max(2, ok.size // 1000)
    g = raster.Gaussians.from_scene(sc)
    out = raster.Rasterizer().forward_dense(g, cam, torch.from_numpy(dense).cuda())
    rgb, depth, sil, sem = (t.cpu().numpy() for t in out)
    _close(rgb, r["rgb"], ok)
    _close(depth, r["depth"], ok)
    _close(sil, r["sil"], ok)
    _close(sem, r["sem"], ok)


@pytest.mark.parametrize("tile", [(16, 16), (16, 8), (8, 8), (32, 8)])
def test_dense_of_sparse_entries_is_the_sparse_render(tile):
    sc = scenes.scene_room(3, n=60_000, m=102, k=3)
    assert all(len(set(r)) == sc.k for r in sc.sem_ids[:1000])  # distinct ids per Gaussian
    cam = scenes.look_camera((0.0, 0.0, 1.5), 30.0, 203, 141, 160.0, pitch_deg=-5.0)
    g = raster.Gaussians.from_scene(sc)
    rast = raster.Rasterizer(tile=tile)
    sparse = [t.cpu().numpy() for t in rast.forward(g, cam)]
    dense = [t.cpu().numpy() for t in rast.forward_dense(g, cam, torch.from_numpy(scenes.sparse_to_dense(sc)).cuda())]
    for a, b in zip(dense, sparse):
        np.testing.assert_array_equal(a, b)


def test_dense_needs_contributor_bits():
    sc = scenes.scene_plain(1, n=500, m=16, k=3)
    cam = scenes.look_camera((0.0, 0.0, 1.5), 10.0, 40, 30, 40.0)
    g = raster.Gaussians.from_scene(sc)
    with pytest.raises(N.GsError) as ei:
        raster.Rasterizer(recompute_bwd=True).forward_dense(g, cam, torch.zeros(sc.n, sc.m, device="cuda"))
    assert ei.value.code == N.GS_ERR_UNSUPPORTED


def test_dense_workload_shape():
    """The comparator workload of the runtime analysis: about 204k Gaussians
    in the rasterization of a 340x600 view, 102 classes, distributions
    summing to 1 with full support."""
    w = scenes.workload("dense204k")
    sc, cam, dense = w["scene"], w["cams"][0], w["sem_dense"]
    assert sc.m == 102 and (cam.height, cam.width) == (340, 600)
    assert dense.shape == (sc.n, sc.m) and (dense > 0).all()
    assert np.abs(dense.sum(1) - 1.0).max() < 1e-5
    g = raster.Gaussians.from_scene(sc)
    rast = raster.Rasterizer()
    rgb, depth, sil, sem = rast.forward_dense(g, cam, torch.from_numpy(dense).cuda())
    torch.cuda.synchronize()
    assert 200_000 <= rast.counters().n_records <= 208_000
    s = sem.sum(-1)
    assert torch.allclose(s, sil, atol=1e-4)  # sum_m P_m = S for normalised distributions
