"""Gaussians whose top-k class ids repeat (the interface accepts any ids in
[0, m), repeated or not): every entry is added, as Eq. 3 sums over the k
entries of each contributor.  The class passes read all of a Gaussian's class
slots before writing any; these cases check that a repeated id still sees the
earlier entry's add, against the oracle, for k = 3 (the chained form) and
k = 8 (the marked form), with and without class chunks, for the semantic map,
the fused mean-L1 loss and the candidate entropy."""
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


def _case(m, k, n=5000, w=96, h=64, seed=11):
    sc = scenes.scene_plain(seed, n=n, m=m, k=k)
    rng = np.random.default_rng(seed)
    ids = sc.sem_ids.copy()
    rows = rng.choice(sc.n, sc.n // 3, replace=False)
    for i in rows:  # one entry repeats an earlier one, every (later, earlier) pattern
        a = int(rng.integers(1, k))
        ids[i, a] = ids[i, int(rng.integers(0, a))]
    ids[rows[:40]] = ids[rows[:40], :1]  # all k entries the same class
    sc.sem_ids = np.ascontiguousarray(ids, np.int32)
    cam = scenes.look_camera((0.0, 0.0, 1.5), 10.0, w, h, 60.0, pitch_deg=-5.0)
    return sc, cam


@pytest.mark.parametrize("m,k", [(16, 3), (40, 8), (300, 8)])
def test_semantic_map_with_repeated_ids(m, k):
    sc, cam = _case(m, k)
    g = raster.Gaussians.from_scene(sc)
    with torch.no_grad():
        _, _, _, sem = raster.Rasterizer().forward(g, cam)
    r = oracle.render(sc, cam, prec="f32")
    ok = r["flag"] & 1 == 0
    err = np.abs(sem.cpu().numpy() - r["sem"]).reshape(ok.shape + (-1,)).max(-1)
    assert err[ok].max(initial=0.0) <= 1e-5, err[ok].max()


@pytest.mark.parametrize("m,k", [(16, 3), (40, 8)])
def test_fused_l1_with_repeated_ids(m, k):
    sc, cam = _case(m, k, seed=12)
    rng = np.random.default_rng(13)
    tgt = sc.subset(np.arange(sc.n))
    tgt.means = (tgt.means + rng.normal(0, 0.01, tgt.means.shape)).astype(np.float32)
    tgt.rgb = np.clip(tgt.rgb + rng.normal(0, 0.05, tgt.rgb.shape), 0, 1).astype(np.float32)
    tgt.sem_w = np.maximum(tgt.sem_w + rng.normal(0, 0.05, tgt.sem_w.shape), 0).astype(np.float32)
    t = oracle.render(tgt, cam, prec="f32")
    r = oracle.render(sc, cam, prec="f32")
    for key in ("rgb", "depth", "sem"):
        # targets within a relative 1e-4 of the render are moved 1e-3 away, so
        # that float32 rounding of the render cannot flip |render - target|
        # by more than its own size (as in the other fused-loss cases)
        a, b = r[key], t[key]
        d = a.astype(np.float64) - b
        near = (np.abs(d) <= 1e-4 * (np.abs(a) + np.abs(b))) & (d != 0)
        b[near] = (b[near] - np.sign(d[near]) * 1e-3 * np.abs(b[near])).astype(np.float32)
    g = raster.Gaussians.from_scene(sc)
    tt = [torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda() for x in (t["rgb"], t["depth"], t["sem"])]
    with torch.no_grad():
        loss = raster.Rasterizer().forward_l1(g, cam, *tt).item()
    ref = (np.abs(r["rgb"].astype(np.float64) - t["rgb"]).mean() + np.abs(r["depth"] - t["depth"]).mean() +
           np.abs(r["sem"].astype(np.float64) - t["sem"]).mean())
    assert abs(loss - ref) <= 1e-5 * ref, (loss, ref)


@pytest.mark.parametrize("m,k", [(16, 3), (40, 8)])
def test_candidates_with_repeated_ids(m, k):
    sc, _ = _case(m, k, n=4000, seed=14)
    sc.geo_unc = np.random.default_rng(15).gamma(2.0, 0.5, size=sc.n).astype(np.float32)
    cams = [scenes.look_camera((0.0, 0.0, 1.5), yaw, w, h, f)
            for yaw, (w, h, f) in zip([0, 40, -30], [(64, 40, 32.0), (128, 72, 64.0), (37, 23, 20.0)])]
    out = raster.Rasterizer().candidates(raster.Gaussians.from_scene(sc), cams).cpu().numpy()
    for v, cam in enumerate(cams):
        su, sh, ns, nf = oracle.candidate(sc, cam)
        assert abs(out[v, 0] - su) <= 1e-5 * abs(su) + 1e-3, (v, out[v, 0], su)
        assert abs(out[v, 1] - sh) <= 1e-5 * abs(sh), (v, out[v, 1], sh)
        assert abs(out[v, 2] - ns) <= nf, (v, out[v, 2], ns, nf)
