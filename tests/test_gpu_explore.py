"""The Eq. 6-8 scoring tail on the device (gs_score_candidates) against the
oracle's float64 scoring: random per-view sums over 1 to 1000 candidates
(more than one CTA's width of threads), sums of the oracle's own candidate
reductions over generated candidate poses, the pruning boundary and empty
pools.  Scores within 1e-12 relative (double on both sides, different
summation order and exp rounding); pool flags and the best index exact."""
import numpy as np
import pytest
import torch

import oracle
from oracle import explore as ex
from paper_2506_00225_gb300 import explore, raster, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_00225_gb300 import build
    build.build()


def _gpu_score(sums, npix, pos, cur, frac=0.005):
    t = lambda a, dt: torch.tensor(np.asarray(a), dtype=dt, device="cuda")
    s, k, b = explore.score_candidates(t(sums, torch.float64), t(npix, torch.int32), t(pos, torch.float32),
                                       t(cur, torch.float32), frac)
    torch.cuda.synchronize()
    return s.cpu().numpy(), k.cpu().numpy().astype(bool), int(b.item())


def _check(sums, npix, pos, cur, frac=0.005):
    s, k, b = _gpu_score(sums, npix, pos, cur, frac)
    # the oracle sees the positions as the device does (float32)
    rs, rk, rb = ex.score(sums, npix, np.asarray(pos, np.float32), np.asarray(cur, np.float32), frac)
    np.testing.assert_allclose(s, rs, rtol=1e-12, atol=1e-300)
    np.testing.assert_array_equal(k, rk)
    assert b == rb
    return s, k, b


@pytest.mark.parametrize("V", [1, 7, 96, 300, 1000])
def test_scores_match_oracle(V):
    rng = np.random.default_rng(V)
    npix = rng.choice([170 * 300, 340 * 600], size=V)
    ns = np.floor(rng.uniform(0, 0.05, size=V) * npix)
    ns[rng.uniform(size=V) < 0.2] = 0.0
    sh = rng.uniform(0.0, 30.0, size=V)  # spread of a few units: a non-degenerate softmax
    sums = np.stack([rng.uniform(0, 1e4, size=V), sh, ns], axis=1)
    pos = rng.uniform(-5, 5, size=(V, 3))
    _check(sums, npix, pos, rng.uniform(-5, 5, size=3))


def test_pruning_boundary_and_empty_pool():
    npix = np.array([1000, 1000, 1000, 2000])
    sums = np.array([[0, 1.0, 5.0], [0, 1.0, 4.0], [0, 1.0, 6.0], [0, 1.0, 9.0]])  # 0.5 %: 5 of 1000, 10 of 2000
    s, k, b = _check(sums, npix, np.zeros((4, 3)), np.zeros(3))
    assert k.tolist() == [True, False, True, False] and b == 2
    # nothing revealed anywhere: all geometric factors 0, every view pruned
    s, k, b = _check(np.zeros((5, 3)), np.full(5, 100), np.zeros((5, 3)), np.ones(3))
    assert not s[:, 0].any() and not k.any() and b == -1


def test_scores_of_oracle_candidate_sums_over_generated_poses():
    """Candidates generated the paper's way (lattice positions over free
    space, 5 Fibonacci directions), their sums from the oracle's candidate
    reductions, scored on the device and by the oracle."""
    sc = scenes.scene_plain(3, n=800, m=16, k=3)  # sparse enough to leave holes: some views kept, some pruned
    rng = np.random.default_rng(2)
    free = rng.uniform([-1.5, -1.5, 1.3], [1.5, 1.5, 1.7], size=(400, 3))
    pos = explore.candidate_positions(free, 1.0, [1.5], 0.25)
    cams = explore.candidate_poses(pos, 5, 48, 32, 30.0)
    sums = np.array([oracle.candidate(sc, c)[:3] for c in cams], np.float64)
    npix = np.array([c.width * c.height for c in cams])
    cur = np.array([0.2, -0.1, 1.5])
    s, k, b = _check(sums, npix, np.stack([c.position() for c in cams]), cur)
    assert len(cams) == 5 * len(pos) and k.any() and not k.all()


def test_next_best_view_pipeline_runs_on_device():
    """render the candidates and score them without leaving the device:
    graph-capturable, and the same result as the two calls made eagerly."""
    sc = scenes.scene_plain(4, n=6000, m=16, k=3)
    g = raster.Gaussians.from_scene(sc)
    pos = np.array([[0.0, 0.0, 1.5], [1.0, 0.0, 1.5], [0.0, 1.0, 1.2]], np.float32)
    cams = explore.candidate_poses(pos, 5, 64, 40, 40.0)
    rast = raster.Rasterizer()
    sums, scores, keep, best = explore.next_best_view(rast, g, cams, (0.1, 0.1, 1.5))
    torch.cuda.synchronize()
    s2, k2, b2 = explore.score_candidates(sums, torch.tensor([64 * 40] * len(cams), device="cuda"),
                                          torch.tensor(np.stack([c.position() for c in cams]), device="cuda"),
                                          torch.tensor([0.1, 0.1, 1.5], device="cuda"))
    torch.cuda.synchronize()
    assert torch.equal(scores, s2) and torch.equal(keep, k2) and torch.equal(best, b2)
    assert -1 <= int(best.item()) < len(cams)
