"""Host-side candidate generation of the library (gs_candidate_poses,
gs_candidate_positions) against the oracle's Fibonacci lattice, look-along
poses and lattice positions; host argument checks of gs_score_candidates.
No GPU needed."""
import ctypes

import numpy as np
import pytest

from oracle import explore as ex
from paper_2506_00225_gb300 import _native as N
from paper_2506_00225_gb300 import build as B


@pytest.fixture(scope="module")
def lib():
    B.build()
    return N.load()


@pytest.mark.parametrize("n_dirs", [1, 5, 15])
def test_candidate_poses_match_oracle(lib, n_dirs):
    from paper_2506_00225_gb300 import explore
    rng = np.random.default_rng(n_dirs)
    pos = rng.uniform(-4, 4, size=(7, 3)).astype(np.float32)
    cams = explore.candidate_poses(pos, n_dirs, 600, 340, 300.0)
    assert len(cams) == 7 * n_dirs
    dirs = ex.fibonacci_directions(n_dirs)
    for p in range(7):
        for i in range(n_dirs):
            c = cams[p * n_dirs + i]
            assert (c.width, c.height, c.fx, c.fy, c.cx, c.cy) == (600, 340, 300.0, 300.0, 300.0, 170.0)
            ref = ex.look_along(pos[p].astype(np.float64), dirs[i]).astype(np.float32)
            np.testing.assert_allclose(c.w2c, ref, atol=2e-6)
            np.testing.assert_allclose(c.position(), pos[p], atol=1e-5)


def test_candidate_positions_match_oracle(lib):
    from paper_2506_00225_gb300 import explore
    rng = np.random.default_rng(3)
    centres = np.concatenate([rng.uniform([-3, -3, 0], [3, 3, 3], size=(5000, 3)),
                              np.array([[0.25, 0.25, 1.5], [-0.25, -0.25, 1.5]])]).astype(np.float32)
    for step, heights, band in [(1.0, [1.5], 0.05), (0.5, [0.75, 1.5, 2.25], 0.05), (0.5, [1.0], 0.0)]:
        got = explore.candidate_positions(centres, step, heights, band)
        ref = ex.candidate_positions(centres, step, heights, band).astype(np.float32)
        np.testing.assert_array_equal(got, ref)
    # exact-half coordinates round up in both (floor(x / step + 0.5))
    assert explore.candidate_positions(np.array([[0.25, -0.25, 1.0]]), 0.5, [1.0], 0.0).tolist() == \
        [[0.5, 0.0, 1.0]]
    assert explore.candidate_positions(np.zeros((0, 3)), 1.0, [1.5], 0.1).shape == (0, 3)


def test_generation_argument_checks(lib):
    cams = (N.GsCamera * 4)()
    p = np.zeros((2, 3), np.float32)
    pp = p.ctypes.data_as(ctypes.c_void_p)
    assert lib.gs_candidate_poses(2, pp, 0, 64, 48, 50.0, 50.0, 0.2, cams) == N.GS_ERR_ARG
    assert lib.gs_candidate_poses(2, pp, 2, 0, 48, 50.0, 50.0, 0.2, cams) == N.GS_ERR_ARG
    assert lib.gs_candidate_poses(2, pp, 2, 64, 48, float("nan"), 50.0, 0.2, cams) == N.GS_ERR_ARG
    h = np.array([1.0], np.float32)
    hp = h.ctypes.data_as(ctypes.c_void_p)
    assert lib.gs_candidate_positions(2, pp, 0.0, 1, hp, 0.1, None, 0) == -1
    assert lib.gs_candidate_positions(2, pp, 1.0, 0, hp, 0.1, None, 0) == -1
    assert lib.gs_candidate_positions(2, pp, 1.0, 1, hp, -1.0, None, 0) == -1
    # counting only (capacity 0) is allowed
    assert lib.gs_candidate_positions(2, pp, 1.0, 1, hp, 1.0, None, 0) == 1


def test_score_argument_checks_on_host(lib):
    fake = ctypes.c_void_p(1 << 40)  # never dereferenced: every call returns before GPU work
    assert lib.gs_score_candidates(0, fake, fake, fake, fake, 0.005, fake, fake, fake, None) == N.GS_ERR_ARG
    assert lib.gs_score_candidates(3, None, fake, fake, fake, 0.005, fake, fake, fake, None) == N.GS_ERR_ARG
    assert lib.gs_score_candidates(3, fake, fake, fake, fake, 1.5, fake, fake, fake, None) == N.GS_ERR_ARG
    assert lib.gs_score_candidates(3, fake, fake, fake, fake, float("nan"), fake, fake, fake, None) == N.GS_ERR_ARG


def test_topk_and_voxel_argument_checks_on_host(lib):
    fake = ctypes.c_void_p(1 << 40)  # never dereferenced: every call returns before GPU work
    assert lib.gs_topk_init(10, 5, 6, fake, None, fake, fake, None) == N.GS_ERR_ARG   # k > m
    assert lib.gs_topk_init(10, 40, 17, fake, None, fake, fake, None) == N.GS_ERR_ARG  # k > 16
    assert lib.gs_topk_init(10, 40, 3, None, None, fake, fake, None) == N.GS_ERR_ARG
    assert lib.gs_topk_init(0, 40, 3, None, None, None, None, None) == N.GS_OK          # nothing to do
    assert lib.gs_topk_gather(10, 40, 0, fake, None, fake, fake, None) == N.GS_ERR_ARG
    g = N.GsVoxelGrid()
    g.voxel, g.nx, g.ny, g.nz = 0.05, 100, 80, 40
    assert lib.gs_voxel_words(ctypes.byref(g)) == (100 * 80 * 40 + 15) // 16
    assert lib.gs_voxel_scratch_words(ctypes.byref(g)) == ((100 * 80 * 40 + 15) // 16 + 2047) // 2048 + 1
    cam = (N.GsCamera * 1)()
    cam[0].width, cam[0].height, cam[0].fx, cam[0].fy = 8, 6, 5.0, 5.0
    assert lib.gs_voxel_update(ctypes.byref(g), fake, fake, cam, 0, 5.0, None) == N.GS_ERR_ARG
    assert lib.gs_voxel_update(ctypes.byref(g), fake, fake, cam, 1, 0.0, None) == N.GS_ERR_ARG
    assert lib.gs_voxel_new_free(ctypes.byref(g), fake, fake, fake, None, 5, fake, None) == N.GS_ERR_ARG
    bad = N.GsVoxelGrid()
    bad.voxel, bad.nx, bad.ny, bad.nz = 0.0, 10, 10, 10
    assert lib.gs_voxel_words(ctypes.byref(bad)) == -1
    bad.voxel, bad.nx = 0.05, 0
    assert lib.gs_voxel_words(ctypes.byref(bad)) == -1
