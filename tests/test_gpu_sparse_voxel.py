"""Top-k initialisation / update of the sparse semantic representation
(gs_topk_init, gs_topk_gather) and the Exploration Map (gs_voxel_update,
gs_voxel_new_free) on the GPU against the oracle.

Bars: top-k ids and weights bit-exact (a selection: integers and copied
floats).  Voxel states: every bit the oracle decides is set exactly as
decided, and bits the oracle leaves as near ties (segments grazing a voxel
edge within 1e-3 voxel; the cells around a point within 1e-3 voxel of a
face) may go either way.  Where ties may occur follows from the geometry
alone (voxel_ties.tie_cells): every tie must lie in the 27 cells around a segment
end within 2e-3 voxel of a face, or among the cells around a voxel edge
that the segment crosses a face within 2e-3 voxel of; so the tie count is
bounded by the size of that set, derived from the rays, not measured.
Newly freed voxels: bit-exact against the oracle on seeded random grids."""
import numpy as np
import pytest
import torch

from oracle import sparse as osp
from oracle import voxel as ovx
from voxel_ties import tie_cells
from paper_2506_00225_gb300 import explore, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_00225_gb300 import build
    build.build()


@pytest.mark.parametrize("k", [1, 3, 8, 16])
def test_topk_init_matches_oracle(k):
    rng = np.random.default_rng(k)
    m = 102
    probs = (rng.integers(0, 40, size=(3000, m)) / 40.0).astype(np.float32)  # many ties
    probs[rng.uniform(size=probs.shape) < 0.01] = np.nan
    rows = rng.integers(0, 3000, size=5000)
    ids, w = explore.topk_init(torch.from_numpy(probs).cuda(), k, torch.from_numpy(rows).cuda())
    rid, rw = osp.topk_init(probs, k, rows)
    np.testing.assert_array_equal(ids.cpu().numpy(), rid)
    np.testing.assert_array_equal(w.cpu().numpy(), rw)


def test_topk_init_all_rows_and_gather():
    rng = np.random.default_rng(7)
    probs = rng.dirichlet(np.full(40, 0.3), size=(64, 48)).astype(np.float32)  # an observed [H, W, M] map
    ids, w = explore.topk_init(torch.from_numpy(probs).cuda(), 3)
    rid, rw = osp.topk_init(probs.reshape(-1, 40), 3)
    np.testing.assert_array_equal(ids.cpu().numpy(), rid)
    np.testing.assert_array_equal(w.cpu().numpy(), rw)
    # a later observation updates the weights at the fixed ids
    obs = rng.dirichlet(np.full(40, 0.3), size=(64 * 48,)).astype(np.float32)
    rows = rng.permutation(64 * 48)
    ids_np = rid.copy()
    ids_np[5, 1] = -3  # an invalid id keeps its weight
    got = explore.topk_gather(torch.from_numpy(obs).cuda(), torch.from_numpy(ids_np).cuda(), w.clone(),
                              torch.from_numpy(rows).cuda())
    np.testing.assert_array_equal(got.cpu().numpy(), osp.topk_gather(obs, ids_np, rw, rows))


def _check_bits(gpu_bits, sure, maybe, tc):
    assert ((sure & ~gpu_bits) == 0).all(), "a decided bit is missing"
    assert ((gpu_bits & ~maybe) == 0).all(), "a bit the oracle rules out is set"
    # the oracle leaves undecided only voxels that the geometry allows
    ties = (sure != maybe)
    assert not (ties & ~tc).any(), int((ties & ~tc).sum())
    assert ties.sum() <= tc.sum() < (maybe != 0).sum() // 5, (ties.sum(), tc.sum())


def _bits_of(vm):
    w = vm.state.cpu().numpy().view(np.uint32)
    b = ((w[:, None] >> (2 * np.arange(16, dtype=np.uint32))[None, :]) & 3).reshape(-1)
    nx, ny, nz = vm.grid.nx, vm.grid.ny, vm.grid.nz
    return b[: nx * ny * nz].astype(np.uint8).reshape(nz, ny, nx)


@pytest.mark.parametrize("stride", [1, 3])
def test_voxel_update_matches_oracle(stride):
    rng = np.random.default_rng(stride)
    origin, vs, dims = (-1.0, -1.2, 0.0), 0.1, (48, 40, 20)
    cam = scenes.look_camera((0.3, 0.1, 1.1), 23.0, 40, 30, 25.0, pitch_deg=-12.0)
    depth = rng.uniform(0.4, 5.0, size=(30, 40)).astype(np.float32)
    depth[rng.uniform(size=depth.shape) < 0.05] = 0.0  # missing depth
    depth[0, :3] = np.nan
    vm = explore.VoxelMap(origin, vs, dims)
    vm.integrate(torch.from_numpy(depth).cuda(), cam, stride=stride, max_depth=3.5)
    torch.cuda.synchronize()
    sure, maybe = ovx.integrate(origin, vs, dims, depth, cam, stride=stride, max_depth=3.5)
    _check_bits(_bits_of(vm), sure, maybe, tie_cells(origin, vs, dims, depth, cam, stride=stride, max_depth=3.5))
    assert (sure & 2).any() and (sure & 1).any()


def test_voxel_two_frames_accumulate_and_camera_outside():
    rng = np.random.default_rng(11)
    origin, vs, dims = (0.0, 0.0, 0.0), 0.15, (30, 30, 14)
    cams = [scenes.look_camera((-0.8, 2.2, 1.0), 10.0, 32, 24, 20.0),
            scenes.look_camera((2.2, 2.2, 1.2), 200.0, 32, 24, 20.0, pitch_deg=8.0)]
    depths = [rng.uniform(0.5, 6.0, size=(24, 32)).astype(np.float32) for _ in cams]
    vm = explore.VoxelMap(origin, vs, dims)
    sure = np.zeros((dims[2], dims[1], dims[0]), np.uint8)
    maybe = np.zeros_like(sure)
    tie = np.zeros(sure.shape, bool)
    for cam, d in zip(cams, depths):
        vm.integrate(torch.from_numpy(d).cuda(), cam)
        s_, m_ = ovx.integrate(origin, vs, dims, d, cam)
        sure |= s_
        maybe |= m_
        tie |= tie_cells(origin, vs, dims, d, cam)
    torch.cuda.synchronize()
    _check_bits(_bits_of(vm), sure, maybe, tie)


@pytest.mark.parametrize("dims", [(16, 16, 16), (37, 23, 11), (130, 130, 40)])
def test_new_free_voxels_match_oracle(dims):
    rng = np.random.default_rng(sum(dims))
    origin, vs = (0.5, -0.25, 0.1), 0.05
    vm = explore.VoxelMap(origin, vs, dims)
    nvox = dims[0] * dims[1] * dims[2]
    prev = rng.choice(4, size=nvox, p=[0.6, 0.2, 0.1, 0.1]).astype(np.uint32)
    cur = prev | rng.choice(4, size=nvox, p=[0.5, 0.3, 0.1, 0.1]).astype(np.uint32)

    def pack(b):
        pad = np.zeros(vm.state.numel() * 16, np.uint32)
        pad[:nvox] = b
        return (pad.reshape(-1, 16) << (2 * np.arange(16, dtype=np.uint32))).sum(1, dtype=np.uint64).astype(
            np.uint32)
    vm.prev.copy_(torch.from_numpy(pack(prev).view(np.int32)))
    vm.state.copy_(torch.from_numpy(pack(cur).view(np.int32)))
    shape = (dims[2], dims[1], dims[0])
    ref = ovx.new_free(prev.reshape(shape).astype(np.uint8), cur.reshape(shape).astype(np.uint8), origin, vs)
    out, cnt = vm.new_free(capacity=len(ref) + 5)
    torch.cuda.synchronize()
    assert int(cnt.item()) == len(ref)
    np.testing.assert_allclose(out[: len(ref)].cpu().numpy(), ref, atol=1e-5)
    # a smaller capacity writes the first ones and still reports the count
    out2, cnt2 = vm.new_free(capacity=max(1, len(ref) // 3))
    torch.cuda.synchronize()
    assert int(cnt2.item()) == len(ref)
    np.testing.assert_array_equal(out2[: max(1, len(ref) // 3)].cpu().numpy(),
                                  out[: max(1, len(ref) // 3)].cpu().numpy())


def test_exploration_loop_on_device():
    """depth of the current view -> map update -> newly freed voxels ->
    lattice positions -> Fibonacci poses -> batched candidate renders ->
    Eq. 6-8 scores -> best view: every step runs, and the best view is a
    kept candidate."""
    from paper_2506_00225_gb300 import raster
    sc = scenes.scene_plain(5, n=1500, m=16, k=3)
    g = raster.Gaussians.from_scene(sc)
    cam = scenes.look_camera((0.0, 0.0, 1.5), 30.0, 64, 48, 40.0)
    rast = raster.Rasterizer()
    _, depth, sil, _ = rast.forward(g, cam)
    depth = torch.where(sil > 0.5, depth / sil.clamp_min(1e-6), torch.zeros_like(depth))
    vm = explore.VoxelMap((-2.0, -2.0, 0.0), 0.05, (80, 80, 60))
    centres, cnt = vm.update(depth, cam, stride=2, max_depth=3.0, capacity=1 << 18)
    n_new = int(cnt.item())
    assert n_new > 0
    pos = explore.candidate_positions(centres[: min(n_new, 1 << 18)].cpu().numpy(), 1.0, [1.5], 0.05)
    assert len(pos) > 0
    cams = explore.candidate_poses(pos, 5, 48, 32, 30.0)
    sums, scores, keep, best = explore.next_best_view(rast, g, cams, cam.position())
    torch.cuda.synchronize()
    b = int(best.item())
    assert b == -1 or bool(keep[b])
