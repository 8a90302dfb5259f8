"""Candidate management around the candidate renders (Sec. 3.2): candidate
positions on a lattice over newly freed space, Fibonacci-lattice viewing
directions, and the Eq. 6-8 scoring tail on the device (argument
marshalling only; the work runs in ``libgs``)."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native as N
from .scenes import Camera


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def candidate_positions(voxel_centres: np.ndarray, step: float, heights, band: float) -> np.ndarray:
    """Lattice points (spacing ``step``) over the given voxel centres at the
    given heights (a voxel counts for a height within ``band`` of it).
    Returns [C, 3] float32, ascending (i, j, height index)."""
    c = np.ascontiguousarray(voxel_centres, dtype=np.float32).reshape(-1, 3)
    h = np.ascontiguousarray(heights, dtype=np.float32).reshape(-1)
    lib = N.load()
    n = lib.gs_candidate_positions(c.shape[0], c.ctypes.data_as(ctypes.c_void_p), float(step), h.size,
                                   h.ctypes.data_as(ctypes.c_void_p), float(band), None, 0)
    if n < 0:
        raise ValueError("invalid candidate position arguments")
    out = np.empty((max(n, 1), 3), np.float32)
    n2 = lib.gs_candidate_positions(c.shape[0], c.ctypes.data_as(ctypes.c_void_p), float(step), h.size,
                                    h.ctypes.data_as(ctypes.c_void_p), float(band),
                                    out.ctypes.data_as(ctypes.c_void_p), n)
    assert n2 == n
    return out[:n]


def candidate_poses(positions: np.ndarray, n_dirs: int, width: int, height: int, f: float,
                    near: float = 0.2) -> list[Camera]:
    """Cameras at every position looking along the n_dirs directions of a
    Fibonacci lattice on the sphere (position-major order)."""
    p = np.ascontiguousarray(positions, dtype=np.float32).reshape(-1, 3)
    arr = (N.GsCamera * max(1, p.shape[0] * n_dirs))()
    N.check(N.load().gs_candidate_poses(p.shape[0], p.ctypes.data_as(ctypes.c_void_p), int(n_dirs), int(width),
                                        int(height), float(f), float(f), float(near), arr), "gs_candidate_poses")
    cams = []
    for i in range(p.shape[0] * n_dirs):
        c = arr[i]
        cams.append(Camera(c.width, c.height, c.fx, c.fy, c.cx, c.cy, c.near_plane,
                           np.array(c.w2c[:], dtype=np.float32).reshape(3, 4)))
    return cams


def score_candidates(sums: torch.Tensor, npix: torch.Tensor, positions: torch.Tensor, current: torch.Tensor,
                     prune_frac: float = 0.005):
    """Eq. 6-8 on the device from the per-view sums of ``Rasterizer.candidates``
    (float64 [V, 3]): returns scores float64 [V, 4] = (I, I_geo, I_sem,
    1 - softmax(l)), keep int32 [V] (0: N_S below prune_frac of the view's
    pixels) and best int32 [1] (largest I among kept views, -1 if none).
    Stream-ordered: no host synchronisation."""
    dev = sums.device
    V = int(sums.shape[0])
    sums = sums.to(torch.float64).contiguous()
    npix = npix.to(device=dev, dtype=torch.int32).contiguous()
    positions = positions.to(device=dev, dtype=torch.float32).contiguous()
    current = current.to(device=dev, dtype=torch.float32).contiguous()
    scores = torch.empty((V, 4), dtype=torch.float64, device=dev)
    keep = torch.empty(V, dtype=torch.int32, device=dev)
    best = torch.empty(1, dtype=torch.int32, device=dev)
    N.check(N.load().gs_score_candidates(V, _ptr(sums), _ptr(npix), _ptr(positions), _ptr(current),
                                         float(prune_frac), _ptr(scores), _ptr(keep), _ptr(best),
                                         ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)),
            "gs_score_candidates")
    return scores, keep, best


def next_best_view(rast, g, cams: list[Camera], current_position, prune_frac: float = 0.005):
    """Renders the candidate views (one batched call) and scores them:
    returns (sums [V, 3], scores [V, 4], keep [V], best [1]) on the device."""
    sums = rast.candidates(g, cams)
    dev = sums.device
    npix = torch.tensor([c.width * c.height for c in cams], dtype=torch.int32, device=dev)
    pos = torch.tensor(np.stack([c.position() for c in cams]), dtype=torch.float32, device=dev)
    cur = torch.tensor(np.asarray(current_position, np.float32), device=dev)
    scores, keep, best = score_candidates(sums, npix, pos, cur, prune_frac)
    return sums, scores, keep, best


# ---------------------------------------------------------------------------
# sparse semantic representation (Sec. 3.1): top-k initialisation, updates
# ---------------------------------------------------------------------------

def topk_init(probs: torch.Tensor, k: int, rows: torch.Tensor | None = None):
    """Top-k (ids int32 [n, k], weights float32 [n, k]) of the observed class
    distributions: rows ``rows`` of ``probs`` [*, m] (all rows if None)."""
    m = int(probs.shape[-1])
    p = probs.reshape(-1, m).to(torch.float32).contiguous()
    r = None if rows is None else rows.to(device=p.device, dtype=torch.int64).contiguous()
    n = p.shape[0] if r is None else r.numel()
    ids = torch.empty((n, k), dtype=torch.int32, device=p.device)
    w = torch.empty((n, k), dtype=torch.float32, device=p.device)
    N.check(N.load().gs_topk_init(n, m, int(k), _ptr(p), _ptr(r), _ptr(ids), _ptr(w),
                                  ctypes.c_void_p(torch.cuda.current_stream(p.device).cuda_stream)), "gs_topk_init")
    return ids, w


def topk_gather(probs: torch.Tensor, ids: torch.Tensor, w: torch.Tensor, rows: torch.Tensor | None = None):
    """Updates w [n, k] in place with the observed probabilities at the fixed
    ids [n, k]."""
    m = int(probs.shape[-1])
    p = probs.reshape(-1, m).to(torch.float32).contiguous()
    r = None if rows is None else rows.to(device=p.device, dtype=torch.int64).contiguous()
    if not (w.is_contiguous() and w.dtype == torch.float32):
        raise ValueError("w must be a contiguous float32 tensor")
    N.check(N.load().gs_topk_gather(int(ids.shape[0]), m, int(ids.shape[1]), _ptr(p), _ptr(r),
                                    _ptr(ids.to(torch.int32).contiguous()), _ptr(w),
                                    ctypes.c_void_p(torch.cuda.current_stream(p.device).cuda_stream)),
            "gs_topk_gather")
    return w


# ---------------------------------------------------------------------------
# Exploration Map (Sec. 3.2): voxel occupancy from depth, newly freed voxels
# ---------------------------------------------------------------------------

class VoxelMap:
    """Voxel occupancy grid on the device (2 bits per voxel).  ``update``
    integrates one depth frame and returns the centres of the voxels it newly
    freed (device float32 [c, 3]) and their count."""

    def __init__(self, origin, voxel: float, dims, device=None):
        self.grid = N.GsVoxelGrid()
        for i in range(3):
            self.grid.origin[i] = float(origin[i])
        self.grid.voxel = float(voxel)
        self.grid.nx, self.grid.ny, self.grid.nz = (int(d) for d in dims)
        lib = N.load()
        words = lib.gs_voxel_words(ctypes.byref(self.grid))
        if words < 0:
            raise ValueError("invalid voxel grid")
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.state = torch.zeros(words, dtype=torch.int32, device=self.device)
        self.prev = torch.zeros_like(self.state)
        self.scratch = torch.empty(lib.gs_voxel_scratch_words(ctypes.byref(self.grid)), dtype=torch.int32,
                                   device=self.device)
        self.count = torch.zeros(1, dtype=torch.int32, device=self.device)

    def integrate(self, depth: torch.Tensor, cam: Camera, stride: int = 1, max_depth: float = 10.0):
        """Sets the free / occupied bits seen in one depth frame."""
        from .raster import cameras_array
        d = depth.to(torch.float32).contiguous()
        N.check(N.load().gs_voxel_update(ctypes.byref(self.grid), _ptr(self.state), _ptr(d), cameras_array([cam]),
                                         int(stride), float(max_depth),
                                         ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)),
                "gs_voxel_update")

    def new_free(self, capacity: int):
        """Centres of the voxels free now and unknown at the last snapshot
        (at most ``capacity`` written), and their total count (device)."""
        out = torch.empty((max(1, capacity), 3), dtype=torch.float32, device=self.device)
        N.check(N.load().gs_voxel_new_free(ctypes.byref(self.grid), _ptr(self.prev), _ptr(self.state),
                                           _ptr(self.scratch), _ptr(out), int(capacity), _ptr(self.count),
                                           ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)),
                "gs_voxel_new_free")
        return out, self.count

    def snapshot(self):
        self.prev.copy_(self.state)

    def update(self, depth: torch.Tensor, cam: Camera, stride: int = 1, max_depth: float = 10.0,
               capacity: int = 1 << 16):
        """snapshot, integrate, and the newly freed voxels."""
        self.snapshot()
        self.integrate(depth, cam, stride, max_depth)
        return self.new_free(capacity)

    def states(self) -> np.ndarray:
        """Per-voxel state [nz, ny, nx] uint8 on the host: 0 unknown, 1 free,
        2 occupied."""
        w = self.state.cpu().numpy().view(np.uint32)
        bits = (w[:, None] >> (2 * np.arange(16, dtype=np.uint32))[None, :]) & 3
        st = bits.reshape(-1)[: self.grid.nx * self.grid.ny * self.grid.nz]
        out = np.where(st & 2, 2, np.where(st & 1, 1, 0)).astype(np.uint8)
        return out.reshape(self.grid.nz, self.grid.ny, self.grid.nx)
