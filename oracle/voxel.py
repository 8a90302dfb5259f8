"""Exploration Map of Sec. 3.2 (voxel occupancy from depth) -- TEST
INFRASTRUCTURE (same rules as the rest of ``oracle``).

Brute force from the definition, in float64: for each sampled pixel the
back-projected point p = R^T (((u + 1/2 - cx) d / fx, (v + 1/2 - cy) d / fy, d) - t)
and the camera centre o = -R^T t; every grid voxel whose closed cube meets
the segment [o, p] is free, except the voxel holding p, which is occupied
(when the depth is at most max_depth; deeper points are cut at max_depth
and mark nothing occupied).  Each (ray, voxel) decision is taken twice,
with the cube grown and shrunk by EPS voxel edges; where the two disagree
the voxel is a near tie (the segment grazes an edge or corner, or p lies on
a face) and is reported as such rather than decided.

Readings where the paper is silent: depth is the
camera-space z of the rendered depth map; a voxel seen both free and
occupied is occupied; the newly freed voxels of an update are those free
now and unknown before.

Parity: pinned by closed forms (an axis-aligned ray, a ray entering the grid
from outside, the max_depth cut, invalid depths) and by dense sampling of
the segment (tests/test_oracle_pins.py).
"""
from __future__ import annotations

import math

import numpy as np

EPS = 1e-3  # voxel edges


def _cam_centre_and_rot(cam):
    w = np.asarray(cam.w2c, np.float32).astype(np.float64).reshape(3, 4)
    r, t = w[:, :3], w[:, 3]
    return -r.T @ t, r


def ray_points(depth, cam, stride, max_depth):
    """[(o, p, hit)] of the sampled pixels with a positive finite depth."""
    o, r = _cam_centre_and_rot(cam)
    out = []
    H, W = np.asarray(depth).shape
    for v in range(0, H, stride):
        for u in range(0, W, stride):
            d = float(np.float32(depth[v, u]))
            if not (d > 0.0) or not math.isfinite(d):
                continue
            hit = d <= float(np.float32(max_depth))
            de = d if hit else float(np.float32(max_depth))
            xc = (u + 0.5 - float(np.float32(cam.cx))) / float(np.float32(cam.fx)) * de
            yc = (v + 0.5 - float(np.float32(cam.cy))) / float(np.float32(cam.fy)) * de
            p = r.T @ np.array([xc, yc, de]) + o
            out.append((o, p, hit))
    return out


def _meets(a, b, lo, hi):
    """[n] bool: the segment a -> b meets the boxes [lo, hi] ([n, 3] each)."""
    d = b - a
    t0 = np.zeros(lo.shape[0])
    t1 = np.ones(lo.shape[0])
    ok = np.ones(lo.shape[0], bool)
    for k in range(3):
        if d[k] == 0.0:
            ok &= (a[k] >= lo[:, k]) & (a[k] <= hi[:, k])
        else:
            ta = (lo[:, k] - a[k]) / d[k]
            tb = (hi[:, k] - a[k]) / d[k]
            t0 = np.maximum(t0, np.minimum(ta, tb))
            t1 = np.minimum(t1, np.maximum(ta, tb))
    return ok & (t0 <= t1)


def integrate(origin, voxel, dims, depth, cam, stride=1, max_depth=10.0):
    """Per-voxel bits seen in one frame, as two [nz, ny, nx] uint8 arrays:
    `sure` (bit 1 free, bit 2 occupied: decided) and `maybe` (the same bits,
    decided or near tie).  A correct implementation's bits lie between the
    two."""
    nx, ny, nz = dims
    n = np.array([nx, ny, nz])
    org = np.asarray(origin, np.float32).astype(np.float64)
    vs = float(np.float32(voxel))
    sure = np.zeros((nz, ny, nx), np.uint8)
    maybe = np.zeros((nz, ny, nx), np.uint8)
    for o, p, hit in ray_points(depth, cam, stride, max_depth):
        a = (o - org) / vs
        b = (p - org) / vs
        end_in = hit and bool(np.all(b >= 0) and np.all(b < n))
        end = np.floor(b).astype(np.int64)
        end_tie = hit and bool(np.any(np.abs(b - np.round(b)) < EPS)) and bool(np.all(b > -EPS)) and \
            bool(np.all(b < n + EPS))
        # cells to test: the 3x3x3 neighbourhoods of points sampled along the
        # segment every 1/4 voxel (a cube the segment meets holds a segment
        # point within 1/8 voxel of a sample, so it lies in that sample's
        # neighbourhood); each is then decided by the slab test below
        ns = max(2, int(math.ceil(np.abs(b - a).max() * 4.0)) + 1)
        smp = np.floor(a[None] + np.linspace(0.0, 1.0, ns)[:, None] * (b - a)[None]).astype(np.int64)
        off = np.stack(np.meshgrid([-1, 0, 1], [-1, 0, 1], [-1, 0, 1], indexing="ij"), -1).reshape(-1, 3)
        cells = np.unique((smp[:, None, :] + off[None]).reshape(-1, 3), axis=0)
        cells = cells[np.all((cells >= 0) & (cells < n), axis=1)]
        lo = cells.astype(np.float64)
        in_sure = _meets(a, b, lo + EPS, lo + 1.0 - EPS)
        in_maybe = _meets(a, b, lo - EPS, lo + 1.0 + EPS)
        is_end = np.all(cells == end, axis=1) if end_in else np.zeros(len(cells), bool)
        # a point within EPS of a face leaves the cells around it undecided
        near_end = np.all(np.abs(cells - end) <= 1, axis=1) if end_tie else np.zeros(len(cells), bool)
        fs = in_sure & ~is_end & ~near_end
        fm = in_maybe & ~is_end
        np.bitwise_or.at(sure, (cells[fs, 2], cells[fs, 1], cells[fs, 0]), 1)
        np.bitwise_or.at(maybe, (cells[fm, 2], cells[fm, 1], cells[fm, 0]), 1)
        if end_in and not end_tie:
            sure[end[2], end[1], end[0]] |= 2
            maybe[end[2], end[1], end[0]] |= 2
        elif end_tie:
            # the holding voxel is one of the cells around p: any of them may
            # be marked occupied (or, not being the end voxel, free)
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dz in (-1, 0, 1):
                        q = np.floor(b + np.array([dx, dy, dz]) * EPS * 2).astype(np.int64)
                        if np.all(q >= 0) and np.all(q < n):
                            maybe[q[2], q[1], q[0]] |= 3
    return sure, maybe


def state_of(bits: np.ndarray) -> np.ndarray:
    """0 unknown, 1 free, 2 occupied (occupied wins)."""
    return np.where(bits & 2, 2, np.where(bits & 1, 1, 0)).astype(np.uint8)


def new_free(prev_bits: np.ndarray, cur_bits: np.ndarray, origin, voxel) -> np.ndarray:
    """Centres [c, 3] (ascending linear index (z ny + y) nx + x) of voxels
    free in cur and unknown in prev."""
    cur, prev = state_of(cur_bits), state_of(prev_bits)
    z, y, x = np.nonzero((cur == 1) & (prev == 0))
    org = np.asarray(origin, np.float64)
    return np.stack([org[0] + (x + 0.5) * voxel, org[1] + (y + 0.5) * voxel, org[2] + (z + 0.5) * voxel], axis=1)
