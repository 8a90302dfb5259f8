"""Where a frame's segments may leave Exploration-Map near ties, from the
geometry alone (test helper, no GPU).

The oracle (Sec. 3.2 Exploration Map) decides each (segment, voxel) pair
twice, with the voxel cube grown and shrunk by ovx.EPS edges, and reports
the voxels where the two disagree.  Such a disagreement needs the segment
to pass within EPS of the cube's boundary without crossing its inside by
more: near a segment end that lies within EPS of a face, or where the
segment crosses a face within EPS of one of its edges.  tie_cells marks
those places from the plane crossings of each segment (not from the
oracle's slab tests), with a 2 EPS margin; the tests require every oracle
tie to lie inside, which bounds the tie count by a size derived from the
rays rather than a measured rate."""
import math

import numpy as np

from oracle import voxel as ovx


def tie_cells(origin, vs, dims, depth, cam, stride=1, max_depth=10.0, tol=2 * ovx.EPS):
    """[nz, ny, nx] bool: the voxels where the segments of this frame may
    leave a near tie, from plane crossings (independent of the oracle's slab
    tests): the 27 cells around a segment end (camera centre or end point)
    within `tol` voxel of a face, and for every crossing of a voxel face
    within `tol` of one of its edges (or corners) the 4 (or 8) cells around
    that edge."""
    nx, ny, nz = dims
    cand = np.zeros((nz, ny, nx), bool)
    org = np.asarray(origin, np.float32).astype(np.float64)
    v = float(np.float32(vs))
    n = np.array([nx, ny, nz])

    def mark(cells):
        cells = np.asarray(cells, np.int64).reshape(-1, 3)
        cells = cells[np.all((cells >= 0) & (cells < n), axis=1)]
        cand[cells[:, 2], cells[:, 1], cells[:, 0]] = True

    off = np.stack(np.meshgrid([-1, 0, 1], [-1, 0, 1], [-1, 0, 1], indexing="ij"), -1).reshape(-1, 3)
    for o, p, _ in ovx.ray_points(depth, cam, stride, max_depth):
        a, b = (o - org) / v, (p - org) / v
        for e in (a, b):
            if np.any(np.abs(e - np.round(e)) < tol):
                mark(np.floor(e).astype(np.int64)[None] + off)
        for k in range(3):
            if b[k] == a[k]:
                continue
            lo, hi = sorted((a[k], b[k]))
            m = np.arange(math.floor(lo) + 1, math.ceil(hi))
            q = a[None] + ((m - a[k]) / (b[k] - a[k]))[:, None] * (b - a)[None]
            for r in range(len(m)):
                near = [j for j in range(3) if j != k and abs(q[r, j] - round(q[r, j])) < tol]
                if not near:
                    continue
                axes = [[int(m[r]) - 1, int(m[r])] if j == k else
                        [int(round(q[r, j])) - 1, int(round(q[r, j]))] if j in near else
                        [int(math.floor(q[r, j]))] for j in range(3)]
                mark(np.array(np.meshgrid(*axes, indexing="ij")).reshape(3, -1).T)
    return cand
