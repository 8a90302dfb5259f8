"""Seeded synthetic scenes and cameras for the rasterizer workloads.

This module only builds inputs: Gaussian parameters (means, linear scales,
quaternions, post-sigmoid opacities, colours, sparse top-k semantics,
per-Gaussian geometric uncertainty) and pinhole cameras.  It contains none
of the rasterizer's arithmetic (projection, binning, compositing, gradients);
both the CPU oracle and the CUDA path consume what it returns, unchanged.

All randomness comes from ``numpy.random.Generator(PCG64(seed))``.

Scene recipes (the paper's Replica/MP3D rooms rendered by Habitat are not
available; these stand in for them with the paper's image sizes, class
counts and a room-scale extent, Sec. 4.1 and the runtime analysis in the
supplement):

* ``scene_plain``: N Gaussians uniform in a 4x4x3 m box, log-scales
  N(-3, 0.5), random unit quaternions, opacity sigmoid(N(0,1)), RGB U[0,1],
  M classes with sparse top-k (ids without replacement, Dirichlet(1) weights
  sorted descending).
* ``scene_room``: rooms of 6x6x3 m; 70 % of the Gaussians on the six planar
  faces (area weighted, 1 m^2 patches with a base colour and a dominant
  class, thin along the face normal), 30 % in 24 object blobs.
* Cameras follow OpenCV axes (x right, y down, z forward) in a z-up world.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Camera", "Scene", "look_camera", "scene_plain", "scene_room", "scene_rooms",
    "perturbed_copy", "candidate_cameras_grid", "workload",
]


@dataclasses.dataclass
class Camera:
    """Pinhole camera: image size, intrinsics, near plane and a world-to-camera
    3x4 row-major [R|t] (float32)."""
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    near: float
    w2c: np.ndarray  # (3, 4) float32

    def position(self) -> np.ndarray:
        r = self.w2c[:, :3].astype(np.float64)
        t = self.w2c[:, 3].astype(np.float64)
        return -r.T @ t


@dataclasses.dataclass
class Scene:
    """Gaussian map in structure-of-arrays form (all float32 except sem_ids)."""
    means: np.ndarray      # (N, 3) world metres
    scales: np.ndarray     # (N, 3) linear scales (after exp)
    quats: np.ndarray      # (N, 4) (w, x, y, z), not necessarily unit
    opacity: np.ndarray    # (N,) in (0, 1) (after sigmoid)
    rgb: np.ndarray        # (N, 3)
    sem_ids: np.ndarray    # (N, k) int32 class ids in [0, m)
    sem_w: np.ndarray      # (N, k) float32 class probabilities
    m: int                 # number of classes (including "unknown")
    geo_unc: np.ndarray | None = None  # (N,) per-Gaussian scalar uncertainty

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @property
    def k(self) -> int:
        return int(self.sem_ids.shape[1])

    def subset(self, idx) -> "Scene":
        return Scene(self.means[idx].copy(), self.scales[idx].copy(), self.quats[idx].copy(),
                     self.opacity[idx].copy(), self.rgb[idx].copy(), self.sem_ids[idx].copy(),
                     self.sem_w[idx].copy(), self.m,
                     None if self.geo_unc is None else self.geo_unc[idx].copy())


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def look_camera(position, yaw_deg, width, height, f, near=0.2, pitch_deg=0.0) -> Camera:
    """Camera at ``position`` looking horizontally along yaw (degrees about
    world +z, 0 = +x).  Principal point at the image centre."""
    th = math.radians(yaw_deg)
    ph = math.radians(pitch_deg)
    fwd = np.array([math.cos(th) * math.cos(ph), math.sin(th) * math.cos(ph), math.sin(ph)])
    up = np.array([0.0, 0.0, 1.0])
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    r = np.stack([right, down, fwd], axis=0)        # rows: camera axes in world
    t = -r @ np.asarray(position, dtype=np.float64)
    w2c = np.concatenate([r, t[:, None]], axis=1)
    return Camera(int(width), int(height), float(np.float32(f)), float(np.float32(f)),
                  float(np.float32(width / 2.0)), float(np.float32(height / 2.0)),
                  float(np.float32(near)), _f32(w2c))


def _rand_quats(rng, n):
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _quat_from_matrix(r):
    """Unit quaternions (w,x,y,z) of a batch of proper rotation matrices
    (Shepperd's method, branch picked per element)."""
    m00, m11, m22 = r[:, 0, 0], r[:, 1, 1], r[:, 2, 2]
    tr = m00 + m11 + m22
    q = np.empty((r.shape[0], 4))
    c0 = tr > 0
    c1 = ~c0 & (m00 > m11) & (m00 > m22)
    c2 = ~c0 & ~c1 & (m11 > m22)
    c3 = ~c0 & ~c1 & ~c2
    with np.errstate(invalid="ignore", divide="ignore"):
        s = np.sqrt(np.maximum(tr + 1.0, 0.0)) * 2
        q[c0] = np.stack([0.25 * s, (r[:, 2, 1] - r[:, 1, 2]) / s, (r[:, 0, 2] - r[:, 2, 0]) / s,
                          (r[:, 1, 0] - r[:, 0, 1]) / s], axis=1)[c0]
        s = np.sqrt(np.maximum(1.0 + m00 - m11 - m22, 0.0)) * 2
        q[c1] = np.stack([(r[:, 2, 1] - r[:, 1, 2]) / s, 0.25 * s, (r[:, 0, 1] + r[:, 1, 0]) / s,
                          (r[:, 0, 2] + r[:, 2, 0]) / s], axis=1)[c1]
        s = np.sqrt(np.maximum(1.0 + m11 - m00 - m22, 0.0)) * 2
        q[c2] = np.stack([(r[:, 0, 2] - r[:, 2, 0]) / s, (r[:, 0, 1] + r[:, 1, 0]) / s, 0.25 * s,
                          (r[:, 1, 2] + r[:, 2, 1]) / s], axis=1)[c2]
        s = np.sqrt(np.maximum(1.0 + m22 - m00 - m11, 0.0)) * 2
        q[c3] = np.stack([(r[:, 1, 0] - r[:, 0, 1]) / s, (r[:, 0, 2] + r[:, 2, 0]) / s,
                          (r[:, 1, 2] + r[:, 2, 1]) / s, 0.25 * s], axis=1)[c3]
    return q


def _sparse_semantics(rng, n, m, k, dominant=None):
    """Top-k (id, weight) pairs: ids distinct, weights Dirichlet(1) sorted
    descending; when ``dominant`` is given it takes the first (largest) slot."""
    ids = np.empty((n, k), dtype=np.int64)
    ids[:, 0] = rng.integers(0, m, size=n) if dominant is None else dominant
    for j in range(1, k):
        col = rng.integers(0, m, size=n)
        while True:
            dup = np.zeros(n, dtype=bool)
            for jj in range(j):
                dup |= col == ids[:, jj]
            if not dup.any():
                break
            col[dup] = rng.integers(0, m, size=int(dup.sum()))
        ids[:, j] = col
    w = rng.dirichlet(np.ones(k), size=n)
    w = -np.sort(-w, axis=1)
    return np.ascontiguousarray(ids, dtype=np.int32), _f32(w)


def scene_plain(seed=0, n=10_000, m=16, k=3) -> Scene:
    """Uniform-box scene (plain forward workload, 10k Gaussians, 16 classes)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    means = rng.uniform([-2.0, -2.0, 0.0], [2.0, 2.0, 3.0], size=(n, 3))
    scales = np.exp(rng.normal(-3.0, 0.5, size=(n, 3)))
    quats = _rand_quats(rng, n)
    opacity = _sigmoid(rng.normal(0.0, 1.0, size=n))
    rgb = rng.uniform(0.0, 1.0, size=(n, 3))
    ids, w = _sparse_semantics(rng, n, m, k)
    return Scene(_f32(means), _f32(scales), _f32(quats), _f32(opacity), _f32(rgb), ids, w, m)


def _room_parts(rng, n, m, k, origin):
    """One 6x6x3 m room whose min corner is ``origin``."""
    ox, oy, oz = origin
    n_face = int(round(0.7 * n))
    n_blob = n - n_face
    # faces: (name, area, point(u,v), tangent1, tangent2, normal, extents)
    faces = [
        ("floor", 36.0, lambda a, b: (a * 6, b * 6, 0.0 * a), (1, 0, 0), (0, 1, 0), (0, 0, 1), (6, 6)),
        ("ceil", 36.0, lambda a, b: (a * 6, b * 6, 3.0 + 0.0 * a), (1, 0, 0), (0, -1, 0), (0, 0, -1), (6, 6)),
        ("wx0", 18.0, lambda a, b: (0.0 * a, a * 6, b * 3), (0, 1, 0), (0, 0, 1), (1, 0, 0), (6, 3)),
        ("wx1", 18.0, lambda a, b: (6.0 + 0.0 * a, a * 6, b * 3), (0, 1, 0), (0, 0, -1), (-1, 0, 0), (6, 3)),
        ("wy0", 18.0, lambda a, b: (a * 6, 0.0 * a, b * 3), (1, 0, 0), (0, 0, -1), (0, 1, 0), (6, 3)),
        ("wy1", 18.0, lambda a, b: (a * 6, 6.0 + 0.0 * a, b * 3), (1, 0, 0), (0, 0, 1), (0, -1, 0), (6, 3)),
    ]
    areas = np.array([f[1] for f in faces])
    face_of = rng.choice(len(faces), size=n_face, p=areas / areas.sum())
    means = np.empty((n, 3))
    log_s = np.empty((n, 3))
    quats = np.empty((n, 4))
    rgb = np.empty((n, 3))
    dominant = np.empty(n, dtype=np.int64)
    pos = 0
    for fi, (name, area, point, t1, t2, nrm, ext) in enumerate(faces):
        sel = np.nonzero(face_of == fi)[0]
        c = sel.size
        a = rng.uniform(0, 1, size=c)
        b = rng.uniform(0, 1, size=c)
        p = np.stack(point(a, b), axis=1).astype(np.float64)
        nrm_v = np.asarray(nrm, dtype=np.float64)
        p += rng.normal(0.0, 0.01, size=(c, 1)) * nrm_v[None, :]
        idx = np.arange(pos, pos + c)
        means[idx] = p + np.array([ox, oy, oz])
        log_s[idx, 0] = rng.normal(-3.5, 0.3, size=c)
        log_s[idx, 1] = rng.normal(-3.5, 0.3, size=c)
        log_s[idx, 2] = rng.normal(-6.0, 0.3, size=c)
        # scale frame: x,y in-plane (random in-plane angle), z along the normal
        ang = rng.uniform(0, 2 * math.pi, size=c)
        t1v = np.asarray(t1, dtype=np.float64)
        t2v = np.asarray(t2, dtype=np.float64)
        ex = np.cos(ang)[:, None] * t1v + np.sin(ang)[:, None] * t2v
        ey = -np.sin(ang)[:, None] * t1v + np.cos(ang)[:, None] * t2v
        ez = np.repeat(nrm_v[None, :], c, axis=0)
        # make a right-handed frame
        flip = np.einsum("ij,ij->i", np.cross(ex, ey), ez) < 0
        ey[flip] *= -1
        rot = np.stack([ex, ey, ez], axis=2)  # columns = local axes
        quats[idx] = _quat_from_matrix(rot)
        # 1 m^2 patches with a base colour and a dominant class
        pu = np.floor(a * ext[0]).astype(np.int64)
        pv = np.floor(b * ext[1]).astype(np.int64)
        npatch = ext[0] * ext[1]
        base = rng.uniform(0.1, 0.9, size=(npatch, 3))
        cls = rng.integers(0, m, size=npatch)
        pid = pu * ext[1] + pv
        rgb[idx] = base[pid] + rng.normal(0.0, 0.05, size=(c, 3))
        dominant[idx] = cls[pid]
        pos += c
    # object blobs
    centres = rng.uniform([0.5, 0.5, 0.0], [5.5, 5.5, 1.5], size=(24, 3))
    blob_rgb = rng.uniform(0.1, 0.9, size=(24, 3))
    blob_cls = rng.integers(0, m, size=24)
    which = rng.integers(0, 24, size=n_blob)
    idx = np.arange(pos, pos + n_blob)
    means[idx] = centres[which] + rng.normal(0.0, 0.25, size=(n_blob, 3)) + np.array([ox, oy, oz])
    log_s[idx] = rng.normal(-3.5, 0.5, size=(n_blob, 3))
    quats[idx] = _rand_quats(rng, n_blob)
    rgb[idx] = blob_rgb[which] + rng.normal(0.0, 0.05, size=(n_blob, 3))
    dominant[idx] = blob_cls[which]
    opacity = _sigmoid(rng.normal(1.0, 1.0, size=n))
    ids, w = _sparse_semantics(rng, n, m, k, dominant=dominant)
    return means, np.exp(log_s), quats, opacity, np.clip(rgb, 0.0, 1.0), ids, w


def scene_rooms(seed, n, m, k, layout=(1, 1), geo_unc=False) -> Scene:
    """``layout`` adjoining 6x6x3 m rooms (e.g. (2, 2) for four rooms), N total."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nr = layout[0] * layout[1]
    counts = [n // nr + (1 if i < n % nr else 0) for i in range(nr)]
    parts = []
    i = 0
    for ry in range(layout[1]):
        for rx in range(layout[0]):
            parts.append(_room_parts(rng, counts[i], m, k, (6.0 * rx, 6.0 * ry, 0.0)))
            i += 1
    cat = [np.concatenate([p[j] for p in parts], axis=0) for j in range(7)]
    perm = rng.permutation(n)  # gid order carries no spatial structure
    means, scales, quats, opacity, rgb, ids, w = [c[perm] for c in cat]
    unc = None
    if geo_unc:
        unc = _f32(rng.gamma(2.0, 0.5, size=n))
    return Scene(_f32(means), _f32(scales), _f32(quats), _f32(opacity), _f32(rgb),
                 np.ascontiguousarray(ids, dtype=np.int32), _f32(w), m, unc)


def scene_room(seed=1, n=300_000, m=102, k=3, geo_unc=False) -> Scene:
    """One 6x6x3 m synthetic room (mapping / candidate workloads)."""
    return scene_rooms(seed, n, m, k, (1, 1), geo_unc)


def perturbed_copy(scene: Scene, seed: int) -> Scene:
    """Target scene for the mapping loss: means +N(0,0.01), rgb +N(0,0.05)
    clipped to [0,1], opacity logits +N(0,0.3), sem weights +N(0,0.05)
    clipped at >= 0."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = scene.n
    means = scene.means + rng.normal(0.0, 0.01, size=(n, 3))
    rgb = np.clip(scene.rgb + rng.normal(0.0, 0.05, size=(n, 3)), 0.0, 1.0)
    o = np.clip(scene.opacity.astype(np.float64), 1e-6, 1 - 1e-6)
    logit = np.log(o / (1 - o)) + rng.normal(0.0, 0.3, size=n)
    w = np.maximum(scene.sem_w + rng.normal(0.0, 0.05, size=scene.sem_w.shape), 0.0)
    return Scene(_f32(means), scene.scales.copy(), scene.quats.copy(), _f32(_sigmoid(logit)),
                 _f32(rgb), scene.sem_ids.copy(), _f32(w), scene.m,
                 None if scene.geo_unc is None else scene.geo_unc.copy())


_RES = [(170, 300, 150.0), (340, 600, 300.0), (680, 1200, 600.0)]


def candidate_cameras_grid(xs, ys, z=1.5, yaws=(0, 60, 120, 180, 240, 300), res_of=None):
    """Candidate poses on a position grid x yaws.  ``res_of(v)`` picks the
    (H, W, f) of view v; default cycles 170x300 / 340x600 / 680x1200."""
    cams = []
    v = 0
    for x in xs:
        for y in ys:
            for yaw in yaws:
                h, w, f = (res_of(v) if res_of else _RES[v % 3])
                cams.append(look_camera((x, y, z), yaw, w, h, f))
                v += 1
    return cams


def dense_distributions(scene: Scene, seed: int, floor: float = 0.1) -> np.ndarray:
    """Full per-Gaussian class distributions [N, M] for the dense comparator:
    (1 - floor) times the Gaussian's top-k weights renormalised to sum 1,
    placed at their class ids, plus floor times a Dirichlet(1) draw over all
    M classes (every class gets some mass)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n, m = scene.n, scene.m
    dense = np.zeros((n, m), np.float64)
    w = scene.sem_w.astype(np.float64)
    w = w / np.maximum(w.sum(1, keepdims=True), 1e-12)
    np.add.at(dense, (np.repeat(np.arange(n), scene.k), scene.sem_ids.reshape(-1)), w.reshape(-1))
    dense = (1.0 - floor) * dense + floor * rng.dirichlet(np.ones(m), size=n)
    return _f32(dense)


def sparse_to_dense(scene: Scene) -> np.ndarray:
    """The scene's top-k (id, weight) entries scattered into [N, M] (zeros
    elsewhere)."""
    dense = np.zeros((scene.n, scene.m), np.float32)
    np.add.at(dense, (np.repeat(np.arange(scene.n), scene.k), scene.sem_ids.reshape(-1)),
              scene.sem_w.reshape(-1))
    return dense


def dense_as_sparse(scene: Scene, dense: np.ndarray) -> Scene:
    """The same Gaussians with k = M entries (id c, weight dense[:, c]): the
    dense representation written in the sparse one's form."""
    n, m = dense.shape
    ids = np.ascontiguousarray(np.broadcast_to(np.arange(m, dtype=np.int32), (n, m)))
    return Scene(scene.means, scene.scales, scene.quats, scene.opacity, scene.rgb, ids,
                 _f32(dense), m, scene.geo_unc)


def workload(name: str):
    """Named workloads.  Returns a dict with the scene(s) and camera(s).

    plain10k   : 10k Gaussians, 16 classes top-3, one 128x128 camera (f=110)
                 at the box centre looking along +x.
    room300k   : 300k-Gaussian room, 102 classes top-3, one 680x1200 view
                 (f=600) at (3,3,1.5) yaw 0, plus the perturbed target scene.
    cand96     : the 300k room with Gamma(2, 0.5) uncertainty and 96 candidate
                 poses (4x4 grid at 0.5 m, 6 yaws, resolutions cycling).
    rooms2m    : 2M Gaussians in 2x2 rooms, 256 classes top-8, 680x1200 view.
    mixed2m    : rooms2m + 128 candidate views (64 @170x300, 48 @340x600,
                 16 @680x1200) on a 0.5 m grid across the rooms, seeded shuffle.
    dense204k  : 290k-Gaussian room, 102 classes top-3, one 340x600 view (f=300)
                 from a corner, (0.4,0.4,1.5) yaw 45, in which about 204k
                 Gaussians are visible, plus full 102-class distributions per
                 Gaussian (the dense comparator's input).
    """
    if name == "plain10k":
        sc = scene_plain(0)
        cam = look_camera((0.0, 0.0, 1.5), 0.0, 128, 128, 110.0)
        return {"scene": sc, "cams": [cam]}
    if name == "room300k":
        sc = scene_room(1, 300_000, 102, 3)
        cam = look_camera((3.0, 3.0, 1.5), 0.0, 1200, 680, 600.0)
        return {"scene": sc, "cams": [cam], "target": perturbed_copy(sc, 101)}
    if name == "cand96":
        sc = scene_room(1, 300_000, 102, 3)
        rng = np.random.Generator(np.random.PCG64(2))
        sc.geo_unc = _f32(rng.gamma(2.0, 0.5, size=sc.n))
        g = [2.25, 2.75, 3.25, 3.75]
        return {"scene": sc, "cams": candidate_cameras_grid(g, g)}
    if name == "rooms2m":
        sc = scene_rooms(3, 2_000_000, 256, 8, (2, 2))
        cam = look_camera((3.0, 3.0, 1.5), 0.0, 1200, 680, 600.0)
        return {"scene": sc, "cams": [cam], "target": perturbed_copy(sc, 103)}
    if name == "mixed2m":
        base = workload("rooms2m")
        sc = base["scene"]
        rng = np.random.Generator(np.random.PCG64(4))
        sc.geo_unc = _f32(rng.gamma(2.0, 0.5, size=sc.n))
        grid = np.arange(0.75, 12.0, 0.5)
        poses = [(x, y, yaw) for x in grid for y in grid for yaw in (0, 60, 120, 180, 240, 300)
                 if abs(x - 6.0) > 0.3 and abs(y - 6.0) > 0.3]
        order = rng.permutation(len(poses))[:128]
        res = [_RES[0]] * 64 + [_RES[1]] * 48 + [_RES[2]] * 16
        cams = [look_camera((poses[i][0], poses[i][1], 1.5), poses[i][2], res[j][1], res[j][0], res[j][2])
                for j, i in enumerate(order)]
        return {"scene": sc, "cams": [base["cams"][0]], "target": base["target"], "cand_cams": cams}
    if name == "dense204k":
        sc = scene_room(6, 290_000, 102, 3)
        cam = look_camera((0.4, 0.4, 1.5), 45.0, 600, 340, 300.0)
        return {"scene": sc, "cams": [cam], "sem_dense": dense_distributions(sc, 7)}
    raise KeyError(name)
