"""CPU oracle for the semantic Gaussian rasterizer -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product library (the CUDA path behind the
C ABI) never imports, links or calls it, and this package imports nothing
from the product.

The arithmetic lives in ``gs_oracle.c`` (plain C, built twice: float for
decisions in the kernel's precision, double for finite-difference checks).
Binning (which tiles a Gaussian's pixel rectangle touches, and the
lexicographic (view, tile, depth, gid) order of Sec. 3.1's front-to-back
sort) is written here with numpy.

Parity status of each function (what pins it) is stated in its docstring.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_LIBS: dict[str, ctypes.CDLL] = {}

_P = ctypes.c_void_p
_I = ctypes.c_int


def _lib(prec: str) -> ctypes.CDLL:
    if prec not in _LIBS:
        path = _build.lib_path(prec)
        if not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_build.SRC):
            _build.build()
        _LIBS[prec] = ctypes.CDLL(path)
    return _LIBS[prec]


def _dt(prec):
    return np.float32 if prec == "f32" else np.float64


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_P)


def cam_array(cam, prec="f32") -> np.ndarray:
    """[fx, fy, cx, cy, near, w2c(12)] in the oracle's precision (the float32
    camera values widen exactly to double)."""
    v = [cam.fx, cam.fy, cam.cx, cam.cy, cam.near] + list(np.asarray(cam.w2c, np.float32).reshape(-1))
    return np.ascontiguousarray(np.asarray(v, dtype=np.float32).astype(_dt(prec)))


def _scene_arrays(scene, prec):
    d = _dt(prec)
    c = lambda a: None if a is None else np.ascontiguousarray(np.asarray(a).astype(d))
    return dict(means=c(scene.means), scales=c(scene.scales), quats=c(scene.quats), opacity=c(scene.opacity),
                rgb=c(scene.rgb), sem_w=c(scene.sem_w), unc=c(scene.geo_unc),
                sem_ids=np.ascontiguousarray(scene.sem_ids, dtype=np.int32))


def project(scene, cam, tile=(16, 16), prec="f32") -> dict:
    """Per-Gaussian projection: 2D mean, conic, depth, radius, pixel and tile
    rectangles, tile count and visibility.

    Pinned by tests against: a closed-form on-axis isotropic footprint; a
    numerically differentiated pinhole Jacobian (EWA linearisation) with
    numpy eigen-decomposition for the radius; a per-pixel brute-force
    rectangle rule."""
    lib = _lib(prec)
    n = scene.n
    a = _scene_arrays(scene, prec)
    d = _dt(prec)
    out = dict(uv=np.zeros((n, 2), d), conic=np.zeros((n, 3), d), depth=np.zeros(n, d), radius=np.zeros(n, d),
               rect=np.zeros((n, 4), np.int32), trect=np.zeros((n, 4), np.int32), ntiles=np.zeros(n, np.int32),
               visible=np.zeros(n, np.int32))
    fn = getattr(lib, f"orc_project_{prec}")
    fn.restype = None
    fn(_I(n), _ptr(a["means"]), _ptr(a["scales"]), _ptr(a["quats"]), _ptr(cam_array(cam, prec)),
       _I(cam.width), _I(cam.height), _I(tile[0]), _I(tile[1]), _ptr(out["uv"]), _ptr(out["conic"]),
       _ptr(out["depth"]), _ptr(out["radius"]), _ptr(out["rect"]), _ptr(out["trect"]), _ptr(out["ntiles"]),
       _ptr(out["visible"]))
    out["visible"] = out["visible"].astype(bool)
    return out


def tiles_of(cam, tile=(16, 16)):
    tw, th = tile
    return (cam.width + tw - 1) // tw, (cam.height + th - 1) // th


def tile_lists(projs, cams, tile=(16, 16)):
    """Binning reference: every visible (view, Gaussian) emits one pair per
    tile of its tile rectangle; pairs are ordered lexicographically by
    (view, tile, depth bits, gid).  Returns (ranges[T_total, 2], gids[K],
    tile_offset[V+1]) with tiles numbered row-major within each view and
    views concatenated.  A sort is a library step (np.lexsort)."""
    offs = [0]
    for cam in cams:
        gx, gy = tiles_of(cam, tile)
        offs.append(offs[-1] + gx * gy)
    tiles_l, depth_l, gid_l, view_l = [], [], [], []
    for v, (p, cam) in enumerate(zip(projs, cams)):
        gx, _ = tiles_of(cam, tile)
        vis = np.nonzero(p["visible"])[0]
        tr = p["trect"][vis]
        for g, (tx0, tx1, ty0, ty1) in zip(vis, tr):
            ty, tx = np.mgrid[ty0:ty1 + 1, tx0:tx1 + 1]
            t = (ty * gx + tx).reshape(-1) + offs[v]
            tiles_l.append(t)
            gid_l.append(np.full(t.size, g, np.int64))
            depth_l.append(np.full(t.size, np.float32(p["depth"][g]).view(np.uint32), np.uint64))
            view_l.append(np.full(t.size, v, np.int64))
    if tiles_l:
        tiles = np.concatenate(tiles_l)
        depth = np.concatenate(depth_l)
        gids = np.concatenate(gid_l)
    else:
        tiles = np.zeros(0, np.int64); depth = np.zeros(0, np.uint64); gids = np.zeros(0, np.int64)
    order = np.lexsort((gids, depth, tiles))
    tiles = tiles[order]
    gids = gids[order]
    total = offs[-1]
    start = np.searchsorted(tiles, np.arange(total), side="left")
    end = np.searchsorted(tiles, np.arange(total), side="right")
    return np.stack([start, end], axis=1).astype(np.int64), gids.astype(np.int64), np.asarray(offs, np.int64)


def render(scene, cam, prec="f32", sem=True, unc=False, rows=None) -> dict:
    """Full-image brute-force forward render (Eq. 1 for colour / depth /
    silhouette, Eq. 3 for the sparse semantic map; optional uncertainty
    channel composited as Eq. 1).  Also returns T_final, contributor counts,
    per-pixel near-threshold flags and stats (N_eval, N_contrib).

    Pinned by tests against: the closed-form isotropic footprint; the
    literal product form of Eq. 1 on tiny scenes; C = S for white Gaussians;
    sum_m P_m = S for weights summing to 1; Eq. 3 per class equal to Eq. 1
    with z_i = p_{i,m}."""
    lib = _lib(prec)
    a = _scene_arrays(scene, prec)
    d = _dt(prec)
    W, H, m = cam.width, cam.height, scene.m
    out = dict(rgb=np.zeros((H, W, 3), d), depth=np.zeros((H, W), d), sil=np.zeros((H, W), d),
               T=np.zeros((H, W), d), n_contrib=np.zeros((H, W), np.int32), n_eval_px=np.zeros((H, W), np.int32),
               flag=np.zeros((H, W), np.int32))
    out["sem"] = np.zeros((H, W, m), d) if sem else None
    out["unc"] = np.zeros((H, W), d) if (unc and scene.geo_unc is not None) else None
    stats = np.zeros(2, np.int64)
    fn = getattr(lib, f"orc_render_{prec}")
    fn.restype = None
    fn(_I(scene.n), _I(scene.k), _I(m), _ptr(a["means"]), _ptr(a["scales"]), _ptr(a["quats"]),
       _ptr(a["opacity"]), _ptr(a["rgb"]), _ptr(a["sem_ids"]), _ptr(a["sem_w"]),
       _ptr(a["unc"]) if out["unc"] is not None else None, _ptr(cam_array(cam, prec)), _I(W), _I(H),
       _ptr(out["rgb"]), _ptr(out["depth"]), _ptr(out["sil"]), _ptr(out["unc"]), _ptr(out["sem"]),
       _ptr(out["T"]), _ptr(out["n_contrib"]), _ptr(out["n_eval_px"]), _ptr(out["flag"]), _ptr(stats),
       *_rows(rows, H))
    out["n_eval"], out["n_contrib_total"] = int(stats[0]), int(stats[1])
    return out


def render_pixels(scene, cam, xs, ys, prec="f32", sem=True) -> dict:
    """Forward render of selected pixels only (same arithmetic as render)."""
    lib = _lib(prec)
    a = _scene_arrays(scene, prec)
    d = _dt(prec)
    xs = np.ascontiguousarray(xs, np.int32)
    ys = np.ascontiguousarray(ys, np.int32)
    npx = xs.size
    m = scene.m
    out = dict(rgb=np.zeros((npx, 3), d), depth=np.zeros(npx, d), sil=np.zeros(npx, d), T=np.zeros(npx, d),
               n_contrib=np.zeros(npx, np.int32), flag=np.zeros(npx, np.int32))
    out["sem"] = np.zeros((npx, m), d) if sem else None
    out["unc"] = np.zeros(npx, d) if scene.geo_unc is not None else None
    fn = getattr(lib, f"orc_render_pixels_{prec}")
    fn.restype = None
    fn(_I(scene.n), _I(scene.k), _I(m), _ptr(a["means"]), _ptr(a["scales"]), _ptr(a["quats"]),
       _ptr(a["opacity"]), _ptr(a["rgb"]), _ptr(a["sem_ids"]), _ptr(a["sem_w"]), _ptr(a["unc"]),
       _ptr(cam_array(cam, prec)), _I(cam.width), _I(cam.height), _I(npx), _ptr(xs), _ptr(ys),
       _ptr(out["rgb"]), _ptr(out["depth"]), _ptr(out["sil"]), _ptr(out["unc"]), _ptr(out["sem"]),
       _ptr(out["T"]), _ptr(out["n_contrib"]), _ptr(out["flag"]))
    return out


def _rows(rows, H):
    """(y_begin, y_end, y_step) of a row sample; None = every row."""
    if rows is None:
        return _I(0), _I(H), _I(1)
    b, e, s = rows
    return _I(b), _I(e), _I(s)


def render_bwd(scene, cam, d_rgb=None, d_depth=None, d_sil=None, d_sem=None, sem_detach=True,
               prec="f64", rows=None) -> dict:
    """Hand-derived adjoint of render(): gradients of sum(d_out * out) w.r.t.
    means, scales, quats, opacity, rgb and sem_w.  With sem_detach the
    semantic upstream gradient reaches sem_w only (Sec. 3.1, semantic loss
    restricted to semantic attributes).

    Pinned by tests against central finite differences of render() in
    double precision, and by the semantic-block invariance."""
    lib = _lib(prec)
    a = _scene_arrays(scene, prec)
    d = _dt(prec)
    n, k = scene.n, scene.k
    c = lambda x: None if x is None else np.ascontiguousarray(np.asarray(x).astype(d))
    g = dict(means=np.zeros((n, 3), d), scales=np.zeros((n, 3), d), quats=np.zeros((n, 4), d),
             opacity=np.zeros(n, d), rgb=np.zeros((n, 3), d), sem_w=np.zeros((n, k), d))
    ups = [c(d_rgb), c(d_depth), c(d_sil), c(d_sem)]
    fn = getattr(lib, f"orc_render_bwd_{prec}")
    fn.restype = None
    fn(_I(n), _I(k), _I(scene.m), _ptr(a["means"]), _ptr(a["scales"]), _ptr(a["quats"]), _ptr(a["opacity"]),
       _ptr(a["rgb"]), _ptr(a["sem_ids"]), _ptr(a["sem_w"]), _ptr(cam_array(cam, prec)), _I(cam.width),
       _I(cam.height), _ptr(ups[0]), _ptr(ups[1]), _ptr(ups[2]), _ptr(ups[3]), _I(1 if sem_detach else 0),
       _ptr(g["means"]), _ptr(g["scales"]), _ptr(g["quats"]), _ptr(g["opacity"]), _ptr(g["rgb"]),
       _ptr(g["sem_w"]), *_rows(rows, cam.height))
    return g


def candidate(scene, cam, prec="f32"):
    """Per-view candidate reductions: (sum_p U(p), sum_p H(p), N_S, n_flag),
    H the entropy (Eq. 4) of the semantic map clipped to [0.001, 1] and
    renormalised (Eq. 7), N_S the count of pixels with S(p) = 0 (Eq. 6).

    Pinned by tests against: the empty view (H = ln M per pixel, N_S = all
    pixels, U = 0); a fully covered view with one class (closed form); U = S
    when every u_i = 1."""
    lib = _lib(prec)
    a = _scene_arrays(scene, prec)
    out = np.zeros(3, np.float64)
    nflag = ctypes.c_long(0)
    fn = getattr(lib, f"orc_candidate_{prec}")
    fn.restype = None
    fn(_I(scene.n), _I(scene.k), _I(scene.m), _ptr(a["means"]), _ptr(a["scales"]), _ptr(a["quats"]),
       _ptr(a["opacity"]), _ptr(a["rgb"]), _ptr(a["sem_ids"]), _ptr(a["sem_w"]), _ptr(a["unc"]),
       _ptr(cam_array(cam, prec)), _I(cam.width), _I(cam.height), _ptr(out), ctypes.byref(nflag))
    return float(out[0]), float(out[1]), int(out[2]), int(nflag.value)
