"""PyTorch-facing layer over the C ABI.

PyTorch supplies device memory, the current CUDA stream and autograd; every
step of the rasterizer runs in the native library (``libgs.so``).  This
module only marshals tensors into the C structs of ``include/gs.h``.
"""
from __future__ import annotations

import ctypes
import dataclasses

import numpy as np
import torch

from . import _native as N


# ---------------------------------------------------------------------------
# scene / camera marshalling
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Gaussians:
    """Device-resident Gaussian map (Sec. 3.1): structure of arrays."""
    means: torch.Tensor     # (n,3) float32
    scales: torch.Tensor    # (n,3) float32, linear
    quats: torch.Tensor     # (n,4) float32, (w,x,y,z)
    opacity: torch.Tensor   # (n,)  float32 in (0,1)
    rgb: torch.Tensor       # (n,3) float32
    sem_ids: torch.Tensor   # (n,k) int32
    sem_w: torch.Tensor     # (n,k) float32
    m: int
    geo_unc: torch.Tensor | None = None

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @property
    def k(self) -> int:
        return int(self.sem_ids.shape[1])

    @staticmethod
    def from_scene(scene, device="cuda") -> "Gaussians":
        f = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(device)
        return Gaussians(f(scene.means), f(scene.scales), f(scene.quats), f(scene.opacity), f(scene.rgb),
                         torch.from_numpy(np.ascontiguousarray(scene.sem_ids, dtype=np.int32)).to(device),
                         f(scene.sem_w), int(scene.m), None if scene.geo_unc is None else f(scene.geo_unc))


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("tensors passed to the rasterizer must be contiguous CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


def _f32(t):
    if t is None:
        return None
    if t.dtype != torch.float32:
        raise TypeError(f"expected float32, got {t.dtype}")
    return t.contiguous()


def scene_struct(means, scales, quats, opacity, rgb, sem_ids, sem_w, m, geo_unc=None) -> N.GsScene:
    s = N.GsScene()
    s.n = int(means.shape[0])
    s.k = int(sem_ids.shape[1])
    s.m = int(m)
    s.means, s.scales, s.quats, s.opacity = _ptr(means), _ptr(scales), _ptr(quats), _ptr(opacity)
    s.rgb, s.sem_ids, s.sem_w = _ptr(rgb), _ptr(sem_ids), _ptr(sem_w)
    s.geo_unc = _ptr(geo_unc)
    return s


def camera_struct(cam) -> N.GsCamera:
    c = N.GsCamera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy, c.near_plane = cam.fx, cam.fy, cam.cx, cam.cy, cam.near
    w = np.asarray(cam.w2c, dtype=np.float32).reshape(-1)
    for i in range(12):
        c.w2c[i] = float(w[i])
    return c


def cameras_array(cams):
    arr = (N.GsCamera * len(cams))()
    for i, cam in enumerate(cams):
        arr[i] = camera_struct(cam)
    return arr


def zero_grads(g: "Gaussians") -> dict:
    """Zeroed gradient buffers for every parameter of ``g``, as views of one
    allocation (one fill instead of six; quaternions first, so every view
    starts 16-byte aligned for its row size)."""
    shapes = dict(quats=tuple(g.quats.shape), means=tuple(g.means.shape), scales=tuple(g.scales.shape),
                  rgb=tuple(g.rgb.shape), sem_w=tuple(g.sem_w.shape), opacity=tuple(g.opacity.shape))
    sizes = {k: int(np.prod(v)) for k, v in shapes.items()}
    flat = torch.zeros(sum(sizes.values()), dtype=torch.float32, device=g.means.device)
    out, off = {}, 0
    for k, shp in shapes.items():
        out[k] = flat[off:off + sizes[k]].view(shp)
        off += sizes[k]
    return {k: out[k] for k in ("means", "scales", "quats", "opacity", "rgb", "sem_w")}


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


# ---------------------------------------------------------------------------
# rasterizer: owns a workspace
# ---------------------------------------------------------------------------

def largest_group(cams, budget: int) -> int:
    """Views in the largest group of a candidate call whose views are
    grouped by `budget` pixels (gs_config.cand_group_pixels: consecutive
    views while their pixels fit, at least one; budget <= 0: one group)."""
    if budget <= 0:
        return len(cams)
    best = n = px = 0
    for c in cams:
        p = c.width * c.height
        if n and px + p > budget:
            n = px = 0
        n, px = n + 1, px + p
        best = max(best, n)
    return best


class Rasterizer:
    """Owns one device workspace and a launch configuration.

    ``recompute_bwd=True`` keeps no per-pixel contributor bits: the semantic
    pass and the adjoint re-test each tile's pairs (less memory, same
    results).

    ``check=True`` calls read the device counters after binning (a host
    synchronisation) and grow the pair capacity and rerun when the workspace
    overflowed; ``check=False`` never synchronises (use after warm-up, e.g.
    inside CUDA-graph capture) and leaves the status for ``counters()``.
    """

    def __init__(self, tile=(16, 16), sem_detach_geometry=True, record_capacity=0, pair_capacity=0,
                 device=None, px_per_thread=0, recompute_bwd=False, spin_limit=0, cand_batch=0,
                 cand_bits_bytes=0, cand_group_pixels=0):
        self.tile = tuple(tile)
        self.cand_batch = int(cand_batch)            # Gaussians per staged batch of the candidate kernels (0: 64)
        self.cand_bits_bytes = int(cand_bits_bytes)  # contributor-bit budget of candidate calls (0: 4 GiB)
        self.cand_group_pixels = int(cand_group_pixels)  # pixels of a candidate view group (0: all views at once)
        self.recompute_bwd = bool(recompute_bwd)
        self.spin_limit = int(spin_limit)  # 0: the library's bound on inter-CTA waits
        self.px_per_thread = int(px_per_thread)
        self.sem_detach_geometry = bool(sem_detach_geometry)
        self.record_capacity = int(record_capacity)
        self.pair_capacity = int(pair_capacity)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.ws: torch.Tensor | None = None
        self._shrink_ws = False  # re-allocate the workspace at its fitted size on the next call
        self.generation = 0
        # optional list collecting (name, cuda.Event) at phase boundaries
        self.phase_events: list | None = None
        self._last = None  # (scene_struct, cams_arr, n_views, cfg) of the last projection
        N.load()

    def _mark(self, name: str):
        if self.phase_events is not None:
            ev = torch.cuda.Event(enable_timing=True)
            ev.record()
            self.phase_events.append((name, ev))

    def config(self, n_gauss: int, n_views: int) -> N.GsConfig:
        c = N.GsConfig()
        c.tile_w, c.tile_h = self.tile
        c.sem_detach_geometry = 1 if self.sem_detach_geometry else 0
        c.px_per_thread = self.px_per_thread
        c.recompute_bwd = 1 if self.recompute_bwd else 0
        c.spin_limit = self.spin_limit
        c.cand_batch = self.cand_batch
        c.cand_bits_bytes = self.cand_bits_bytes
        c.cand_group_pixels = self.cand_group_pixels
        # capacities start at a bound that never overflows for small problems
        # and grow on reported overflow (check=True)
        c.record_capacity = self.record_capacity if self.record_capacity > 0 else max(1, min(n_gauss * n_views,
                                                                                              1 << 26))
        c.pair_capacity = self.pair_capacity if self.pair_capacity > 0 else max(1 << 20, min(8 * c.record_capacity,
                                                                                            1 << 30))
        c.pair_capacity = min(c.pair_capacity, (1 << 31) - 1)
        return c

    def _ensure_ws(self, sc, cams_arr, n_views, cfg):
        need = N.load().gs_workspace_size(ctypes.byref(sc), cams_arr, n_views, ctypes.byref(cfg))
        if need == 0:
            raise ValueError("invalid scene / camera / config for the rasterizer")
        if self.ws is None or self.ws.numel() < need or (self._shrink_ws and self.ws.numel() > need + need // 8):
            self.ws = None
            self.ws = torch.empty(int(need), dtype=torch.uint8, device=self.device)
        self._shrink_ws = False
        return ctypes.c_void_p(self.ws.data_ptr())

    def counters(self) -> N.GsCounters:
        c = N.GsCounters()
        N.load().gs_read_counters(ctypes.c_void_p(self.ws.data_ptr()), ctypes.byref(c), _stream())
        return c

    def _project_bin(self, g: Gaussians, cams, check: bool):
        lib = N.load()
        sc = scene_struct(g.means, g.scales, g.quats, g.opacity, g.rgb, g.sem_ids, g.sem_w, g.m, g.geo_unc)
        cams_arr = cameras_array(cams)
        V = len(cams)
        for _ in range(8):
            cfg = self.config(g.n, V)
            ws = self._ensure_ws(sc, cams_arr, V, cfg)
            N.check(lib.gs_project(ctypes.byref(sc), cams_arr, V, ctypes.byref(cfg), ws, _stream()), "gs_project")
            N.check(lib.gs_bin_sort(ctypes.byref(sc), cams_arr, V, ctypes.byref(cfg), ws, _stream()), "gs_bin_sort")
            if not check:
                break
            cnt = N.GsCounters()
            st = lib.gs_read_counters(ws, ctypes.byref(cnt), _stream())
            if st == N.GS_OK:
                break
            if st != N.GS_ERR_CAPACITY:
                N.check(st, "gs_bin_sort (device status)")
            if cnt.n_records > cfg.record_capacity:
                self.record_capacity = int(cnt.n_records * 1.1) + 1024
            if cnt.n_pairs > cfg.pair_capacity:
                self.pair_capacity = int(cnt.n_pairs * 1.25) + 4096
        self._last = (sc, cams_arr, V, cfg)
        return sc, cams_arr, cfg, ws

    # -- single view --------------------------------------------------------
    def forward(self, g: Gaussians, cam, want_sem=True, check=True):
        """Project, bin and render one view.  Returns rgb [H,W,3], depth
        [H,W], sil [H,W], sem [H,W,m] (or None)."""
        self._mark("project")
        sc, cams_arr, cfg, ws = self._project_bin(g, [cam], check)
        self._mark("render_fwd")
        H, W = cam.height, cam.width
        dev = self.device
        rgb = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
        depth = torch.empty((H, W), dtype=torch.float32, device=dev)
        sil = torch.empty((H, W), dtype=torch.float32, device=dev)
        sem = torch.empty((H, W, g.m), dtype=torch.float32, device=dev) if want_sem else None
        N.check(N.load().gs_render_fwd(ctypes.byref(sc), cams_arr, ctypes.byref(cfg), ws, _ptr(rgb), _ptr(depth),
                                       _ptr(sil), _ptr(sem), _stream()), "gs_render_fwd")
        self._mark("fwd_end")
        self.generation += 1
        return rgb, depth, sil, sem

    def forward_dense(self, g: Gaussians, cam, sem_dense: torch.Tensor, check=True):
        """Dense-semantic comparator: project, bin and render one view with
        every Gaussian carrying all m class probabilities (``sem_dense``
        [n, m] float32 on the device).  Returns rgb, depth, sil, sem."""
        self._mark("project")
        sc, cams_arr, cfg, ws = self._project_bin(g, [cam], check)
        self._mark("render_fwd")
        H, W = cam.height, cam.width
        dev = self.device
        rgb = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
        depth = torch.empty((H, W), dtype=torch.float32, device=dev)
        sil = torch.empty((H, W), dtype=torch.float32, device=dev)
        sem = torch.empty((H, W, g.m), dtype=torch.float32, device=dev)
        dense = _f32(sem_dense)
        if tuple(dense.shape) != (g.n, g.m):
            raise ValueError(f"sem_dense must be [{g.n}, {g.m}], got {tuple(dense.shape)}")
        N.check(N.load().gs_render_fwd_dense(ctypes.byref(sc), cams_arr, ctypes.byref(cfg), ws, _ptr(dense),
                                             _ptr(rgb), _ptr(depth), _ptr(sil), _ptr(sem), _stream()),
                "gs_render_fwd_dense")
        self._mark("fwd_end")
        self.generation += 1
        return rgb, depth, sil, sem

    def backward(self, g: Gaussians, cam, d_rgb=None, d_depth=None, d_sil=None, d_sem=None, grads=None):
        """Adjoint of the last forward.  Returns (or accumulates into) a dict of
        gradients for means, scales, quats, opacity, rgb, sem_w."""
        if self._last is None:
            raise RuntimeError("backward before forward")
        sc, cams_arr, V, cfg = self._last
        if grads is None:
            grads = zero_grads(g)
        ws = ctypes.c_void_p(self.ws.data_ptr())
        self._mark("render_bwd")
        N.check(N.load().gs_render_bwd(ctypes.byref(sc), cams_arr, ctypes.byref(cfg), ws, _ptr(_f32(d_rgb)),
                                       _ptr(_f32(d_depth)), _ptr(_f32(d_sil)), _ptr(_f32(d_sem)),
                                       _ptr(grads["means"]), _ptr(grads["scales"]), _ptr(grads["quats"]),
                                       _ptr(grads["opacity"]), _ptr(grads["rgb"]), _ptr(grads["sem_w"]),
                                       _stream()), "gs_render_bwd")
        self._mark("bwd_end")
        return grads

    def forward_l1(self, g: Gaussians, cam, t_rgb, t_depth, t_sem=None, check=True, outputs=False):
        """Project, bin, render and compare with the targets in one pass
        (fused mean-L1).  Returns the loss (0-dim device tensor) and, when
        ``outputs``, (rgb, depth, sil, sem) as well."""
        self._mark("project")
        sc, cams_arr, cfg, ws = self._project_bin(g, [cam], check)
        self._mark("render_fwd")
        H, W = cam.height, cam.width
        dev = self.device
        loss = torch.empty((), dtype=torch.float32, device=dev)
        outs = (None, None, None, None)
        if outputs:
            outs = (torch.empty((H, W, 3), dtype=torch.float32, device=dev),
                    torch.empty((H, W), dtype=torch.float32, device=dev),
                    torch.empty((H, W), dtype=torch.float32, device=dev),
                    torch.empty((H, W, g.m), dtype=torch.float32, device=dev))
        N.check(N.load().gs_render_fwd_l1(ctypes.byref(sc), cams_arr, ctypes.byref(cfg), ws, _ptr(_f32(t_rgb)),
                                          _ptr(_f32(t_depth)), _ptr(_f32(t_sem)), *[_ptr(o) for o in outs],
                                          _ptr(loss), _stream()), "gs_render_fwd_l1")
        self._mark("fwd_end")
        self.generation += 1
        return (loss, outs) if outputs else loss

    def backward_l1(self, g: Gaussians, cam, loss_scale: torch.Tensor, grads=None):
        """Adjoint of the last forward_l1, scaled by the device scalar
        ``loss_scale`` (dL/dloss)."""
        if self._last is None:
            raise RuntimeError("backward before forward")
        sc, cams_arr, V, cfg = self._last
        if grads is None:
            grads = zero_grads(g)
        ws = ctypes.c_void_p(self.ws.data_ptr())
        ls = loss_scale.to(torch.float32).contiguous()
        self._mark("render_bwd")
        N.check(N.load().gs_render_bwd_l1(ctypes.byref(sc), cams_arr, ctypes.byref(cfg), ws, _ptr(ls),
                                          _ptr(grads["means"]), _ptr(grads["scales"]), _ptr(grads["quats"]),
                                          _ptr(grads["opacity"]), _ptr(grads["rgb"]), _ptr(grads["sem_w"]),
                                          _stream()), "gs_render_bwd_l1")
        self._mark("bwd_end")
        return grads

    def forward_objective(self, g: Gaussians, cam, t_rgb, t_depth, t_sem=None, check=True, outputs=False):
        """Project, bin, render and evaluate the Sec. 3.1 mapping objective
        (silhouette-masked depth / colour L1 sum + mean entropy-masked
        Hellinger + cosine semantic term) inside the render passes.  Returns
        the loss (0-dim device tensor) and, when ``outputs``, (rgb, depth,
        sil) as well.  Raises GsError(GS_ERR_UNSUPPORTED) when the
        configuration has no fused form (semantics not detached from the
        geometry, the recompute mode, or too many classes for one tile
        accumulator)."""
        self._mark("project")
        sc, cams_arr, cfg, ws = self._project_bin(g, [cam], check)
        self._mark("render_fwd")
        H, W = cam.height, cam.width
        dev = self.device
        loss = torch.empty((), dtype=torch.float32, device=dev)
        outs = (None, None, None)
        if outputs:
            outs = (torch.empty((H, W, 3), dtype=torch.float32, device=dev),
                    torch.empty((H, W), dtype=torch.float32, device=dev),
                    torch.empty((H, W), dtype=torch.float32, device=dev))
        N.check(N.load().gs_render_fwd_objective(ctypes.byref(sc), cams_arr, ctypes.byref(cfg), ws,
                                                 _ptr(_f32(t_rgb)), _ptr(_f32(t_depth)), _ptr(_f32(t_sem)),
                                                 *[_ptr(o) for o in outs], _ptr(loss), _stream()),
                "gs_render_fwd_objective")
        self._mark("fwd_end")
        self.generation += 1
        return (loss, outs) if outputs else loss

    def backward_objective(self, g: Gaussians, cam, loss_scale: torch.Tensor, grads=None):
        """Adjoint of the last forward_objective, scaled by the device scalar
        ``loss_scale`` (dL/dloss)."""
        if self._last is None:
            raise RuntimeError("backward before forward")
        sc, cams_arr, V, cfg = self._last
        if grads is None:
            grads = zero_grads(g)
        ws = ctypes.c_void_p(self.ws.data_ptr())
        ls = loss_scale.to(torch.float32).contiguous()
        self._mark("render_bwd")
        N.check(N.load().gs_render_bwd_objective(ctypes.byref(sc), cams_arr, ctypes.byref(cfg), ws, _ptr(ls),
                                                 _ptr(grads["means"]), _ptr(grads["scales"]), _ptr(grads["quats"]),
                                                 _ptr(grads["opacity"]), _ptr(grads["rgb"]), _ptr(grads["sem_w"]),
                                                 _stream()), "gs_render_bwd_objective")
        self._mark("bwd_end")
        return grads

    # -- candidates -----------------------------------------------------------
    def candidates(self, g: Gaussians, cams, check=True, out=None) -> torch.Tensor:
        """Per-view (sum U, sum H, N_S) for candidate poses: float64 [V,3]."""
        lib = N.load()
        sc = scene_struct(g.means, g.scales, g.quats, g.opacity, g.rgb, g.sem_ids, g.sem_w, g.m, g.geo_unc)
        cams_arr = cameras_array(cams)
        V = len(cams)
        if out is None:
            out = torch.empty((V, 3), dtype=torch.float64, device=self.device)
        for _ in range(8):
            cfg = self.config(g.n, largest_group(cams, self.cand_group_pixels))
            ws = self._ensure_ws(sc, cams_arr, V, cfg)
            N.check(lib.gs_render_candidates(ctypes.byref(sc), cams_arr, V, ctypes.byref(cfg), ws, _ptr(out),
                                             _stream()), "gs_render_candidates")
            if not check:
                break
            cnt = N.GsCounters()
            st = lib.gs_read_counters(ws, ctypes.byref(cnt), _stream())
            if st == N.GS_OK:
                self._fit_capacities(cnt, cfg)
                break
            if st != N.GS_ERR_CAPACITY:
                N.check(st, "gs_render_candidates (device status)")
            if cnt.n_records > cfg.record_capacity:
                self.record_capacity = int(cnt.n_records * 1.1) + 1024
            if cnt.n_pairs > cfg.pair_capacity:
                self.pair_capacity = int(cnt.n_pairs * 1.25) + 4096
        self._last = None
        return out

    def work_counts(self, g: Gaussians, cams, check=True, per_pixel=False) -> dict:
        """Work counters of the blend passes for the views `cams` (project,
        bin, then gs_count_work): n_eval (pixel-rectangle pairs up to each
        pixel's stop), n_eval_box (those inside the alpha box), n_contrib,
        n_touched (classes above the 0.001 clip floor) and n_pixels; with
        per_pixel (one view) also "per_pixel": int32 [H, W, 2] of each
        pixel's (n_eval, n_contrib)."""
        cams = list(cams)
        sc, cams_arr, cfg, ws = self._project_bin(g, cams, check)
        out = torch.zeros(5, dtype=torch.int64, device=self.device)
        pp = None
        if per_pixel:
            pp = torch.zeros((cams[0].height, cams[0].width, 2), dtype=torch.int32, device=self.device)
        N.check(N.load().gs_count_work(ctypes.byref(sc), cams_arr, len(cams), ctypes.byref(cfg), ws, _ptr(out),
                                       _ptr(pp), _stream()), "gs_count_work")
        res = dict(zip(("n_eval", "n_eval_box", "n_contrib", "n_touched", "n_pixels"), out.cpu().tolist()))
        if pp is not None:
            res["per_pixel"] = pp.cpu().numpy()
        return res

    def _fit_capacities(self, cnt, cfg):
        """After a checked candidate call: capacities well above the counts
        are cut to 1.15x the counts, and the workspace is re-laid at the
        next call (the default capacities are sized for the worst case; the
        fitted layout also lets the contributor bits of the two-pass
        candidate kernels fit).  Later calls whose counts exceed the fitted
        capacities report the capacity status and regrow under check=True."""
        rc = int(cnt.n_records * 1.15) + 4096
        pc = int(cnt.n_pairs * 1.15) + 65536
        if cfg.pair_capacity > pc + pc // 4 or cfg.record_capacity > rc + rc // 4:
            self.record_capacity, self.pair_capacity = rc, pc
            self._shrink_ws = True

    # -- inspection -------------------------------------------------------------
    def workspace_views(self) -> dict:
        """Tensor views of the records and sorted pairs of the last
        projection (for parity tests)."""
        sc, cams_arr, V, cfg = self._last
        mp = N.GsWorkspaceMap()
        ws = ctypes.c_void_p(self.ws.data_ptr())
        N.check(N.load().gs_workspace_layout(ctypes.byref(sc), cams_arr, V, ctypes.byref(cfg), ws, ctypes.byref(mp)),
                "gs_workspace_layout")
        base = self.ws.data_ptr()
        cnt = self.counters()
        nr = min(cnt.n_records, mp.record_capacity)
        npairs = min(cnt.n_pairs, mp.pair_capacity)

        def view(ptr, count, dtype, width=1):
            off = ptr - base
            nbytes = count * width * torch.tensor([], dtype=dtype).element_size()
            t = self.ws[off:off + nbytes].view(dtype)
            return t.view(count, width) if width > 1 else t

        return dict(n_records=nr, n_pairs=npairs, status=cnt.status,
                    uv=view(mp.rec_uv, nr, torch.float32, 2), conic=view(mp.rec_conic, nr, torch.float32, 4),
                    depth=view(mp.rec_depth, nr, torch.float32), rect=view(mp.rec_rect, nr, torch.int16, 4),
                    gid=view(mp.rec_gid, nr, torch.int32), view=view(mp.rec_view, nr, torch.int32),
                    pair_tile=view(mp.pair_tile, npairs, torch.int32), pair_rec=view(mp.pair_rec, npairs, torch.int32),
                    ranges=view(mp.tile_ranges, mp.total_tiles, torch.int32, 2),
                    tile_offset=view(mp.tile_offset, V + 1, torch.int32))


# ---------------------------------------------------------------------------
# autograd
# ---------------------------------------------------------------------------

class _RasterizeFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rast, cam, sem_ids, m, want_sem, check, means, scales, quats, opacity, rgb, sem_w):
        g = Gaussians(means.detach(), scales.detach(), quats.detach(), opacity.detach(), rgb.detach(), sem_ids,
                      sem_w.detach(), m)
        out_rgb, depth, sil, sem = rast.forward(g, cam, want_sem=want_sem, check=check)
        ctx.rast = rast
        ctx.cam = cam
        ctx.gen = rast.generation
        ctx.g = g
        if sem is None:
            sem = torch.zeros(0, device=means.device)
            ctx.mark_non_differentiable(sem)
        return out_rgb, depth, sil, sem

    @staticmethod
    def backward(ctx, d_rgb, d_depth, d_sil, d_sem):
        rast = ctx.rast
        if rast.generation != ctx.gen:
            raise RuntimeError("the rasterizer's workspace was reused by another forward before this backward")
        c = lambda t: None if t is None or t.numel() == 0 else t.contiguous()
        grads = rast.backward(ctx.g, ctx.cam, c(d_rgb), c(d_depth), c(d_sil), c(d_sem))
        return (None, None, None, None, None, None, grads["means"], grads["scales"], grads["quats"],
                grads["opacity"], grads["rgb"], grads["sem_w"])


def rasterize(rast: Rasterizer, g: Gaussians, cam, means=None, scales=None, quats=None, opacity=None, rgb=None,
              sem_w=None, want_sem=True, check=True):
    """Differentiable render of one view (Eq. 1, Eq. 3).  Parameter tensors
    default to those of ``g``; pass leaf tensors with requires_grad to get
    gradients.  Returns (rgb, depth, sil, sem)."""
    means = g.means if means is None else means
    scales = g.scales if scales is None else scales
    quats = g.quats if quats is None else quats
    opacity = g.opacity if opacity is None else opacity
    rgb = g.rgb if rgb is None else rgb
    sem_w = g.sem_w if sem_w is None else sem_w
    return _RasterizeFn.apply(rast, cam, g.sem_ids, g.m, want_sem, check, means, scales, quats, opacity, rgb, sem_w)


class _RenderL1Fn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rast, cam, sem_ids, m, check, t_rgb, t_depth, t_sem, means, scales, quats, opacity, rgb,
                sem_w):
        g = Gaussians(means.detach(), scales.detach(), quats.detach(), opacity.detach(), rgb.detach(), sem_ids,
                      sem_w.detach(), m)
        loss = rast.forward_l1(g, cam, t_rgb, t_depth, t_sem, check=check)
        ctx.rast, ctx.cam, ctx.gen, ctx.g = rast, cam, rast.generation, g
        return loss

    @staticmethod
    def backward(ctx, gl):
        rast = ctx.rast
        if rast.generation != ctx.gen:
            raise RuntimeError("the rasterizer's workspace was reused by another forward before this backward")
        grads = rast.backward_l1(ctx.g, ctx.cam, gl)
        return (None, None, None, None, None, None, None, None, grads["means"], grads["scales"], grads["quats"],
                grads["opacity"], grads["rgb"], grads["sem_w"])


def render_l1(rast: Rasterizer, g: Gaussians, cam, t_rgb, t_depth, t_sem=None, means=None, scales=None, quats=None,
              opacity=None, rgb=None, sem_w=None, check=True):
    """Differentiable fused render + mean-L1 loss against targets (colour
    [H,W,3], depth [H,W], semantic map [H,W,m] or None).  Returns the scalar
    loss; its backward runs the adjoint from 2-bit sign codes, so no
    per-pixel gradient map is materialised."""
    means = g.means if means is None else means
    scales = g.scales if scales is None else scales
    quats = g.quats if quats is None else quats
    opacity = g.opacity if opacity is None else opacity
    rgb = g.rgb if rgb is None else rgb
    sem_w = g.sem_w if sem_w is None else sem_w
    return _RenderL1Fn.apply(rast, cam, g.sem_ids, g.m, check, t_rgb, t_depth, t_sem, means, scales, quats, opacity,
                             rgb, sem_w)


class _RenderObjectiveFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rast, cam, sem_ids, m, check, t_rgb, t_depth, t_sem, means, scales, quats, opacity, rgb,
                sem_w):
        g = Gaussians(means.detach(), scales.detach(), quats.detach(), opacity.detach(), rgb.detach(), sem_ids,
                      sem_w.detach(), m)
        loss = rast.forward_objective(g, cam, t_rgb, t_depth, t_sem, check=check)
        ctx.rast, ctx.cam, ctx.gen, ctx.g = rast, cam, rast.generation, g
        return loss

    @staticmethod
    def backward(ctx, gl):
        rast = ctx.rast
        if rast.generation != ctx.gen:
            raise RuntimeError("the rasterizer's workspace was reused by another forward before this backward")
        grads = rast.backward_objective(ctx.g, ctx.cam, gl)
        return (None, None, None, None, None, None, None, None, grads["means"], grads["scales"], grads["quats"],
                grads["opacity"], grads["rgb"], grads["sem_w"])


def render_objective(rast: Rasterizer, g: Gaussians, cam, t_rgb, t_depth, t_sem=None, means=None, scales=None,
                     quats=None, opacity=None, rgb=None, sem_w=None, check=True, fused=None):
    """Differentiable render + Sec. 3.1 mapping objective against targets
    (colour [H,W,3], depth [H,W], class distribution [H,W,m] or None).
    Returns the scalar loss.  ``fused=None`` takes the fused kernels where the
    configuration allows and otherwise renders the maps and evaluates
    ``mapping_loss`` on them (both on the GPU); True / False force one."""
    means = g.means if means is None else means
    scales = g.scales if scales is None else scales
    quats = g.quats if quats is None else quats
    opacity = g.opacity if opacity is None else opacity
    rgb = g.rgb if rgb is None else rgb
    sem_w = g.sem_w if sem_w is None else sem_w
    if fused is not False:
        try:
            return _RenderObjectiveFn.apply(rast, cam, g.sem_ids, g.m, check, t_rgb, t_depth, t_sem, means, scales,
                                            quats, opacity, rgb, sem_w)
        except N.GsError as e:
            if fused or e.code != N.GS_ERR_UNSUPPORTED:
                raise
    out = rasterize(rast, g, cam, means, scales, quats, opacity, rgb, sem_w, want_sem=t_sem is not None,
                    check=check)
    return mapping_loss(out[0], out[1], out[2], out[3], t_rgb, t_depth, t_sem, g.k)


# ---------------------------------------------------------------------------
# fused L1 loss
# ---------------------------------------------------------------------------

_PARTIAL = {}


def l1_loss_and_grads(rgb, depth, sem, t_rgb, t_depth, t_sem):
    """Mean-L1 loss over colour, depth and (optional) semantic map, and its
    gradients, in one native pass.  Returns (loss[()], d_rgb, d_depth, d_sem)."""
    dev = rgb.device
    npix = int(depth.numel())
    m = int(sem.shape[-1]) if sem is not None else 0
    part = _PARTIAL.get(dev)
    if part is None:
        part = _PARTIAL[dev] = torch.empty(2048, dtype=torch.float64, device=dev)
    loss = torch.empty((), dtype=torch.float32, device=dev)
    d_rgb = torch.empty_like(rgb)
    d_depth = torch.empty_like(depth)
    d_sem = torch.empty_like(sem) if sem is not None else None
    N.check(N.load().gs_l1_loss(npix, m, _ptr(rgb), _ptr(t_rgb), _ptr(depth), _ptr(t_depth), _ptr(sem),
                                _ptr(t_sem), _ptr(d_rgb), _ptr(d_depth), _ptr(d_sem), _ptr(loss), _ptr(part),
                                _stream()), "gs_l1_loss")
    return loss, d_rgb, d_depth, d_sem


_PARTIAL_ML = {}


def mapping_loss_and_grads(rgb, depth, sil, sem, t_rgb, t_depth, t_sem, k: int):
    """The mapping objective of Sec. 3.1 on rendered maps (silhouette-masked
    depth / colour L1, summed; entropy-masked Hellinger + cosine semantic
    term, averaged) and its gradients with respect to rgb, depth and sem, in
    one native pass.  Returns (loss[()], d_rgb, d_depth, d_sem)."""
    dev = rgb.device
    npix = int(depth.numel())
    m = int(sem.shape[-1]) if sem is not None else 0
    part = _PARTIAL_ML.get(dev)
    if part is None:
        part = _PARTIAL_ML[dev] = torch.empty(N.GS_MAPPING_LOSS_PARTIALS, dtype=torch.float64, device=dev)
    loss = torch.empty((), dtype=torch.float32, device=dev)
    d_rgb = torch.empty_like(rgb)
    d_depth = torch.empty_like(depth)
    d_sem = torch.empty_like(sem) if sem is not None else None
    c = lambda t: None if t is None else t.contiguous()
    N.check(N.load().gs_mapping_loss(npix, m, int(k), _ptr(c(rgb)), _ptr(c(t_rgb)), _ptr(c(depth)), _ptr(c(t_depth)),
                                     _ptr(c(sil)), _ptr(c(sem)), _ptr(c(t_sem)), _ptr(d_rgb), _ptr(d_depth),
                                     _ptr(d_sem), _ptr(loss), _ptr(part), _stream()), "gs_mapping_loss")
    return loss, d_rgb, d_depth, d_sem


class _MappingLossFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, k, t_rgb, t_depth, t_sem, rgb, depth, sil, sem):
        loss, d_rgb, d_depth, d_sem = mapping_loss_and_grads(rgb.detach(), depth.detach(), sil.detach(),
                                                             None if sem is None else sem.detach(), t_rgb, t_depth,
                                                             t_sem, k)
        ctx.save_for_backward(d_rgb, d_depth, d_sem if d_sem is not None else torch.zeros(0, device=rgb.device))
        ctx.has_sem = d_sem is not None
        return loss

    @staticmethod
    def backward(ctx, gl):
        d_rgb, d_depth, d_sem = ctx.saved_tensors
        return (None, None, None, None, d_rgb * gl, d_depth * gl, None, d_sem * gl if ctx.has_sem else None)


def mapping_loss(rgb, depth, sil, sem, t_rgb, t_depth, t_sem, k: int):
    """Differentiable mapping objective of Sec. 3.1 on rendered maps (e.g. the
    outputs of ``rasterize``): its backward feeds the rasterizer's adjoint."""
    return _MappingLossFn.apply(int(k), t_rgb, t_depth, t_sem, rgb, depth, sil, sem)
