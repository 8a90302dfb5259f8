"""Launch-configuration autotuner for the tile kernels.

Times the fused mapping step (project, bin/sort, forward + mean-L1, adjoint)
for every compiled tile shape and pixels-per-thread mapping on the caller's
own scene, view and targets, and returns the fastest.  The rendered values
and gradients do not depend on the choice (every pixel sees the same
Gaussians in the same order); only the time does.  Results are cached per
(Gaussians, image size, k, m).
"""
from __future__ import annotations

import statistics

import torch

from . import raster

SHAPES = ((16, 16), (16, 8), (32, 8), (8, 8))
PPTS = (4, 2, 1)  # 4: tiles whose height is a multiple of 16 only


def _valid(tile, ppt):
    return ppt != 4 or tile[1] % 16 == 0

_CACHE: dict = {}


def _time_config(g, cam, targets, tile, ppt, reps, device):
    rast = raster.Rasterizer(tile=tile, px_per_thread=ppt, device=device)
    loss = rast.forward_l1(g, cam, *targets, check=True)  # sizes the workspace
    rast.backward_l1(g, cam, torch.ones((), device=device))
    ones = torch.ones((), device=device)
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        torch.cuda._sleep(2_000_000)  # let the host enqueue the whole step first
        s.record()
        rast.forward_l1(g, cam, *targets, check=False)
        rast.backward_l1(g, cam, ones)
        e.record()
        torch.cuda.synchronize()
        times.append(s.elapsed_time(e))
    del loss
    return statistics.median(times), rast


def tune_mapping(g: raster.Gaussians, cam, t_rgb, t_depth, t_sem, reps: int = 5, device=None):
    """Returns (best {tile, px_per_thread, ms}, table of all timings)."""
    key = (g.n, cam.width, cam.height, g.k, g.m)
    if key in _CACHE:
        return _CACHE[key]
    device = device or g.means.device
    table = []
    for tile in SHAPES:
        for ppt in PPTS:
            if not _valid(tile, ppt):
                continue
            ms, _ = _time_config(g, cam, (t_rgb, t_depth, t_sem), tile, ppt, reps, device)
            table.append({"tile": f"{tile[0]}x{tile[1]}", "px_per_thread": ppt, "ms": round(ms, 4)})
    best = min(table, key=lambda r: r["ms"])
    w, h = (int(x) for x in best["tile"].split("x"))
    res = ({"tile": (w, h), "px_per_thread": best["px_per_thread"], "ms": best["ms"]}, table)
    _CACHE[key] = res
    return res


CAND_BATCHES = (32, 64, 128)
_CAND_CACHE: dict = {}


def tune_candidates(g: raster.Gaussians, cams, reps: int = 5, device=None):
    """Times the batched candidate render of the caller's own views for
    every compiled tile shape and staged batch size (32, 64, 128 Gaussians)
    and returns (best {tile, cand_batch, ms}, table of all timings).  The
    per-view sums do not depend on the choice.  Cached per (Gaussians,
    view sizes, k, m)."""
    key = (g.n, tuple((c.width, c.height) for c in cams), g.k, g.m)
    if key in _CAND_CACHE:
        return _CAND_CACHE[key]
    device = device or g.means.device
    table = []
    for tile in SHAPES:
        for batch in CAND_BATCHES:
            rast = raster.Rasterizer(tile=tile, cand_batch=batch, device=device)
            out = rast.candidates(g, cams, check=True)  # sizes and fits the workspace
            rast.candidates(g, cams, check=False, out=out)
            torch.cuda.synchronize()
            times = []
            for _ in range(reps):
                s = torch.cuda.Event(enable_timing=True)
                e = torch.cuda.Event(enable_timing=True)
                torch.cuda._sleep(2_000_000)
                s.record()
                rast.candidates(g, cams, check=False, out=out)
                e.record()
                torch.cuda.synchronize()
                times.append(s.elapsed_time(e))
            table.append({"tile": f"{tile[0]}x{tile[1]}", "cand_batch": batch,
                          "ms": round(statistics.median(times), 4)})
            del rast
    best = min(table, key=lambda r: r["ms"])
    w, h = (int(x) for x in best["tile"].split("x"))
    res = ({"tile": (w, h), "cand_batch": best["cand_batch"], "ms": best["ms"]}, table)
    _CAND_CACHE[key] = res
    return res


def fit_candidate_budget(g: raster.Gaussians, cams, ws_bytes: int, tile=(16, 16), cand_batch: int = 0,
                         device=None):
    """Largest pixel budget of the candidate view groups
    (gs_config.cand_group_pixels) whose workspace stays within `ws_bytes`:
    starts with all views in one group and halves the budget until the
    workspace, laid out at the capacities fitted to a checked call's counts,
    fits, or the budget reaches the largest view.  Returns (a Rasterizer
    fitted to the views, the budget (0: one group), its workspace bytes).
    The per-view sums do not depend on the budget."""
    device = device or g.means.device
    total = sum(c.width * c.height for c in cams)
    floor = max(c.width * c.height for c in cams)
    budget = total
    while True:
        gp = 0 if budget >= total else budget
        rast = raster.Rasterizer(tile=tile, cand_batch=cand_batch, cand_group_pixels=gp, device=device)
        out = rast.candidates(g, cams, check=True)  # counts -> fitted capacities
        rast.candidates(g, cams, check=True, out=out)  # workspace re-laid at them
        ws = int(rast.ws.numel())
        if ws <= ws_bytes or budget <= floor:
            return rast, gp, ws
        del rast, out
        budget = max(floor, budget // 2)
