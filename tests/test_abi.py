"""The C ABI library builds, loads and exports every symbol declared in
include/gs.h; host-side argument validation works without a GPU."""
import ctypes
import os
import re

import pytest

from paper_2506_00225_gb300 import _native as N
from paper_2506_00225_gb300 import build as B
from paper_2506_00225_gb300 import raster, scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return N.load()


def test_exports_every_declared_symbol(lib):
    names = header_functions()
    assert len(names) >= 10
    assert sorted(N.EXPORTS) == names
    for name in names:
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for code in range(7):
        assert lib.gs_status_string(code)
    assert b"capacity" in lib.gs_status_string(N.GS_ERR_CAPACITY)


def _structs(n=100, views=1, w=64, h=48, tile=(16, 16)):
    sc = N.GsScene()
    sc.n, sc.k, sc.m = n, 3, 16
    cams = raster.cameras_array([scenes.look_camera((0, 0, 1.5), 0.0, w, h, 50.0)] * views)
    cfg = N.GsConfig()
    cfg.tile_w, cfg.tile_h = tile
    cfg.sem_detach_geometry = 1
    return sc, cams, cfg


def test_workspace_size_and_layout_host_only(lib):
    sc, cams, cfg = _structs()
    size = lib.gs_workspace_size(ctypes.byref(sc), cams, 1, ctypes.byref(cfg))
    assert size > 0 and size % 256 == 0
    mp = N.GsWorkspaceMap()
    base = 1 << 40  # a fake, never dereferenced device address
    assert lib.gs_workspace_layout(ctypes.byref(sc), cams, 1, ctypes.byref(cfg), ctypes.c_void_p(base),
                                   ctypes.byref(mp)) == N.GS_OK
    ptrs = [mp.counters, mp.rec_uv, mp.rec_conic, mp.rec_depth, mp.rec_rect, mp.rec_gid, mp.rec_view, mp.pair_tile,
            mp.pair_rec, mp.tile_ranges, mp.tile_offset]
    assert all(base <= p < base + size for p in ptrs)
    assert mp.record_capacity == 100 and mp.total_tiles == 4 * 3
    # more candidate views -> more tiles and records
    sc2, cams2, cfg2 = _structs(views=2)
    sc5, cams5, cfg5 = _structs(views=5)
    assert lib.gs_workspace_size(ctypes.byref(sc5), cams5, 5, ctypes.byref(cfg5)) > \
        lib.gs_workspace_size(ctypes.byref(sc2), cams2, 2, ctypes.byref(cfg2)) > 0
    # recomputation mode keeps no contributor bits: 8 bytes per tile pixel
    # per 64 pairs of capacity less
    cfg.pair_capacity = 1 << 16
    keep = lib.gs_workspace_size(ctypes.byref(sc), cams, 1, ctypes.byref(cfg))
    cfg.recompute_bwd = 1
    lean = lib.gs_workspace_size(ctypes.byref(sc), cams, 1, ctypes.byref(cfg))
    assert 0 < lean and keep - lean >= 8 * ((1 << 16) // 64) * 16 * 16


@pytest.mark.parametrize("bad", ["k0", "k17", "m0", "views0", "views257", "tile0", "width0", "near0", "fx_nan",
                                 "ppt3", "ppt4_h8", "recompute2", "spin_neg"])
def test_invalid_arguments_rejected_on_host(lib, bad):
    sc, cams, cfg = _structs()
    views = 1
    if bad == "k0":
        sc.k = 0
    elif bad == "k17":
        sc.k = 17
    elif bad == "m0":
        sc.m = 0
    elif bad == "views0":
        views = 0
    elif bad == "views257":
        views = 257
    elif bad == "tile0":
        cfg.tile_w = 0
    elif bad == "width0":
        cams[0].width = 0
    elif bad == "near0":
        cams[0].near_plane = 0.0
    elif bad == "fx_nan":
        cams[0].fx = float("nan")
    elif bad == "ppt3":
        cfg.px_per_thread = 3
    elif bad == "ppt4_h8":
        cfg.px_per_thread, cfg.tile_h = 4, 8
    elif bad == "spin_neg":
        cfg.spin_limit = -1
    elif bad == "recompute2":
        cfg.recompute_bwd = 2
    assert lib.gs_workspace_size(ctypes.byref(sc), cams, views, ctypes.byref(cfg)) == 0
    # every entry point refuses before touching the GPU
    fake = ctypes.c_void_p(1 << 40)
    assert lib.gs_project(ctypes.byref(sc), cams, views, ctypes.byref(cfg), fake, None) == N.GS_ERR_ARG
    assert lib.gs_bin_sort(ctypes.byref(sc), cams, views, ctypes.byref(cfg), fake, None) == N.GS_ERR_ARG


def test_null_workspace_and_misaligned_rejected(lib):
    sc, cams, cfg = _structs()
    assert lib.gs_project(ctypes.byref(sc), cams, 1, ctypes.byref(cfg), None, None) == N.GS_ERR_ARG
    assert lib.gs_project(ctypes.byref(sc), cams, 1, ctypes.byref(cfg), ctypes.c_void_p((1 << 40) + 8),
                          None) == N.GS_ERR_ARG
    out = ctypes.c_void_p(1 << 41)
    assert lib.gs_render_candidates(ctypes.byref(sc), cams, 1, ctypes.byref(cfg), None, out, None) == N.GS_ERR_ARG
    assert lib.gs_l1_loss(0, 1, None, None, None, None, None, None, None, None, None, None, None,
                          None) == N.GS_ERR_ARG


def test_scene_pointer_checks(lib):
    sc, cams, cfg = _structs()
    fake = ctypes.c_void_p(1 << 40)
    # n > 0 with NULL means -> refused
    assert lib.gs_project(ctypes.byref(sc), cams, 1, ctypes.byref(cfg), fake, None) == N.GS_ERR_ARG
    # quaternions must be 16-byte aligned
    sc.means = sc.scales = sc.opacity = ctypes.c_void_p(1 << 40)
    sc.quats = ctypes.c_void_p((1 << 40) + 4)
    assert lib.gs_project(ctypes.byref(sc), cams, 1, ctypes.byref(cfg), fake, None) == N.GS_ERR_ARG


def test_unsupported_tile_shape(lib):
    sc, cams, cfg = _structs(n=0, tile=(12, 12))
    fake = ctypes.c_void_p(1 << 40)
    assert lib.gs_render_fwd(ctypes.byref(sc), cams, ctypes.byref(cfg), fake, None, None, None, None,
                             None) == N.GS_ERR_UNSUPPORTED


def test_product_has_no_oracle_dependency():
    """The product package never imports or links the oracle."""
    pkg = os.path.join(ROOT, "paper_2506_00225_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "gs_oracle" not in txt, f


@pytest.mark.parametrize("case", ["attached", "recompute", "m256k8", "ok_n0"])
def test_objective_preconditions_on_host(lib, case):
    """gs_render_fwd_objective / gs_render_bwd_objective refuse, before any GPU
    work, the configurations without a fused form: semantics reaching the
    geometry, the recompute mode (no contributor bits), a class accumulator
    that does not fit one shared-memory chunk (256 classes, top-8, 16x16)."""
    sc, cams, cfg = _structs(n=0)
    if case == "attached":
        cfg.sem_detach_geometry = 0
    elif case == "recompute":
        cfg.recompute_bwd = 1
    elif case == "m256k8":
        sc.m, sc.k = 256, 8
    fake = ctypes.c_void_p(1 << 40)  # never dereferenced: every call below returns before GPU work
    t = ctypes.c_void_p(1 << 41)
    if case == "ok_n0":
        # accepted configuration: a missing target is the only error left
        assert lib.gs_render_fwd_objective(ctypes.byref(sc), cams, ctypes.byref(cfg), fake, None, t, t, None, None,
                                           None, t, None) == N.GS_ERR_ARG
        assert lib.gs_render_bwd_objective(ctypes.byref(sc), cams, ctypes.byref(cfg), fake, None, None, None, None,
                                           None, None, None, None) == N.GS_ERR_ARG
        return
    fwd = lib.gs_render_fwd_objective(ctypes.byref(sc), cams, ctypes.byref(cfg), fake, t, t, t, None, None, None,
                                      t, None)
    bwd = lib.gs_render_bwd_objective(ctypes.byref(sc), cams, ctypes.byref(cfg), fake, t, None, None, None, None,
                                      None, None, None)
    assert fwd == N.GS_ERR_UNSUPPORTED and bwd == N.GS_ERR_UNSUPPORTED


def test_dense_preconditions_on_host(lib):
    """gs_render_fwd_dense: a semantic output without the dense array is an
    argument error; the recompute mode has no contributor bits."""
    sc, cams, cfg = _structs(n=0)
    fake = ctypes.c_void_p(1 << 40)  # never dereferenced: both calls return before GPU work
    t = ctypes.c_void_p(1 << 41)
    sc.n = 5
    sc.means = sc.scales = sc.opacity = sc.rgb = sc.sem_ids = sc.sem_w = t
    sc.quats = t
    assert lib.gs_render_fwd_dense(ctypes.byref(sc), cams, ctypes.byref(cfg), fake, None, None, None, None, t,
                                   None) == N.GS_ERR_ARG
    sc.n = 0
    cfg.recompute_bwd = 1
    assert lib.gs_render_fwd_dense(ctypes.byref(sc), cams, ctypes.byref(cfg), fake, None, None, None, None, None,
                                   None) == N.GS_ERR_UNSUPPORTED


def test_noalloc_size_and_argument_checks_on_host(lib):
    """The allocation-free entry point refuses, before any GPU work, sizes
    whose workspace would exceed its fixed scratch array and invalid
    arguments (no device is touched: the pointers are never dereferenced)."""
    fake = ctypes.c_void_p(1 << 40)

    def call(sc, cams, cfg):
        return lib.gs_render_fwd_noalloc(ctypes.byref(sc), cams, ctypes.byref(cfg), fake, fake, fake, None, None,
                                         None)

    def with_pointers(sc):
        sc.means = sc.scales = sc.quats = sc.opacity = sc.rgb = sc.sem_ids = sc.sem_w = fake
        return sc

    sc, cams, cfg = _structs(n=4_000_000, w=1200, h=680)
    size = lib.gs_workspace_size(ctypes.byref(sc), cams, 1, ctypes.byref(cfg))
    assert size > N.GS_NOALLOC_SCRATCH_BYTES
    assert call(with_pointers(sc), cams, cfg) == N.GS_ERR_TOO_LARGE
    # NULL scene arrays with n > 0, misaligned quaternions, a tile shape without kernels
    sc, cams, cfg = _structs(n=100)
    assert call(sc, cams, cfg) == N.GS_ERR_ARG
    sc = with_pointers(sc)
    sc.quats = ctypes.c_void_p((1 << 40) + 4)
    assert call(sc, cams, cfg) == N.GS_ERR_ARG
    sc, cams, cfg = _structs(n=100, tile=(12, 12))
    assert call(with_pointers(sc), cams, cfg) == N.GS_ERR_UNSUPPORTED


@pytest.mark.parametrize("sms", [1, 100, 152, 160, 600])
def test_grids_follow_the_sm_count(lib, sms):
    """The grid-stride kernels size their grids from the device's SM count
    (queried per device), not a fixed GB300 figure: with the query stubbed,
    every grid scales with the stubbed count."""
    calls = []

    def query():
        calls.append(1)
        return sms

    cb = N.SM_QUERY(query)
    lib.gs_testing_set_sm_query(ctypes.cast(cb, ctypes.c_void_p))
    try:
        assert lib.gs_testing_grid(N.GS_GRID_EMIT_CHUNKS) == min(2 * sms, 1024)
        assert lib.gs_testing_grid(N.GS_GRID_EMIT_WRITE) == 8 * sms
        assert lib.gs_testing_grid(N.GS_GRID_SORT_RESET) == 2 * sms
        assert lib.gs_testing_grid(N.GS_GRID_RANGES) == 4 * sms
        assert lib.gs_testing_grid(N.GS_GRID_ZERO_GRAD) == 2 * sms
        assert lib.gs_testing_grid(99) == -1
        assert calls
    finally:
        lib.gs_testing_set_sm_query(None)


def test_grid_without_a_device_is_zero(lib):
    """Without a device (this CPU container) the SM count is unknown and the
    library reports a zero grid instead of a guessed one; launch chains then
    fail with a CUDA error rather than running a wrong-sized grid."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    lib.gs_testing_set_sm_query(None)
    assert lib.gs_testing_grid(N.GS_GRID_SORT_RESET) == 0


def test_candidate_config_checked_on_host(lib):
    """Candidate batch sizes other than 32, 64, 128 and a negative bit
    budget are refused; a budget bounds the workspace of a multi-view
    layout (the bits of 8 large views would need far more)."""
    sc, cams, cfg = _structs(n=2_000_000, views=8, w=1200, h=680)
    for bad in (16, 48, 256, -1):
        cfg.cand_batch = bad
        assert lib.gs_workspace_size(ctypes.byref(sc), cams, 8, ctypes.byref(cfg)) == 0
    cfg.cand_batch = 0
    cfg.cand_bits_bytes = -5
    assert lib.gs_workspace_size(ctypes.byref(sc), cams, 8, ctypes.byref(cfg)) == 0
    cfg.cand_bits_bytes = 0
    sizes = {}
    for budget in (1 << 30, 4 << 30):
        cfg.cand_bits_bytes = budget
        sizes[budget] = lib.gs_workspace_size(ctypes.byref(sc), cams, 8, ctypes.byref(cfg))
        assert sizes[budget] > 0
    assert 2.5 * (1 << 30) < sizes[4 << 30] - sizes[1 << 30] <= 3 * (1 << 30) + (1 << 20)
    for b in (32, 64, 128):
        cfg.cand_batch = b
        assert lib.gs_workspace_size(ctypes.byref(sc), cams, 8, ctypes.byref(cfg)) > 0


def test_grouped_candidate_workspace(lib):
    """cand_group_pixels: a grouped candidate call is laid out one group of
    consecutive views at a time (views added while their pixels fit the
    budget, at least one), so its workspace is the largest group's
    (computed here group by group), well below the whole list's; a negative
    budget is refused, a budget covering every view changes nothing, and
    the entry points that run all views at once refuse a list that needs
    several groups."""
    sc = N.GsScene()
    sc.n, sc.k, sc.m = 500_000, 3, 16
    sizes = [(300, 170, 150.0), (600, 340, 300.0), (1200, 680, 600.0)] * 3
    cams = raster.cameras_array([scenes.look_camera((0, 0, 1.5), 40.0 * i, w, h, f)
                                 for i, (w, h, f) in enumerate(sizes)])
    cfg = N.GsConfig()
    cfg.tile_w, cfg.tile_h = 16, 16
    nv, budget = len(sizes), 900_000
    # 51k, 204k, 816k pixels: groups [0, 1], [2, 3], [4], [5, 6], [7], [8]
    groups = [(0, 2), (2, 4), (4, 5), (5, 7), (7, 8), (8, 9)]
    whole = lib.gs_workspace_size(ctypes.byref(sc), cams, nv, ctypes.byref(cfg))
    per = [lib.gs_workspace_size(ctypes.byref(sc), ctypes.cast(ctypes.addressof(cams) + a * ctypes.sizeof(N.GsCamera),
                                                               ctypes.POINTER(N.GsCamera)), b - a, ctypes.byref(cfg))
           for a, b in groups]
    cfg.cand_group_pixels = budget
    grouped = lib.gs_workspace_size(ctypes.byref(sc), cams, nv, ctypes.byref(cfg))
    assert grouped == max(per) and 0 < grouped < 0.5 * whole, (grouped, per, whole)
    assert raster.largest_group([scenes.look_camera((0, 0, 1.5), 0.0, w, h, f) for w, h, f in sizes], budget) == 2
    cfg.cand_group_pixels = 3 * (51_000 + 204_000 + 816_000)
    assert lib.gs_workspace_size(ctypes.byref(sc), cams, nv, ctypes.byref(cfg)) == whole
    cfg.cand_group_pixels = -1
    assert lib.gs_workspace_size(ctypes.byref(sc), cams, nv, ctypes.byref(cfg)) == 0
    fake = ctypes.c_void_p(1 << 40)  # never dereferenced: the calls fail on the host
    out = ctypes.c_void_p(1 << 41)
    assert lib.gs_render_candidates(ctypes.byref(sc), cams, nv, ctypes.byref(cfg), fake, out, None) == N.GS_ERR_ARG
    cfg.cand_group_pixels = budget
    assert lib.gs_project(ctypes.byref(sc), cams, nv, ctypes.byref(cfg), fake, None) == N.GS_ERR_ARG
    mp = N.GsWorkspaceMap()
    assert lib.gs_workspace_layout(ctypes.byref(sc), cams, nv, ctypes.byref(cfg), fake,
                                   ctypes.byref(mp)) == N.GS_ERR_ARG
