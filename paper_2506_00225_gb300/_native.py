"""ctypes declarations of the C ABI in ``include/gs.h`` (argument
marshalling only).  Loading fails loudly when ``libgs.so`` has not been
built: there is no CPU fallback for any entry point."""
from __future__ import annotations

import ctypes
import os

from . import build as _build

c_int32, c_int64, c_uint32, c_void_p, c_size_t, c_double = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                                             ctypes.c_void_p, ctypes.c_size_t, ctypes.c_double)

GS_OK, GS_ERR_ARG, GS_ERR_CAPACITY, GS_ERR_CUDA, GS_ERR_TIMEOUT, GS_ERR_UNSUPPORTED, GS_ERR_TOO_LARGE = range(7)
GS_NOALLOC_SCRATCH_BYTES = 32 << 20
GS_MAPPING_LOSS_PARTIALS = 2048

EXPORTS = ["gs_workspace_size", "gs_workspace_layout", "gs_project", "gs_bin_sort", "gs_render_fwd",
           "gs_render_bwd", "gs_render_fwd_l1", "gs_render_bwd_l1", "gs_render_fwd_dense", "gs_render_fwd_objective",
           "gs_render_bwd_objective", "gs_render_candidates", "gs_l1_loss", "gs_mapping_loss", "gs_render_fwd_noalloc",
           "gs_score_candidates", "gs_candidate_poses", "gs_candidate_positions", "gs_topk_init", "gs_topk_gather",
           "gs_voxel_words", "gs_voxel_scratch_words", "gs_voxel_update", "gs_voxel_new_free", "gs_read_counters",
           "gs_status_string", "gs_testing_set_sm_query", "gs_testing_grid", "gs_count_work"]


class GsScene(ctypes.Structure):
    _fields_ = [("n", c_int32), ("k", c_int32), ("m", c_int32), ("means", c_void_p), ("scales", c_void_p),
                ("quats", c_void_p), ("opacity", c_void_p), ("rgb", c_void_p), ("sem_ids", c_void_p),
                ("sem_w", c_void_p), ("geo_unc", c_void_p)]


class GsCamera(ctypes.Structure):
    _fields_ = [("width", c_int32), ("height", c_int32), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("near_plane", ctypes.c_float),
                ("w2c", ctypes.c_float * 12)]


class GsConfig(ctypes.Structure):
    _fields_ = [("tile_w", c_int32), ("tile_h", c_int32), ("sem_detach_geometry", c_int32), ("px_per_thread", c_int32),
                ("record_capacity", c_int64), ("pair_capacity", c_int64), ("recompute_bwd", c_int32),
                ("spin_limit", c_int32), ("cand_bits_bytes", c_int64), ("cand_batch", c_int32),
                ("cand_group_pixels", c_int64)]


class GsVoxelGrid(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_float * 3), ("voxel", ctypes.c_float), ("nx", c_int32), ("ny", c_int32),
                ("nz", c_int32)]


class GsCounters(ctypes.Structure):
    _fields_ = [("status", c_uint32), ("n_records", c_uint32), ("n_pairs", c_uint32), ("n_contrib", c_uint32)]


class GsWorkspaceMap(ctypes.Structure):
    _fields_ = [("counters", c_void_p), ("rec_uv", c_void_p), ("rec_conic", c_void_p), ("rec_depth", c_void_p),
                ("rec_rect", c_void_p), ("rec_gid", c_void_p), ("rec_view", c_void_p), ("pair_tile", c_void_p),
                ("pair_rec", c_void_p), ("tile_ranges", c_void_p), ("tile_offset", c_void_p),
                ("record_capacity", c_int64), ("pair_capacity", c_int64), ("total_tiles", c_int64)]


P = ctypes.POINTER
_SIGS = {
    "gs_workspace_size": (c_size_t, [P(GsScene), P(GsCamera), ctypes.c_int, P(GsConfig)]),
    "gs_workspace_layout": (ctypes.c_int, [P(GsScene), P(GsCamera), ctypes.c_int, P(GsConfig), c_void_p,
                                           P(GsWorkspaceMap)]),
    "gs_project": (ctypes.c_int, [P(GsScene), P(GsCamera), ctypes.c_int, P(GsConfig), c_void_p, c_void_p]),
    "gs_bin_sort": (ctypes.c_int, [P(GsScene), P(GsCamera), ctypes.c_int, P(GsConfig), c_void_p, c_void_p]),
    "gs_render_fwd": (ctypes.c_int, [P(GsScene), P(GsCamera), P(GsConfig), c_void_p, c_void_p, c_void_p, c_void_p,
                                     c_void_p, c_void_p]),
    "gs_render_bwd": (ctypes.c_int, [P(GsScene), P(GsCamera), P(GsConfig), c_void_p] + [c_void_p] * 4 +
                      [c_void_p] * 6 + [c_void_p]),
    "gs_render_fwd_l1": (ctypes.c_int, [P(GsScene), P(GsCamera), P(GsConfig), c_void_p] + [c_void_p] * 3 +
                         [c_void_p] * 5 + [c_void_p]),
    "gs_render_bwd_l1": (ctypes.c_int, [P(GsScene), P(GsCamera), P(GsConfig), c_void_p, c_void_p] +
                         [c_void_p] * 6 + [c_void_p]),
    "gs_render_fwd_dense": (ctypes.c_int, [P(GsScene), P(GsCamera), P(GsConfig), c_void_p, c_void_p] +
                            [c_void_p] * 4 + [c_void_p]),
    "gs_render_fwd_objective": (ctypes.c_int, [P(GsScene), P(GsCamera), P(GsConfig), c_void_p] + [c_void_p] * 3 +
                                [c_void_p] * 4 + [c_void_p]),
    "gs_render_bwd_objective": (ctypes.c_int, [P(GsScene), P(GsCamera), P(GsConfig), c_void_p, c_void_p] +
                                [c_void_p] * 6 + [c_void_p]),
    "gs_render_candidates": (ctypes.c_int, [P(GsScene), P(GsCamera), ctypes.c_int, P(GsConfig), c_void_p, c_void_p,
                                            c_void_p]),
    "gs_l1_loss": (ctypes.c_int, [c_int64, ctypes.c_int] + [c_void_p] * 6 + [c_void_p] * 3 + [c_void_p, c_void_p,
                                                                                             c_void_p]),
    "gs_mapping_loss": (ctypes.c_int, [c_int64, ctypes.c_int, ctypes.c_int] + [c_void_p] * 7 + [c_void_p] * 3 +
                        [c_void_p, c_void_p, c_void_p]),
    "gs_render_fwd_noalloc": (ctypes.c_int, [P(GsScene), P(GsCamera), P(GsConfig)] + [c_void_p] * 4 +
                              [c_void_p, c_void_p]),
    "gs_score_candidates": (ctypes.c_int, [ctypes.c_int] + [c_void_p] * 4 + [c_double] + [c_void_p] * 3 +
                            [c_void_p]),
    "gs_candidate_poses": (ctypes.c_int, [ctypes.c_int, c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_float, ctypes.c_float, ctypes.c_float, P(GsCamera)]),
    "gs_candidate_positions": (c_int64, [c_int64, c_void_p, ctypes.c_float, ctypes.c_int, c_void_p, ctypes.c_float,
                                         c_void_p, c_int64]),
    "gs_topk_init": (ctypes.c_int, [c_int64, ctypes.c_int, ctypes.c_int] + [c_void_p] * 4 + [c_void_p]),
    "gs_topk_gather": (ctypes.c_int, [c_int64, ctypes.c_int, ctypes.c_int] + [c_void_p] * 4 + [c_void_p]),
    "gs_voxel_words": (c_int64, [P(GsVoxelGrid)]),
    "gs_voxel_scratch_words": (c_int64, [P(GsVoxelGrid)]),
    "gs_voxel_update": (ctypes.c_int, [P(GsVoxelGrid), c_void_p, c_void_p, P(GsCamera), ctypes.c_int, ctypes.c_float,
                                       c_void_p]),
    "gs_voxel_new_free": (ctypes.c_int, [P(GsVoxelGrid), c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p,
                                         c_void_p]),
    "gs_read_counters": (ctypes.c_int, [c_void_p, P(GsCounters), c_void_p]),
    "gs_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "gs_testing_set_sm_query": (None, [c_void_p]),
    "gs_testing_grid": (c_int64, [ctypes.c_int]),
    "gs_count_work": (ctypes.c_int, [P(GsScene), P(GsCamera), ctypes.c_int, P(GsConfig), c_void_p, c_void_p,
                                     c_void_p, c_void_p]),
}

# gs_testing_grid ids (include/gs.h)
GS_GRID_EMIT_CHUNKS, GS_GRID_EMIT_WRITE, GS_GRID_SORT_RESET, GS_GRID_RANGES, GS_GRID_ZERO_GRAD = range(5)
SM_QUERY = ctypes.CFUNCTYPE(ctypes.c_int)

_LIB = None


def library_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Load ``libgs.so`` (built in-tree by ``build.build()``)."""
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"native rasterizer library missing at {path}; build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


class GsError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = load().gs_status_string(code).decode()
        super().__init__(f"{where}: {msg} (status {code})")
        self.code = code


def check(code: int, where: str) -> None:
    if code != GS_OK:
        raise GsError(code, where)
