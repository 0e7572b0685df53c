"""ctypes declarations of the C ABI in include/ag.h (argument marshalling only).

The shared library is built in-tree by ``paper_2605_26137_b300.build`` and is
required: there is no fallback implementation, so a missing library raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from ctypes import POINTER, c_char_p, c_float, c_int32, c_int64, c_void_p

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libagbake.so")

AG_OK = 0
AG_ERR_INVALID_ARG = 1
AG_ERR_OOM = 2
AG_ERR_CUDA = 3
AG_ERR_TRAVERSAL_LIMIT = 4
AG_ERR_BAD_HANDLE = 5

AG_BVH_Q8 = 0
AG_BVH_F32 = 1
AG_COLLAPSE_AREA = 0
AG_COLLAPSE_AREA_COUNT = 1
AG_COLLAPSE_COUNT = 2
AG_COLLAPSE_SAH = 3
AG_TILE_8x8 = 0
AG_TILE_16x16 = 1
AG_TILE_32x8 = 2
AG_TILE_4x4 = 3
AG_SCHED_AUTO = -1
AG_SCHED_BATCH = 0
AG_SCHED_REFILL = 1
AG_SCHED_COOP4 = 2
AG_SCHED_COOP8 = 3
AG_SCHED_COOP2 = 4
AG_QUERY_RAY = 0
AG_QUERY_CLOSEST = 1
AG_RENDER_RASTER = 0
AG_RENDER_TRACE = 1
AG_FILTER_ANISO = 0
AG_FILTER_BILINEAR = 1
AG_QEM_OPTIMAL = 0
AG_QEM_MIDPOINT = 1

# every symbol include/ag.h declares
EXPORTS = ("ag_opts_default", "ag_bvh_build", "ag_bvh_free", "ag_bvh_free_async", "ag_bvh_info", "ag_bvh_copy_out", "ag_bake", "ag_bake_batch",
           "ag_batch_plan_create", "ag_batch_plan_launch", "ag_batch_plan_free", "ag_bake_backward",
           "ag_sync_status", "ag_last_error", "ag_status_string", "ag_version", "ag_vertex_normals_noalloc",
           "ag_autotune", "ag_visibility", "ag_exterior_fill", "ag_qem_simplify",
           "ag_point_distance", "ag_render_views", "ag_backproject", "ag_normal_map_error")


class AgOpts(ctypes.Structure):
    _fields_ = [("bvh_layout", c_int32), ("gutter", c_int32), ("disp_fp16", c_int32), ("schedule", c_int32),
                ("block_size", c_int32), ("blocks_per_sm", c_int32), ("max_steps", c_int32),
                ("collapse", c_int32), ("ray_tile", c_int32), ("query", c_int32), ("render", c_int32),
                ("filter", c_int32), ("build_async", c_int32), ("stack_limit", c_int32), ("reserved", c_int32 * 2)]


class AgBakeAux(ctypes.Structure):
    _fields_ = [("normal_ts", c_void_p), ("disp_f32", c_void_p), ("face", c_void_p), ("bary", c_void_p),
                ("hit_tri", c_void_p), ("hit_t", c_void_p), ("counters", c_void_p), ("n_rays", c_void_p),
                ("events", c_void_p)]


class AgAssetDesc(ctypes.Structure):
    _fields_ = [("bvh", c_void_p), ("lverts", c_void_p), ("lnormals", c_void_p), ("luv", c_void_p),
                ("lfaces", c_void_p), ("n_lverts", c_int64), ("n_lfaces", c_int64), ("W", c_int32),
                ("H", c_int32), ("max_dist", c_float), ("normal_rgba8", c_void_p), ("mask", c_void_p),
                ("disp", c_void_p)]


class AgBvhInfo(ctypes.Structure):
    _fields_ = [("n_tris", c_int64), ("n_verts", c_int64), ("n_nodes", c_int64), ("node_bytes", c_int64),
                ("tri_bytes", c_int64), ("normal_bytes", c_int64), ("layout", c_int32), ("node_size", c_int32),
                ("max_depth", c_int32), ("reserved", c_int32), ("scene_lo", c_float * 3),
                ("scene_hi", c_float * 3), ("diam", c_float), ("build_ms", c_float)]


class AgError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{status_name(status)}: {message}")
        self.status = status


_lib = None
_lock = threading.Lock()


def load():
    """Load libagbake.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA extension with __graft_entry__.build()")
        lib = ctypes.CDLL(LIB_PATH)
        S = c_int32
        lib.ag_opts_default.argtypes = [POINTER(AgOpts)]
        lib.ag_opts_default.restype = None
        lib.ag_bvh_build.argtypes = [c_void_p, c_int64, c_void_p, c_int64, POINTER(AgOpts), c_void_p,
                                     POINTER(c_void_p)]
        lib.ag_bvh_build.restype = S
        lib.ag_bvh_free.argtypes = [c_void_p]
        lib.ag_bvh_free.restype = S
        lib.ag_bvh_free_async.argtypes = [c_void_p, c_void_p]
        lib.ag_bvh_free_async.restype = S
        lib.ag_bvh_info.argtypes = [c_void_p, POINTER(AgBvhInfo)]
        lib.ag_bvh_info.restype = S
        lib.ag_bvh_copy_out.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
        lib.ag_bvh_copy_out.restype = S
        lib.ag_bake.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_int64, c_int32, c_int32,
                                c_float, POINTER(AgOpts), c_void_p, c_void_p, c_void_p, c_void_p, POINTER(AgBakeAux)]
        lib.ag_bake.restype = S
        lib.ag_bake_batch.argtypes = [c_int32, POINTER(AgAssetDesc), POINTER(AgOpts), c_void_p]
        lib.ag_bake_batch.restype = S
        lib.ag_batch_plan_create.argtypes = [c_int32, POINTER(AgAssetDesc), POINTER(AgOpts), c_void_p,
                                             POINTER(c_void_p)]
        lib.ag_batch_plan_create.restype = S
        lib.ag_batch_plan_launch.argtypes = [c_void_p, c_void_p]
        lib.ag_batch_plan_launch.restype = S
        lib.ag_batch_plan_free.argtypes = [c_void_p]
        lib.ag_batch_plan_free.restype = S
        lib.ag_bake_backward.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_int64, c_int32, c_int32,
                                         c_float, c_float, POINTER(AgOpts), c_void_p, c_void_p, c_void_p]
        lib.ag_bake_backward.restype = S
        lib.ag_autotune.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_int64, c_int32,
                                    c_int32, c_float, c_void_p, POINTER(AgOpts), POINTER(c_float)]
        lib.ag_autotune.restype = S
        lib.ag_visibility.argtypes = [c_void_p, c_int32, c_int32, POINTER(AgOpts), c_void_p, c_void_p, c_void_p,
                                      c_void_p]
        lib.ag_visibility.restype = S
        lib.ag_exterior_fill.argtypes = [c_void_p, c_int64, c_void_p, c_int64, c_void_p, c_void_p, c_void_p]
        lib.ag_exterior_fill.restype = S
        lib.ag_qem_simplify.argtypes = [c_void_p, c_int64, c_void_p, c_int64, c_int64, c_int32, c_int32, c_void_p,
                                        c_void_p, c_void_p, c_void_p, c_void_p]
        lib.ag_point_distance.argtypes = [c_void_p, c_void_p, c_int64, c_float, POINTER(AgOpts), c_void_p, c_void_p,
                                          c_void_p]
        lib.ag_point_distance.restype = S
        lib.ag_normal_map_error.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_int64, c_int32, c_int32,
                                            c_void_p, c_void_p, c_void_p, c_int64, c_float, POINTER(AgOpts), c_void_p,
                                            c_void_p]
        lib.ag_normal_map_error.restype = S
        lib.ag_render_views.argtypes = [c_void_p, c_int32, c_void_p, c_int32, c_int32, c_float, POINTER(AgOpts),
                                        c_void_p, c_void_p, c_void_p, c_void_p]
        lib.ag_render_views.restype = S
        lib.ag_backproject.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_int64, c_int32, c_int32,
                                       c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_int32,
                                       c_float, c_float, c_float, POINTER(AgOpts), c_void_p, c_void_p, c_void_p]
        lib.ag_backproject.restype = S
        lib.ag_qem_simplify.restype = S
        lib.ag_sync_status.argtypes = [c_void_p]
        lib.ag_sync_status.restype = S
        lib.ag_last_error.argtypes = []
        lib.ag_last_error.restype = c_char_p
        lib.ag_status_string.argtypes = [c_int32]
        lib.ag_status_string.restype = c_char_p
        lib.ag_version.argtypes = []
        lib.ag_version.restype = c_int32
        _lib = lib
        return lib


def status_name(s: int) -> str:
    try:
        return load().ag_status_string(s).decode()
    except Exception:  # noqa: BLE001 - naming must not mask the original error
        return f"status {s}"


def check(status: int) -> None:
    if status != AG_OK:
        msg = load().ag_last_error().decode(errors="replace")
        raise AgError(status, msg)


def default_opts(**kw) -> AgOpts:
    o = AgOpts()
    load().ag_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if v is not None:
            setattr(o, k, int(v))
    return o
