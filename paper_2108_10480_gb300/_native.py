"""ctypes declarations of libsd (include/sd.h). Argument marshalling only:
every step of the computation runs in the CUDA library. Importing this
module loads the library and raises if it is missing; there is no CPU
fallback."""
from __future__ import annotations

import ctypes
import os

from . import build_ext

c_void_p, c_int64, c_int32, c_float, c_double = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                                 ctypes.c_float, ctypes.c_double)

SD_OK = 0
STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "out of device memory",
          4: "non-finite coordinate", 5: "primitive index out of range", 6: "size too large",
          7: "device wait timed out"}


class SdPoints(ctypes.Structure):
    _fields_ = [("xyz", c_void_p), ("n", c_int64)]


class SdEdges(ctypes.Structure):
    _fields_ = [("V", c_void_p), ("nv", c_int64), ("E", c_void_p), ("ne", c_int64)]


class SdTris(ctypes.Structure):
    _fields_ = [("V", c_void_p), ("nv", c_int64), ("F", c_void_p), ("nf", c_int64)]


class SdGeometry(ctypes.Structure):
    _fields_ = [("pts", SdPoints), ("edges", SdEdges), ("tris", SdTris)]


class SdBuildOpts(ctypes.Structure):
    _fields_ = [("alpha_u", c_float), ("leaf_size", c_int32), ("weights", c_int32), ("paper_metric", c_int32),
                ("defer_checks", c_int32)]


class SdQueryOpts(ctypes.Structure):
    _fields_ = [("sort_queries", c_int32), ("block", c_int32), ("counts", c_void_p), ("order", c_void_p)]


class SdTraceOpts(ctypes.Structure):
    _fields_ = [("eye", c_float * 3), ("target", c_float * 3), ("up", c_float * 3), ("fov_y", c_float),
                ("width", c_int32), ("height", c_int32), ("eps", c_float), ("t_max", c_float),
                ("max_steps", c_int32), ("block", c_int32)]


class SdTreeInfo(ctypes.Structure):
    _fields_ = [("n_prims", c_int64), ("n_points", c_int64), ("n_edges", c_int64), ("n_tris", c_int64),
                ("n_buckets", c_int64), ("leaf_size", c_int32),
                ("alpha", c_float), ("beta", c_float), ("alpha_u", c_float), ("S", c_float),
                ("A_E", c_float), ("A_T", c_float), ("w_far", c_float),
                ("scene_lo", c_float * 3), ("scene_hi", c_float * 3), ("device_bytes", c_int64)]


class SdTreeView(ctypes.Structure):
    _fields_ = [("codes", c_void_p), ("sorted", c_void_p), ("left", c_void_p), ("right", c_void_p),
                ("node_lo", c_void_p), ("node_hi", c_void_p), ("node_count", c_void_p),
                ("leaf_lo", c_void_p), ("leaf_hi", c_void_p), ("leaf_count", c_void_p), ("params", c_void_p)]


# every symbol include/sd.h declares, with (restype, argtypes)
SIGNATURES = {
    "sd_default_build_opts": (None, [ctypes.POINTER(SdBuildOpts)]),
    "sd_default_query_opts": (None, [ctypes.POINTER(SdQueryOpts)]),
    "sd_build": (ctypes.c_int, [ctypes.POINTER(SdGeometry), c_float, c_float, ctypes.POINTER(SdBuildOpts),
                                c_void_p, ctypes.POINTER(c_void_p)]),
    "sd_query": (ctypes.c_int, [c_void_p, c_void_p, c_int64, c_void_p, c_void_p, ctypes.POINTER(SdQueryOpts),
                                c_void_p]),
    "sd_query_brute": (ctypes.c_int, [c_void_p, c_void_p, c_int64, c_void_p, c_void_p,
                                      ctypes.POINTER(SdQueryOpts), c_void_p]),
    "sd_query_order": (ctypes.c_int, [c_void_p, c_void_p, c_int64, c_void_p, c_void_p]),
    "sd_query_noalloc": (ctypes.c_int, [c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_void_p]),
    "sd_pose_query": (ctypes.c_int, [c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p,
                                     ctypes.POINTER(SdQueryOpts), c_void_p]),
    "sd_pose_reduce": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_float,
                                      c_void_p, c_void_p, c_void_p]),
    "sd_pose_partial": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_float,
                                       c_void_p, c_void_p]),
    "sd_pose_merge": (ctypes.c_int, [c_void_p, c_int32, c_void_p, c_float, c_void_p]),
    "sd_batch_create": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_int32, ctypes.POINTER(c_void_p)]),
    "sd_batch_set_poses": (ctypes.c_int, [c_void_p, c_void_p, c_void_p]),
    "sd_batch_run": (ctypes.c_int, [c_void_p, c_float, c_int32, c_void_p, c_void_p]),
    "sd_batch_vertex_outputs": (ctypes.c_int, [c_void_p, ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p),
                                               ctypes.POINTER(c_void_p)]),
    "sd_batch_free": (None, [c_void_p]),
    "sd_mlp_num_params": (ctypes.c_int64, []),
    "sd_mlp_workspace_bytes": (ctypes.c_size_t, [c_int64]),
    "sd_mlp_forward": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_void_p]),
    "sd_mlp_train_step": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_int32, c_float, c_void_p, c_void_p,
                                         c_void_p, c_int64, c_void_p, c_void_p, c_void_p, ctypes.c_size_t,
                                         c_void_p]),
    "sd_query_prims": (ctypes.c_int, [c_void_p, c_void_p, c_int64, c_void_p, ctypes.c_int32, c_int64, c_void_p,
                                      c_void_p, ctypes.POINTER(SdQueryOpts), c_void_p]),
    "sd_mesh_reduce": (ctypes.c_int, [c_void_p, ctypes.c_int32, c_int64, c_int64, c_void_p, c_void_p, c_float,
                                      c_void_p, c_void_p, c_void_p, c_void_p]),
    "sd_sphere_trace": (ctypes.c_int, [c_void_p, ctypes.POINTER(SdTraceOpts), c_void_p, c_void_p,
                                       ctypes.POINTER(c_int64), c_void_p]),
    "sd_lower_bound": (ctypes.c_int, [c_void_p, c_void_p, c_int64, c_float, c_void_p, c_void_p, c_void_p, c_void_p]),
    "sd_surrogate_query": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_float, c_void_p, c_int64, c_void_p,
                                          c_void_p, c_void_p, ctypes.POINTER(c_int64), c_void_p]),
    "sd_query_status": (ctypes.c_int, [c_void_p, c_void_p]),
    "sd_kernel_launches": (ctypes.c_int64, []),
    "sd_tree_get_info": (ctypes.c_int, [c_void_p, ctypes.POINTER(SdTreeInfo)]),
    "sd_tree_export": (ctypes.c_int, [c_void_p, ctypes.POINTER(SdTreeView)]),
    "sd_free": (None, [c_void_p]),
    "sd_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "sd_last_error": (ctypes.c_char_p, []),
    "sd_weight_basis": (ctypes.c_int, [c_void_p]),
    "sd_weight_horner_tables": (ctypes.c_int, [c_void_p]),
    "sd_peak_probe": (ctypes.c_int, [c_int32, c_int32, c_int32, c_void_p, ctypes.POINTER(c_double), c_void_p]),
}

_lib = None


def lib():
    """Load (building first if needed) libsd.so and declare its symbols."""
    global _lib
    if _lib is not None:
        return _lib
    # SD_AUTOBUILD=0 loads the prebuilt library only (ctypes raises OSError
    # if it is missing); otherwise a stale or missing library is rebuilt.
    if os.environ.get("SD_AUTOBUILD", "1") == "1":
        path = build_ext.build()
    else:
        path = build_ext.LIB
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


class SdError(RuntimeError):
    def __init__(self, code, where=""):
        msg = STATUS.get(code, f"status {code}")
        extra = ""
        if code == 2 and _lib is not None:
            extra = ": " + (_lib.sd_last_error() or b"").decode()
        super().__init__(f"{where}: {msg}{extra}" if where else msg + extra)
        self.code = code


def check(code, where=""):
    if code != SD_OK:
        raise SdError(code, where)
