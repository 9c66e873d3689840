"""ctypes binding of ``libdiffrestore.so`` (declared in ``include/diffrestore.h``).

Argument marshalling only: every function here forwards to the C ABI function
of the same name.  There is no CPU fallback: if the library cannot be built or
loaded, importing it raises."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdiffrestore.so")

DR_OK = 0
DR_ERR_INVALID_ARG = -1
DR_ERR_STATE = -2
DR_ERR_CUDA = -3
DR_ERR_OOM = -4
DR_ERR_DEVICE_CHECK = -5
DR_ERR_TIMEOUT = -6
ERR_NAMES = {0: "DR_OK", -1: "DR_ERR_INVALID_ARG", -2: "DR_ERR_STATE", -3: "DR_ERR_CUDA", -4: "DR_ERR_OOM",
             -5: "DR_ERR_DEVICE_CHECK", -6: "DR_ERR_TIMEOUT"}
DR_DRIFT_NONE, DR_DRIFT_FD, DR_DRIFT_ADJOINT, DR_DRIFT_MALA = 0, 1, 2, 3

# every entry point declared in include/diffrestore.h
EXPORTS = ["dr_version", "dr_last_error", "dr_create", "dr_destroy", "dr_scene_upload", "dr_target_mixture",
           "dr_chains_init", "dr_step", "dr_splat", "dr_resolve", "dr_readback_state", "dr_readback_accum",
           "dr_get_counters", "dr_eval_logp", "dr_trace_closest", "dr_philox", "dr_splat_records",
           "dr_clear_image", "dr_state_save", "dr_state_load", "dr_set_stats", "dr_get_traversal_stats",
           "dr_bvh_info", "dr_get_launch_count", "dr_get_chain_shape", "dr_pt_render", "dr_set_bvh_builder",
           "dr_splat_records_noalloc", "dr_set_option", "dr_get_profile", "dr_frame", "dr_bvh4_info", "dr_bvh4_sah", "dr_bvh8_info", "dr_get_bounce_profile", "dr_get_bounce_rays", "dr_trace_closest_counted", "dr_bvh4_download",
           "dr_scenes_upload_batch", "dr_resolve_scene", "dr_get_scene_counters", "dr_scene_upload_instanced",
           "dr_two_level_info", "dr_splat_records_noalloc_status", "dr_resolve_accum", "dr_get_p_sum",
           "dr_k0_from_p_sum", "dr_lstar_over_p"]
DR_OPT_WORK_ORDER, DR_OPT_WAVEFRONT, DR_OPT_PROFILE, DR_OPT_BVH_WIDTH = 1, 2, 3, 4
DR_OPT_TRAVERSE_BLOCKS, DR_OPT_REFILL, DR_OPT_RAY_ORDER, DR_OPT_TAIL_BOUNCE = 5, 6, 7, 8
DR_OPT_TWO_LEVEL = 9
DR_PHASES = 11
PHASE_NAMES = ["wf_begin", "trace", "shade", "shadow", "finish", "adjoint", "fused_step", "fd_score", "splat",
               "work_order", "tail"]
DR_NOALLOC_MAX_RECORDS = 65536
DR_BVH_LBVH, DR_BVH_PLOC = 0, 1


class dr_scene_desc(C.Structure):
    _fields_ = [("verts", C.c_void_p), ("nv", C.c_int32), ("tris", C.c_void_p), ("normals", C.c_void_p),
                ("nt", C.c_int32), ("tri_mat", C.c_void_p), ("mats", C.c_void_p), ("nm", C.c_int32),
                ("camera", C.c_void_p), ("width", C.c_int32), ("height", C.c_int32),
                ("max_path_len", C.c_int32), ("n_chains", C.c_uint64)]


class dr_mesh_desc(C.Structure):
    _fields_ = [("verts", C.c_void_p), ("nv", C.c_int32), ("tris", C.c_void_p), ("nt", C.c_int32),
                ("normals", C.c_void_p), ("tri_mat", C.c_void_p)]


class dr_instance_desc(C.Structure):
    _fields_ = [("mesh", C.c_int32), ("material", C.c_int32), ("xform", C.c_float * 12)]


class dr_params(C.Structure):
    _fields_ = [("max_path_len", C.c_int32), ("drift_mode", C.c_int32), ("rb_weight", C.c_int32),
                ("steps_per_splat", C.c_int32), ("stddev", C.c_float), ("dt", C.c_float),
                ("gamma_tilde", C.c_float), ("eps", C.c_float), ("fd_h", C.c_float), ("m", C.c_float),
                ("k0", C.c_double)]


class DRError(RuntimeError):
    def __init__(self, code, fn, msg):
        super().__init__(f"{fn} -> {ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


def signatures():
    """ctypes (argtypes, restype) of every entry point, in the order and widths
    of the prototypes in include/diffrestore.h."""
    P, I32, I64, U32, U64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_uint64
    return {
        "dr_version": ([], C.c_int),
        "dr_last_error": ([], C.c_char_p),
        "dr_create": ([C.POINTER(P), C.c_int, P], C.c_int),
        "dr_destroy": ([P], C.c_int),
        "dr_scene_upload": ([P, P, I32, P, P, I32, P, P, I32, P, I32, I32], C.c_int),
        "dr_target_mixture": ([P, I32, I32, P, P, P, C.c_float, I32, I32], C.c_int),
        "dr_chains_init": ([P, U64, U64, U32, C.POINTER(dr_params)], C.c_int),
        "dr_step": ([P, U32], C.c_int),
        "dr_splat": ([P], C.c_int),
        "dr_resolve": ([P, P], C.c_int),
        "dr_readback_state": ([P, P, P, P, P, P, P], C.c_int),
        "dr_readback_accum": ([P, P], C.c_int),
        "dr_get_counters": ([P, P, P, P, P, P], C.c_int),
        "dr_eval_logp": ([P, I32, P, I64, P, P, P, P], C.c_int),
        "dr_trace_closest": ([P, P, I64, I32, P, P], C.c_int),
        "dr_trace_closest_counted": ([P, P, I64, I32, P, P, P, P], C.c_int),
        "dr_bvh4_download": ([P, P, P], C.c_int),
        "dr_philox": ([P, P, P, I64, P], C.c_int),
        "dr_splat_records": ([P, P, I64], C.c_int),
        "dr_clear_image": ([P], C.c_int),
        "dr_state_save": ([P, P, C.POINTER(C.c_size_t)], C.c_int),
        "dr_state_load": ([P, P, C.c_size_t], C.c_int),
        "dr_set_stats": ([P, C.c_int], C.c_int),
        "dr_get_traversal_stats": ([P, P, P, P], C.c_int),
        "dr_bvh_info": ([P, P, P, P], C.c_int),
        "dr_get_launch_count": ([P, P], C.c_int),
        "dr_get_chain_shape": ([P, P, P, P], C.c_int),
        "dr_pt_render": ([P, I32, U32, U64, P], C.c_int),
        "dr_set_bvh_builder": ([P, I32, I32], C.c_int),
        "dr_splat_records_noalloc": ([P, I64, I32, P, P], C.c_int),
        "dr_set_option": ([P, I32, I32], C.c_int),
        "dr_get_profile": ([P, P, P, I32], C.c_int),
        "dr_frame": ([P, U32], C.c_int),
        "dr_bvh4_info": ([P, P, P, P], C.c_int),
        "dr_bvh8_info": ([P, P, P], C.c_int),
        "dr_bvh4_sah": ([P, P, P], C.c_int),
        "dr_get_bounce_profile": ([P, P, I32], C.c_int),
        "dr_get_bounce_rays": ([P, P, I32], C.c_int),
        "dr_scenes_upload_batch": ([P, P, I32], C.c_int),
        "dr_resolve_scene": ([P, I32, P], C.c_int),
        "dr_get_scene_counters": ([P, I32, P, P], C.c_int),
        "dr_scene_upload_instanced": ([P, P, I32, P, I32, P, I32, P, I32, I32], C.c_int),
        "dr_two_level_info": ([P, P, P, P], C.c_int),
        "dr_splat_records_noalloc_status": ([P], C.c_int),
        "dr_resolve_accum": ([P, I64, U64, C.c_double, P, P], C.c_int),
        "dr_get_p_sum": ([P, P, P], C.c_int),
        "dr_k0_from_p_sum": ([C.c_double, U64, C.POINTER(dr_params), P], C.c_int),
        "dr_lstar_over_p": ([P, C.POINTER(dr_params), P, I64, C.c_float, I32, P], C.c_int),
    }


_lib = None


def load(build_if_missing=True):
    """Loads the in-tree library (building it first if it is missing or out of
    date when ``build_if_missing``)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        from . import build as _b
        _b.build()
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libdiffrestore.so not found at {LIB_PATH}; run paper_2605_08916_gb300.build")
    L = C.CDLL(LIB_PATH)
    for name, (args, res) in signatures().items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def last_error():
    return load().dr_last_error().decode()


def check(code, fn):
    if code != DR_OK:
        raise DRError(code, fn, last_error())
    return code


def call(name, *args):
    """Calls a C-ABI function and raises DRError on a non-zero status."""
    return check(getattr(load(), name)(*args), name)
