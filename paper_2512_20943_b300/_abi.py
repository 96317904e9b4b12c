"""ctypes declarations of the libairgs C ABI (include/airgs.h)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libairgs.so")

AIRGS_OK = 0
AIRGS_E_ARG = -1
AIRGS_E_OOM = -2
AIRGS_E_CAPACITY = -3
AIRGS_E_TIMEOUT = -4
AIRGS_E_CUDA = -5
AIRGS_E_STATE = -6
ERROR_NAMES = {
    AIRGS_E_ARG: "AIRGS_E_ARG",
    AIRGS_E_OOM: "AIRGS_E_OOM",
    AIRGS_E_CAPACITY: "AIRGS_E_CAPACITY",
    AIRGS_E_TIMEOUT: "AIRGS_E_TIMEOUT",
    AIRGS_E_CUDA: "AIRGS_E_CUDA",
    AIRGS_E_STATE: "AIRGS_E_STATE",
}

AIRGS_DELTA_PREV = 0
AIRGS_DELTA_ANCHOR = 1
AIRGS_QUAT_ADD = 2
AIRGS_UPDATE_CHANNELS = 7
AIRGS_MAX_VIEWS = 256
AIRGS_NUM_STAGES = 9
AIRGS_PROFILE_OFF = 0
AIRGS_PROFILE_ALL = 1
AIRGS_PROFILE_BLEND = 2
AIRGS_NOALLOC_SORT_MAX_PAIRS = 1 << 20


class airgs_config(ctypes.Structure):
    _fields_ = [
        ("dilation", ctypes.c_float),
        ("alpha_max", ctypes.c_float),
        ("alpha_min", ctypes.c_float),
        ("T_min", ctypes.c_float),
        ("bg", ctypes.c_float * 3),
        ("kernel_shape", ctypes.c_int),
        ("sort_mode", ctypes.c_int),
        ("autotune_cache", ctypes.c_char_p),
        ("cull_lists", ctypes.c_int),
    ]


class airgs_camera(ctypes.Structure):
    _fields_ = [
        ("width", ctypes.c_int),
        ("height", ctypes.c_int),
        ("fx", ctypes.c_float),
        ("fy", ctypes.c_float),
        ("cx", ctypes.c_float),
        ("cy", ctypes.c_float),
        ("viewmat", ctypes.c_float * 16),
        ("near_plane", ctypes.c_float),
    ]


class airgs_gaussians(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("sh_degree", ctypes.c_int),
        ("means", ctypes.c_void_p),
        ("log_scales", ctypes.c_void_p),
        ("quats", ctypes.c_void_p),
        ("opacity_logit", ctypes.c_void_p),
        ("sh", ctypes.c_void_p),
    ]


class airgs_backward_args(ctypes.Structure):
    _fields_ = [
        ("dL_drgb", ctypes.c_void_p),
        ("target", ctypes.c_void_p),
        ("loss_out", ctypes.c_void_p),
        ("g_means", ctypes.c_void_p),
        ("g_log_scales", ctypes.c_void_p),
        ("g_quats", ctypes.c_void_p),
        ("g_opacity_logit", ctypes.c_void_p),
        ("g_sh", ctypes.c_void_p),
        ("importance_w", ctypes.c_void_p),
        ("importance_cnt", ctypes.c_void_p),
        ("densify_grad", ctypes.c_void_p),
        ("densify_views", ctypes.c_void_p),
    ]


class airgs_stats(ctypes.Structure):
    _fields_ = [
        ("n_instances", ctypes.c_int64),
        ("n_tiles", ctypes.c_int64),
        ("n_pixels", ctypes.c_int64),
        ("pairs_forward", ctypes.c_int64),
        ("pairs_backward", ctypes.c_int64),
        ("kernel_shape", ctypes.c_int),
    ]


class airgs_densify_out(ctypes.Structure):
    _fields_ = [
        ("capacity", ctypes.c_int64),
        ("means", ctypes.c_void_p),
        ("log_scales", ctypes.c_void_p),
        ("quats", ctypes.c_void_p),
        ("opacity_logit", ctypes.c_void_p),
        ("sh", ctypes.c_void_p),
        ("parent", ctypes.c_void_p),
        ("n_out", ctypes.c_void_p),
    ]


P = ctypes.c_void_p
I = ctypes.c_int
I64 = ctypes.c_int64
CTX = ctypes.c_void_p
STATE = ctypes.c_void_p

# name -> (restype, argtypes); every function declared in include/airgs.h
SIGNATURES = {
    "airgs_default_config": (None, [ctypes.POINTER(airgs_config)]),
    "airgs_create": (I, [ctypes.POINTER(CTX), ctypes.POINTER(airgs_config), P]),
    "airgs_destroy": (I, [CTX]),
    "airgs_set_stream": (I, [CTX, P]),
    "airgs_sync": (I, [CTX]),
    "airgs_last_error": (ctypes.c_char_p, [CTX]),
    "airgs_set_anchor": (I, [CTX, I64, I, P, P, P, P, P]),
    "airgs_apply_frame_update": (I, [CTX, P, I, I, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), I,
                                     I64]),
    "airgs_get_frame_state": (I, [CTX, P, P]),
    "airgs_render": (I, [CTX, ctypes.POINTER(airgs_camera), I, P, P, P, P, P, ctypes.POINTER(STATE)]),
    "airgs_render_gaussians": (I, [CTX, ctypes.POINTER(airgs_gaussians), ctypes.POINTER(airgs_camera), I, P, P, P,
                                   P, P, ctypes.POINTER(STATE)]),
    "airgs_render_backward": (I, [CTX, STATE, P, P, P, P, P, P, P, P]),
    "airgs_render_backward_l1": (I, [CTX, STATE, P, P, P, P, P, P, P, P, P]),
    "airgs_render_backward_ex": (I, [CTX, STATE, ctypes.POINTER(airgs_backward_args)]),
    "airgs_densify_select": (I, [CTX, P, P, I64, ctypes.c_float, P]),
    "airgs_densify_apply": (I, [CTX, ctypes.POINTER(airgs_gaussians), P, P, ctypes.c_float, ctypes.c_float,
                                ctypes.c_float, ctypes.POINTER(airgs_densify_out)]),
    "airgs_gaussian_importance": (I, [CTX, ctypes.POINTER(airgs_camera), I, P, P]),
    "airgs_prune_mask": (I, [CTX, P, I64, I64, P]),
    "airgs_prune_delta": (I, [CTX, I64, I, P, P, P, P, P]),
    "airgs_apply_frame_delta": (I, [CTX, P, I, I64]),
    "airgs_image_sse": (I, [CTX, ctypes.POINTER(airgs_camera), I, P, P, P]),
    "airgs_l3dgs_loss": (I, [CTX, ctypes.POINTER(airgs_camera), I, P, P, ctypes.c_float, P, P]),
    "airgs_release_state": (I, [CTX, STATE]),
    "airgs_state_stats": (I, [CTX, STATE, ctypes.POINTER(airgs_stats)]),
    "airgs_state_view_info": (I, [CTX, STATE, I, ctypes.POINTER(I64), ctypes.POINTER(I64)]),
    "airgs_state_projection": (I, [CTX, STATE, I, P, P, P]),
    "airgs_state_tile_lists": (I, [CTX, STATE, I, P, P]),
    "airgs_sort_pairs": (I, [CTX, P, P, P, P, I64, I]),
    "airgs_sort_pairs_noalloc": (I, [P, P, P, P, I64, I, P]),
    "airgs_autotune": (I, [CTX, ctypes.POINTER(airgs_camera), I, ctypes.POINTER(I), ctypes.POINTER(ctypes.c_float),
                           ctypes.POINTER(ctypes.c_float)]),
    "airgs_set_profiling": (I, [CTX, I]),
    "airgs_stage_times": (I, [CTX, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I64), ctypes.POINTER(I64)]),
    "airgs_stage_name": (ctypes.c_char_p, [I]),
    "airgs_measure_fp32_peak": (I, [CTX, ctypes.POINTER(ctypes.c_double)]),
    "airgs_measure_smem_peak": (I, [CTX, ctypes.POINTER(ctypes.c_double)]),
    "airgs_kernel_launch_count": (I64, []),
    "airgs_shape_count": (I, []),
    "airgs_shape_name": (ctypes.c_char_p, [I]),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libairgs.so.  There is no fallback: a missing library is an error."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"libairgs.so not found at {path}; build it with `python -m paper_2512_20943_b300.build` "
            "(nvcc, sm_103a). There is no CPU fallback.")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
