"""ctypes declarations of the C ABI in include/afr.h (argument marshalling only).

Loading fails loudly when libafr.so has not been built: there is no CPU
fallback for any step of the reconstruction path.
"""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libafr.so")
DEBUG_LIB_PATH = os.path.join(_PKG, "libafr_debug.so")   # AFR_DEBUG build: device checks and test hooks

c_i32, c_u32, c_u64, c_f32, c_p = ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_float, ctypes.c_void_p

AFR_OK, AFR_ERR_INVALID_ARG, AFR_ERR_BAD_STATE, AFR_ERR_OOM, AFR_ERR_CUDA, AFR_ERR_TIMEOUT, AFR_ERR_DEVICE_CHECK = range(7)
AFR_INSERT_RESET = 1
STATUS_NAMES = ["AFR_OK", "AFR_ERR_INVALID_ARG", "AFR_ERR_BAD_STATE", "AFR_ERR_OOM", "AFR_ERR_CUDA",
                "AFR_ERR_TIMEOUT", "AFR_ERR_DEVICE_CHECK"]
AFR_F32, AFR_F16, AFR_BF16 = 0, 1, 2
AFR_MAP_LBAR, AFR_MAP_GX, AFR_MAP_GY, AFR_MAP_GT, AFR_MAP_SIGMA_S, AFR_MAP_SIGMA_T = range(6)
AFR_MAP_FOOTPRINT, AFR_MAP_COVERAGE = 6, 7
AFR_RECON_KEEP_SIGMA, AFR_RECON_ADAPTIVE_SUPPORT, AFR_RECON_COVERAGE_RESET = 1, 2, 4
AFR_PROFILE_MAX_LAUNCHES = 256

EXPORTED = [
    "afr_create", "afr_destroy", "afr_reset", "afr_reserve", "afr_insert_samples", "afr_estimate_gradients",
    "afr_reproject", "afr_reconstruct", "afr_reconstruct_ex", "afr_tile_feedback", "afr_reconstruct_backward",
    "afr_get_status", "afr_last_error", "afr_query", "afr_num_tiles", "afr_export_ring", "afr_export_frame",
    "afr_export_map", "afr_import_map", "afr_set_frame_colors", "afr_reproject_batch_static", "afr_set_tuning",
    "afr_profile_filter", "afr_profile_read", "afr_tile_error", "afr_reproject_camera",
    "afr_batch_create", "afr_batch_destroy", "afr_batch_reconstruct", "afr_measure_alu_peaks",
    "afr_batch_refresh", "afr_insert_samples_ex",
]


class AfrConfig(ctypes.Structure):
    _fields_ = [("width", c_i32), ("height", c_i32), ("depth", c_i32), ("tile", c_i32), ("radius", c_i32),
                ("color_type", c_i32), ("window", c_f32), ("eps_grad", c_f32), ("undersample_m", c_f32),
                ("fifo_capacity", c_u32), ("world_points", c_u32)]


class AfrParams(ctypes.Structure):
    _fields_ = [("alpha_s", c_f32), ("beta_s", c_f32), ("clamp_s", c_f32), ("alpha_t", c_f32),
                ("beta_t", c_f32), ("clamp_t", c_f32)]


class AfrSampleBatch(ctypes.Structure):
    _fields_ = [("pos_dev", c_p), ("color_dev", c_p), ("motion_dev", c_p), ("world_dev", c_p)]


class AfrTileStats(ctypes.Structure):
    _fields_ = [("n", c_u32), ("empty_slots", c_u32), ("mean_L", c_f32), ("var_L", c_f32), ("mean_Gx", c_f32),
                ("mean_Gy", c_f32), ("mean_Gt", c_f32), ("u", c_f32)]


class AfrInfo(ctypes.Structure):
    _fields_ = [("inserted", c_u64), ("rejected", c_u64), ("resident", c_u64), ("frame", c_u64),
                ("dropped", c_u64), ("unsorted_bins", c_u64)]


_lock = threading.Lock()
_lib = None
_debug_lib = None
DEBUG_EXPORTED = ["afr_debug_fail_alloc", "afr_debug_set_frame_offsets"]


def _declare(L):
    S = c_i32
    sig = {
        "afr_create": (S, [ctypes.POINTER(AfrConfig), ctypes.POINTER(c_p)]),
        "afr_destroy": (None, [c_p]),
        "afr_reset": (S, [c_p, c_p]),
        "afr_reserve": (S, [c_p, c_u32]),
        "afr_insert_samples": (S, [c_p, ctypes.POINTER(AfrSampleBatch), c_u32, c_p]),
        "afr_insert_samples_ex": (S, [c_p, ctypes.POINTER(AfrSampleBatch), c_u32, c_u32, c_p, c_p]),
        "afr_estimate_gradients": (S, [c_p, c_f32, c_p]),
        "afr_reproject": (S, [c_p, c_f32, c_p]),
        "afr_reconstruct": (S, [c_p, c_f32, ctypes.POINTER(AfrParams), c_p, c_p]),
        "afr_reconstruct_ex": (S, [c_p, c_f32, ctypes.POINTER(AfrParams), c_u32, c_p, c_p]),
        "afr_tile_feedback": (S, [c_p, c_p, c_p]),
        "afr_reconstruct_backward": (S, [c_p, c_p, c_p, c_p, c_p]),
        "afr_get_status": (S, [c_p, c_p]),
        "afr_last_error": (ctypes.c_char_p, [c_p]),
        "afr_query": (S, [c_p, ctypes.POINTER(AfrInfo), c_p]),
        "afr_num_tiles": (S, [c_p, ctypes.POINTER(c_u32)]),
        "afr_export_ring": (S, [c_p, c_p, c_p, c_p]),
        "afr_export_frame": (S, [c_p, c_p, c_p, c_p, c_u64]),
        "afr_export_map": (S, [c_p, c_i32, c_p]),
        "afr_import_map": (S, [c_p, c_i32, c_p]),
        "afr_set_frame_colors": (S, [c_p, c_p, c_p]),
        "afr_reproject_batch_static": (S, [ctypes.POINTER(AfrSampleBatch), c_u32, c_i32, c_i32, c_i32, c_f32,
                                           c_p, c_p, c_p, c_p, c_p, c_p]),
        "afr_set_tuning": (S, [c_p, c_i32, c_i32]),
        "afr_profile_filter": (S, [c_p, c_i32]),
        "afr_tile_error": (S, [c_p, c_f32, c_f32, c_f32, c_p, c_p, c_p, c_p]),
        "afr_reproject_camera": (S, [c_p, c_f32, c_p, c_p]),
        "afr_profile_read": (S, [c_p, c_p, c_i32, ctypes.POINTER(c_i32)]),
        "afr_batch_create": (S, [ctypes.POINTER(c_p), c_i32, ctypes.POINTER(c_p)]),
        "afr_batch_destroy": (None, [c_p]),
        "afr_batch_reconstruct": (S, [c_p, c_f32, ctypes.POINTER(AfrParams), ctypes.POINTER(c_p), c_p]),
        "afr_measure_alu_peaks": (S, [c_p]),
        "afr_batch_refresh": (S, [c_p, c_f32, ctypes.POINTER(AfrParams), ctypes.POINTER(c_p), c_p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args


def load():
    """Load libafr.so (built by __graft_entry__.build() or build.py)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                                   "(python -c 'import __graft_entry__ as g; g.build()')")
            L = ctypes.CDLL(LIB_PATH)
            _declare(L)
            _lib = L
    return _lib


def load_debug():
    """Load libafr_debug.so, the AFR_DEBUG build (device-side checks and the
    test hooks of include/afr_debug.h); the same ABI as libafr.so besides."""
    global _debug_lib
    with _lock:
        if _debug_lib is None:
            if not os.path.exists(DEBUG_LIB_PATH):
                raise RuntimeError(f"{DEBUG_LIB_PATH} is missing: build the CUDA library first")
            L = ctypes.CDLL(DEBUG_LIB_PATH)
            _declare(L)
            L.afr_debug_fail_alloc.restype = None
            L.afr_debug_fail_alloc.argtypes = [c_i32]
            L.afr_debug_set_frame_offsets.restype = c_i32
            L.afr_debug_set_frame_offsets.argtypes = [c_p, c_p]
            _debug_lib = L
    return _debug_lib


class AfrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
