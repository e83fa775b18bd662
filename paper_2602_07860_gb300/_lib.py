"""ctypes binding of libmbr.so (the C ABI in include/mbr.h).  Argument marshalling only: every
step of the renderer runs in the library's CUDA kernels.  There is no CPU fallback: if the
library is missing or no CUDA device is present, calls raise."""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_float, c_int32, c_int64, c_void_p

from . import build as _build

MBR_OK, MBR_ERR_ARG, MBR_ERR_CUDA, MBR_ERR_OOM, MBR_ERR_TIMEOUT, MBR_ERR_DEVICE = range(6)
MBR_PLAIN, MBR_FAST = 0, 1
MBR_TRANSLATE, MBR_ROTATE, MBR_PARABOLIC = 0, 1, 2
MBR_TIME_PAPER, MBR_TIME_MIDPOINT = 0, 1
MBR_PROB_EXP, MBR_PROB_SIGMOID = 0, 1
MBR_INTERP_SCREEN, MBR_INTERP_PERSPECTIVE = 0, 1
SOLVERS = {"plain": MBR_PLAIN, "fast": MBR_FAST}

EXPORTS = ["mbr_create", "mbr_destroy", "mbr_render_blur", "mbr_render_blur_backward",
           "mbr_render_blur_backward_reuse", "mbr_render_blur_batch",
           "mbr_debug_winners", "mbr_count_candidates", "mbr_count_work", "mbr_set_tuning", "mbr_set_profiling", "mbr_get_stats",
           "mbr_render_blur_noalloc", "mbr_autotune", "mbr_set_state_budget", "mbr_sdf_extract", "mbr_sdf_extract_backward", "mbr_measure_fp32_peak", "mbr_debug_wait_limit", "mbr_last_error"]


class MbrMesh(ctypes.Structure):
    _fields_ = [("V", c_int32), ("F", c_int32), ("verts", c_void_p), ("faces", c_void_p), ("albedo", c_void_p),
                ("uv", c_void_p), ("texture", c_void_p), ("tex_h", c_int32), ("tex_w", c_int32),
                ("dl_dtexture", c_void_p)]


class MbrMotion(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("segments", c_int32), ("offset", c_float * 3), ("dir", c_float * 3),
                ("axis", c_float * 3), ("omega", c_float), ("acc", c_float * 3)]


class MbrCamera(ctypes.Structure):
    _fields_ = [("view", c_float * 12), ("tan_half_fov", c_float), ("znear", c_float), ("light_dir", c_float * 3),
                ("k_ambient", c_float), ("k_diffuse", c_float), ("delta", c_float), ("time_rule", c_int32),
                ("prob", c_int32), ("interp", c_int32)]


class MbrItem(ctypes.Structure):
    _fields_ = [("mesh", MbrMesh), ("motion", MbrMotion), ("camera", MbrCamera), ("T", c_int32), ("H", c_int32),
                ("W", c_int32), ("solver", c_int32), ("image", c_void_p), ("dl_dimage", c_void_p),
                ("dl_dverts", c_void_p), ("dl_dalbedo", c_void_p)]


class MbrStats(ctypes.Structure):
    _fields_ = [("launches", c_int64), ("bin_entries", c_int64), ("raster_fwd_ms", ctypes.c_double),
                ("raster_bwd_ms", ctypes.c_double), ("raster_fwd_count", c_int64), ("raster_bwd_count", c_int64),
                ("n_split", c_int32), ("groups", c_int32), ("reused", c_int64)]


class MbrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mbr error {code}: {msg}")
        self.code = code


_lib = None


def library_path():
    return _build.library_path()


def load(build_if_missing=True):
    """Load libmbr.so (building it in-tree first if it is missing and nvcc is available)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library {path} is not built; run __graft_entry__.build()")
        _build.build()
    L = ctypes.CDLL(path)
    P = POINTER
    L.mbr_create.argtypes = [P(c_void_p)]
    L.mbr_create.restype = c_int32
    L.mbr_destroy.argtypes = [c_void_p]
    L.mbr_destroy.restype = None
    common = [c_void_p, P(MbrMesh), P(MbrMotion), P(MbrCamera), c_int32, c_int32, c_int32, c_int32]
    L.mbr_render_blur.argtypes = common + [c_void_p, c_void_p]
    L.mbr_render_blur.restype = c_int32
    L.mbr_render_blur_backward.argtypes = common + [c_void_p, c_void_p, c_void_p, c_void_p]
    L.mbr_render_blur_backward.restype = c_int32
    L.mbr_render_blur_backward_reuse.argtypes = common + [c_void_p, c_void_p, c_void_p, c_void_p]
    L.mbr_render_blur_backward_reuse.restype = c_int32
    L.mbr_debug_winners.argtypes = common + [c_int32, c_void_p, c_void_p]
    L.mbr_debug_winners.restype = c_int32
    L.mbr_count_candidates.argtypes = common + [P(c_int64), c_void_p]
    L.mbr_count_candidates.restype = c_int32
    L.mbr_count_work.argtypes = common + [c_void_p, P(c_int64), c_void_p]
    L.mbr_count_work.restype = c_int32
    L.mbr_render_blur_batch.argtypes = [c_void_p, c_int32, P(MbrItem), c_int32, c_void_p]
    L.mbr_render_blur_batch.restype = c_int32
    L.mbr_autotune.argtypes = [c_void_p, c_int32, P(MbrItem), c_int32, P(c_int32), P(c_int32), P(c_float), c_void_p]
    L.mbr_autotune.restype = c_int32
    L.mbr_set_state_budget.argtypes = [c_void_p, c_int64]
    L.mbr_set_state_budget.restype = c_int32
    L.mbr_set_tuning.argtypes = [c_void_p, c_int32, c_int32, c_int32]
    L.mbr_set_tuning.restype = c_int32
    L.mbr_set_profiling.argtypes = [c_void_p, c_int32]
    L.mbr_set_profiling.restype = c_int32
    L.mbr_get_stats.argtypes = [c_void_p, P(MbrStats)]
    L.mbr_get_stats.restype = c_int32
    L.mbr_render_blur_noalloc.argtypes = [P(MbrMesh), P(MbrMotion), P(MbrCamera), c_int32, c_int32, c_int32,
                                          c_int32, c_void_p, c_void_p, ctypes.c_char_p, c_int32]
    L.mbr_render_blur_noalloc.restype = c_int32
    L.mbr_sdf_extract.argtypes = [c_void_p, c_int32, c_void_p, P(c_float), c_float, c_int32, c_int32, c_void_p,
                                  c_void_p, c_void_p, P(c_int32), c_void_p]
    L.mbr_sdf_extract.restype = c_int32
    L.mbr_sdf_extract_backward.argtypes = [c_void_p, c_int32, c_void_p, c_float, c_int32, c_void_p, c_void_p,
                                           c_void_p, c_void_p]
    L.mbr_sdf_extract_backward.restype = c_int32
    L.mbr_measure_fp32_peak.argtypes = [c_void_p, c_int32, c_int32, P(ctypes.c_double), P(c_float), c_void_p]
    L.mbr_measure_fp32_peak.restype = c_int32
    L.mbr_debug_wait_limit.argtypes = [c_int32, c_int32, c_int32]
    L.mbr_debug_wait_limit.restype = c_int32
    L.mbr_last_error.argtypes = [c_void_p]
    L.mbr_last_error.restype = ctypes.c_char_p
    _lib = L
    return L
