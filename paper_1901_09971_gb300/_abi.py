"""ctypes declarations of libdegraf.so (the C ABI in include/degraf.h).

Loading never falls back to anything: a missing or unloadable library raises.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

DGF_OK = 0
DGF_ERR_ARG = -1
DGF_ERR_WORKSPACE = -2
DGF_ERR_LEVELS = -3
DGF_ERR_CUDA = -4
DGF_ERR_TIMEOUT = -5
DGF_ERR_DEVICE = -6

TRACKED, OOB, SMALL_EIG, SINGULAR, MAXITER, FB_REJECTED = 0, 1, 2, 3, 4, 5
F32, F16 = 0, 1
STAGE_DETECT, STAGE_PYRAMID, STAGE_TRACK, STAGE_ALL = 1, 2, 4, 7
MAX_LEVELS = 6
MAX_RADIUS = 7
RLOF_PARAMS_VERSION = 2
GM_PARAMS_VERSION = 1
EPIC_PARAMS_VERSION = 1
EPIC_MAX_K = 256
DGF_NOALLOC_SCRATCH_BYTES = 24 << 20  # scratch of rlof_track_pair_noalloc
PYR_APRON = 12  # replicated border of every pyramid plane (pixels)

# Every entry point that include/degraf.h declares.
EXPORTS = (
    "dgf_strerror", "dgf_version", "dgf_degraf_count", "degraf_detect", "dgf_pyramid_layout_get",
    "dgf_pyramid_bytes", "pyramid_build", "dgf_rlof_params_default", "dgf_rlof_set_lanes", "rlof_track",
    "dgf_track_many_workspace", "rlof_track_many", "rlof_track_pair_noalloc",
    "dgf_degraf_backward_workspace", "degraf_detect_backward", "dgf_rlof_backward_workspace", "rlof_track_backward",
    "dgf_gm_params_default", "dgf_gm_workspace", "rlof_track_gm", "dgf_fb_workspace", "rlof_track_fb",
    "dgf_epic_params_default", "dgf_epic_workspace", "epic_interpolate",
    "dgf_fp32_probe", "dgf_fp32_probe_flops", "dgf_epic_exp_neg", "dgf_device_status",
)


class PyramidLayout(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("storage", ctypes.c_int), ("with_grad", ctypes.c_int),
                ("W", ctypes.c_int * MAX_LEVELS), ("H", ctypes.c_int * MAX_LEVELS),
                ("pitch", ctypes.c_int * MAX_LEVELS),
                ("off_I", ctypes.c_size_t * MAX_LEVELS), ("off_Ix", ctypes.c_size_t * MAX_LEVELS),
                ("off_Iy", ctypes.c_size_t * MAX_LEVELS), ("bytes", ctypes.c_size_t)]


class RlofParamsC(ctypes.Structure):
    _fields_ = [("version", ctypes.c_int), ("levels", ctypes.c_int), ("radius", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("model", ctypes.c_int), ("storage", ctypes.c_int),
                ("eps", ctypes.c_float), ("hampel_a", ctypes.c_float), ("hampel_b", ctypes.c_float),
                ("hampel_c", ctypes.c_float), ("min_eig", ctypes.c_float), ("cross_tau", ctypes.c_float)]


class GmParamsC(ctypes.Structure):
    _fields_ = [("version", ctypes.c_int), ("stride", ctypes.c_int), ("extra_levels", ctypes.c_int),
                ("iters", ctypes.c_int), ("c0", ctypes.c_double), ("c_min", ctypes.c_double)]


class EpicParamsC(ctypes.Structure):
    _fields_ = [("version", ctypes.c_int), ("k", ctypes.c_int), ("model", ctypes.c_int), ("cost_base", ctypes.c_int),
                ("cost_gain", ctypes.c_int), ("a", ctypes.c_double), ("min_spread", ctypes.c_double)]


class EpicDebugC(ctypes.Structure):
    _fields_ = [("labels", ctypes.c_void_p), ("dist", ctypes.c_void_p), ("knn_idx", ctypes.c_void_p),
                ("knn_dist", ctypes.c_void_p), ("knn_count", ctypes.c_void_p), ("models", ctypes.c_void_p),
                ("fit_kind", ctypes.c_void_p), ("retried", ctypes.c_void_p)]


class PairC(ctypes.Structure):
    _fields_ = [("frame1", ctypes.c_void_p), ("frame2", ctypes.c_void_p), ("W", ctypes.c_int),
                ("H", ctypes.c_int), ("pitch", ctypes.c_int), ("win", ctypes.c_int), ("step", ctypes.c_int),
                ("pts", ctypes.c_void_p), ("flow", ctypes.c_void_p), ("status", ctypes.c_void_p),
                ("iters", ctypes.c_void_p)]


class DegrafError(RuntimeError):
    def __init__(self, fn: str, code: int, msg: str):
        super().__init__(f"{fn} failed: {msg} ({code})")
        self.code = code


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libdegraf.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libdegraf.so not found at {path}; run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    P, I, Z, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_longlong
    L.dgf_strerror.argtypes, L.dgf_strerror.restype = [I], ctypes.c_char_p
    L.dgf_version.argtypes, L.dgf_version.restype = [], I
    L.dgf_degraf_count.argtypes, L.dgf_degraf_count.restype = [I, I, I, I, I], LL
    L.degraf_detect.argtypes, L.degraf_detect.restype = [P, I, I, I, I, I, I, P, P, P], I
    L.dgf_pyramid_layout_get.argtypes = [I, I, I, I, I, ctypes.POINTER(PyramidLayout)]
    L.dgf_pyramid_layout_get.restype = I
    L.dgf_pyramid_bytes.argtypes, L.dgf_pyramid_bytes.restype = [I, I, I, I, I], Z
    L.pyramid_build.argtypes, L.pyramid_build.restype = [P, I, I, I, I, I, I, P, Z, P], I
    L.dgf_rlof_params_default.argtypes = [ctypes.POINTER(RlofParamsC)]
    L.dgf_rlof_params_default.restype = None
    L.dgf_rlof_set_lanes.argtypes, L.dgf_rlof_set_lanes.restype = [I], I
    L.rlof_track.argtypes = [P, P, I, I, P, I, ctypes.POINTER(RlofParamsC), P, P, P, P, P]
    L.rlof_track.restype = I
    L.dgf_track_many_workspace.argtypes = [ctypes.POINTER(PairC), I, ctypes.POINTER(RlofParamsC)]
    L.dgf_track_many_workspace.restype = Z
    L.rlof_track_many.argtypes = [ctypes.POINTER(PairC), I, ctypes.POINTER(RlofParamsC), P, Z, I, I, P]
    L.rlof_track_many.restype = I
    L.dgf_degraf_backward_workspace.argtypes = [I, I, I, I, I]
    L.dgf_degraf_backward_workspace.restype = Z
    L.degraf_detect_backward.argtypes = [P, I, I, I, I, I, I, P, P, Z, P, I, P]
    L.degraf_detect_backward.restype = I
    L.dgf_rlof_backward_workspace.argtypes = [I, I]
    L.dgf_rlof_backward_workspace.restype = Z
    L.rlof_track_backward.argtypes = [P, P, I, I, P, I, ctypes.POINTER(RlofParamsC), P, P, P, P, P, P, Z, P, P, I, P]
    L.rlof_track_backward.restype = I
    L.rlof_track_pair_noalloc.argtypes = [ctypes.POINTER(PairC), ctypes.POINTER(RlofParamsC), P]
    L.rlof_track_pair_noalloc.restype = I
    L.dgf_gm_params_default.argtypes = [ctypes.POINTER(GmParamsC)]
    L.dgf_gm_params_default.restype = None
    L.dgf_gm_workspace.argtypes, L.dgf_gm_workspace.restype = [I, ctypes.POINTER(GmParamsC)], Z
    L.rlof_track_gm.argtypes = [P, P, I, I, I, P, I, ctypes.POINTER(RlofParamsC), ctypes.POINTER(GmParamsC), P, P, P,
                                P, P, Z, P]
    L.rlof_track_gm.restype = I
    L.dgf_fb_workspace.argtypes, L.dgf_fb_workspace.restype = [I], Z
    L.rlof_track_fb.argtypes = [P, P, Z, I, I, P, I, ctypes.POINTER(RlofParamsC), ctypes.c_float, P, P, P, P, Z, P]
    L.rlof_track_fb.restype = I
    L.dgf_epic_params_default.argtypes, L.dgf_epic_params_default.restype = [ctypes.POINTER(EpicParamsC)], I
    L.dgf_epic_workspace.argtypes, L.dgf_epic_workspace.restype = [I, I, I], Z
    L.epic_interpolate.argtypes = [P, I, I, I, P, P, P, I, ctypes.POINTER(EpicParamsC), P, ctypes.POINTER(EpicDebugC),
                                   P, Z, P]
    L.epic_interpolate.restype = I
    L.dgf_fp32_probe.argtypes, L.dgf_fp32_probe.restype = [P, I, I, I, I, P], I
    L.dgf_fp32_probe_flops.argtypes, L.dgf_fp32_probe_flops.restype = [I, I, I, I], ctypes.c_double
    L.dgf_epic_exp_neg.argtypes, L.dgf_epic_exp_neg.restype = [P, P, I, P], I
    L.dgf_device_status.argtypes, L.dgf_device_status.restype = [ctypes.POINTER(ctypes.c_uint), I], I
    _lib = L
    return L


def check(fn: str, rc: int) -> None:
    if rc != DGF_OK:
        raise DegrafError(fn, rc, load().dgf_strerror(rc).decode())
