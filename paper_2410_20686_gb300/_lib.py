"""ctypes mirror of ``include/odgs.h`` (argument marshalling only).

Loading fails loudly if ``libodgs.so`` has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libodgs.so")

ODGS_OK = 0
ODGS_ERR_INVALID_ARG, ODGS_ERR_CAPACITY, ODGS_ERR_CUDA, ODGS_ERR_TIMEOUT, ODGS_ERR_NONFINITE = -1, -2, -3, -4, -5
ODGS_ERR_STATE, ODGS_ERR_WORKSPACE = -6, -7
STATUS_NAMES = {0: "ODGS_OK", -1: "ODGS_ERR_INVALID_ARG", -2: "ODGS_ERR_CAPACITY", -3: "ODGS_ERR_CUDA",
                -4: "ODGS_ERR_TIMEOUT", -5: "ODGS_ERR_NONFINITE", -6: "ODGS_ERR_STATE", -7: "ODGS_ERR_WORKSPACE"}
DEV_CAPACITY = 1
DEV_TIMEOUT = 2
DEV_NONFINITE = 4
MAX_VIEWS = 64

# every symbol include/odgs.h declares
EXPORTED = ("odgs_create", "odgs_destroy", "odgs_workspace_size", "odgs_pair_buffer_size",
            "odgs_preprocess", "odgs_query_pairs", "odgs_bin_sort", "odgs_render_fwd",
            "odgs_render_bwd", "odgs_preprocess_bwd", "odgs_frame_stats", "odgs_get_status",
            "odgs_render_fwd_static", "odgs_measure_peaks", "odgs_last_launch_count", "odgs_status_string",
            "odgs_densify_select", "odgs_densify_scratch_size", "odgs_densify_apply", "odgs_adam_step",
            "odgs_loss_scratch_size", "odgs_loss_l1_dssim", "odgs_set_wait_limit", "odgs_debug_lists",
            "odgs_debug_screen_grads")


class OdgsError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)} ({status_string(status)})")


class View(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("R_wc", C.c_float * 9), ("t_wc", C.c_float * 3),
                ("model", C.c_int), ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float)]


class Settings(C.Structure):
    _fields_ = [("sh_degree", C.c_int), ("sh_coeffs", C.c_int), ("tile_w", C.c_int), ("tile_h", C.c_int),
                ("batch", C.c_int), ("cov_dilation", C.c_float), ("r_near", C.c_float), ("r_far", C.c_float),
                ("bg", C.c_float * 3), ("recompute_lists", C.c_int), ("grad_accumulate", C.c_int),
                ("pixels_per_thread", C.c_int), ("raw_params", C.c_int), ("pixels_per_thread_bwd", C.c_int),
                ("checked", C.c_int), ("full_lists", C.c_int)]


class Gaussians(C.Structure):
    _fields_ = [("means", C.c_void_p), ("scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity", C.c_void_p), ("sh", C.c_void_p), ("n", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("pairs", C.c_uint64), ("pairs_sorted", C.c_uint64), ("evals_fwd", C.c_uint64),
                ("evals_bwd", C.c_uint64), ("blended", C.c_uint64), ("entries_tile", C.c_uint64),
                ("visible", C.c_uint64), ("status", C.c_uint32)]


class DensifyParams(C.Structure):
    _fields_ = [("tau_min", C.c_float), ("tau_max", C.c_float), ("percent_dense", C.c_float),
                ("scene_extent", C.c_float), ("min_opacity", C.c_float), ("max_scale", C.c_float),
                ("raw_params", C.c_int)]


class ParamsOut(C.Structure):
    _fields_ = [("means", C.c_void_p), ("scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity", C.c_void_p), ("sh", C.c_void_p)]


class AdamGroup(C.Structure):
    _fields_ = [("param", C.c_void_p), ("grad", C.c_void_p), ("m", C.c_void_p), ("v", C.c_void_p),
                ("count", C.c_size_t), ("lr", C.c_float), ("lr_tail", C.c_float), ("row", C.c_int),
                ("head", C.c_int)]


class AdamParams(C.Structure):
    _fields_ = [("beta1", C.c_double), ("beta2", C.c_double), ("eps", C.c_double), ("step", C.c_int)]


class LossParams(C.Structure):
    _fields_ = [("lambda_", C.c_float), ("area_weight", C.c_int), ("wrap_u", C.c_int), ("accumulate", C.c_int)]


class Peaks(C.Structure):
    _fields_ = [("ffma_tflops", C.c_double), ("ex2_gops", C.c_double), ("sms", C.c_int)]


class Grads(C.Structure):
    _fields_ = [("means", C.c_void_p), ("scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity", C.c_void_p), ("sh", C.c_void_p), ("densify_grad", C.c_void_p),
                ("densify_elev", C.c_void_p), ("densify_count", C.c_void_p)]


_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"ODGS CUDA library not built: {path} is missing (run "
                          f"paper_2410_20686_gb300.build.build())")
    L = C.CDLL(path)
    vp, sz = C.c_void_p, C.c_size_t
    L.odgs_create.argtypes = [C.POINTER(C.c_void_p)]
    L.odgs_destroy.argtypes = [vp]
    L.odgs_destroy.restype = None
    L.odgs_workspace_size.argtypes = [C.c_int, C.POINTER(View), C.c_int, C.POINTER(Settings), C.POINTER(sz)]
    L.odgs_pair_buffer_size.argtypes = [sz, C.POINTER(sz)]
    L.odgs_preprocess.argtypes = [vp, C.POINTER(Gaussians), C.POINTER(View), C.c_int, C.POINTER(Settings),
                                  vp, sz, vp]
    L.odgs_query_pairs.argtypes = [vp, C.POINTER(sz), vp]
    L.odgs_bin_sort.argtypes = [vp, vp, sz, vp]
    L.odgs_render_fwd.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), vp]
    L.odgs_render_bwd.argtypes = [vp, C.POINTER(vp), vp]
    L.odgs_preprocess_bwd.argtypes = [vp, C.POINTER(Grads), vp]
    L.odgs_frame_stats.argtypes = [vp, C.POINTER(Stats), vp]
    L.odgs_get_status.argtypes = [vp, C.POINTER(C.c_uint32), vp]
    L.odgs_render_fwd_static.argtypes = [C.POINTER(Gaussians), C.POINTER(View), C.POINTER(Settings), vp, vp, vp, vp]
    L.odgs_measure_peaks.argtypes = [C.POINTER(Peaks), vp]
    L.odgs_densify_select.argtypes = [vp, vp, vp, vp, vp, C.c_int, C.POINTER(DensifyParams), vp, vp]
    L.odgs_densify_scratch_size.argtypes = [C.c_int, C.POINTER(sz)]
    L.odgs_adam_step.argtypes = [C.POINTER(AdamGroup), C.c_int, C.POINTER(AdamParams), vp]
    L.odgs_loss_scratch_size.argtypes = [C.c_int, C.c_int, C.POINTER(sz)]
    L.odgs_loss_l1_dssim.argtypes = [vp, vp, C.c_int, C.c_int, C.POINTER(LossParams), vp, vp, vp, sz, vp]
    L.odgs_densify_apply.argtypes = [C.POINTER(Gaussians), C.c_int, C.c_int, vp, vp, C.POINTER(ParamsOut), C.c_int,
                                     vp, vp, sz, vp]
    L.odgs_set_wait_limit.argtypes = [vp, C.c_uint32]
    L.odgs_debug_lists.argtypes = [vp, vp, vp, sz, vp, vp, sz, vp, sz, vp]
    L.odgs_debug_screen_grads.argtypes = [vp, vp, sz, vp]
    L.odgs_last_launch_count.argtypes = [vp]
    L.odgs_last_launch_count.restype = C.c_int
    L.odgs_status_string.argtypes = [C.c_int]
    L.odgs_status_string.restype = C.c_char_p
    for name in ("odgs_create", "odgs_workspace_size", "odgs_pair_buffer_size", "odgs_preprocess",
                 "odgs_query_pairs", "odgs_bin_sort", "odgs_render_fwd", "odgs_render_bwd",
                 "odgs_preprocess_bwd", "odgs_frame_stats", "odgs_get_status", "odgs_render_fwd_static",
                 "odgs_measure_peaks", "odgs_densify_select", "odgs_densify_scratch_size", "odgs_densify_apply",
                 "odgs_adam_step", "odgs_loss_scratch_size", "odgs_loss_l1_dssim", "odgs_set_wait_limit",
                 "odgs_debug_lists", "odgs_debug_screen_grads"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def status_string(st: int) -> str:
    try:
        return load().odgs_status_string(int(st)).decode()
    except ImportError:
        return STATUS_NAMES.get(st, str(st))


def check(st: int, where: str):
    if st != ODGS_OK:
        raise OdgsError(st, where)


def make_view(width, height, R_wc, t_wc, model=0, fx=0.0, fy=0.0, cx=0.0, cy=0.0) -> View:
    """model 0: ERP; model 1: pinhole with focal lengths fx, fy and principal point cx, cy (pixels)."""
    v = View()
    v.width, v.height = int(width), int(height)
    v.R_wc[:] = [float(x) for x in list(_flat(R_wc))]
    v.t_wc[:] = [float(x) for x in list(_flat(t_wc))]
    v.model = int(model)
    v.fx, v.fy, v.cx, v.cy = float(fx), float(fy), float(cx), float(cy)
    return v


def _flat(a):
    try:
        import numpy as np
        return np.asarray(a, dtype=np.float32).ravel().tolist()
    except Exception:  # pragma: no cover
        return list(a)
