"""ctypes declarations of the C ABI in include/rt.h (argument marshalling only).

Loading fails loudly when the CUDA library is missing or no GPU is visible:
there is no CPU fallback.
"""
import ctypes
import os

from . import build as _build

RT_OK, RT_ERR_ARG, RT_ERR_MESH, RT_ERR_CUDA, RT_ERR_OOM = 0, -1, -2, -3, -4
RT_ERR_CFL, RT_ERR_NONCONV, RT_ERR_NONFINITE, RT_ERR_STATE = -5, -6, -7, -8
RT_FP64, RT_FP32 = 0, 1
RT_FIRST_ORDER, RT_VAN_LEER = 0, 1
_NAMES = {0: "RT_OK", -1: "RT_ERR_ARG", -2: "RT_ERR_MESH", -3: "RT_ERR_CUDA", -4: "RT_ERR_OOM",
          -5: "RT_ERR_CFL", -6: "RT_ERR_NONCONV", -7: "RT_ERR_NONFINITE", -8: "RT_ERR_STATE"}

# every symbol include/rt.h declares (checked by the CPU tests)
EXPORTS = ["rt_create", "rt_set_gas", "rt_set_gas_energy", "rt_set_cells", "rt_set_intensity", "rt_get_intensity",
           "rt_get_gas", "rt_dt_limits", "rt_step", "rt_step_io", "rt_run", "rt_launch", "rt_moments", "rt_totals", "rt_totals_noalloc",
           "rt_sync", "rt_adjoint_step", "rt_hydro_step", "rt_hydro_dt", "rt_radhydro_step",
           "rt_get_density", "rt_get_state", "rt_set_state", "rt_device_bytes", "rt_launch_count",
           "rt_last_error", "rt_destroy"]


class RTError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class MeshDesc(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_int64), ("n_faces", ctypes.c_int64),
                ("n_angles", ctypes.c_int32), ("n_groups", ctypes.c_int32),
                ("cell_volume", ctypes.c_void_p), ("cell_centroid", ctypes.c_void_p),
                ("face_cells", ctypes.c_void_p), ("face_area", ctypes.c_void_p),
                ("face_normal", ctypes.c_void_p), ("face_centroid", ctypes.c_void_p),
                ("face_w", ctypes.c_void_p), ("cell_face_ptr", ctypes.c_void_p),
                ("cell_face_idx", ctypes.c_void_p), ("angle_dir", ctypes.c_void_p),
                ("angle_w", ctypes.c_void_p), ("face_offset", ctypes.c_void_p),
                ("group_w", ctypes.c_void_p)]


class Params(ctypes.Structure):
    _fields_ = [("cbar", ctypes.c_double), ("c", ctypes.c_double), ("a_rad", ctypes.c_double),
                ("gamma_gas", ctypes.c_double), ("r_gas", ctypes.c_double),
                ("cfl", ctypes.c_double), ("precision", ctypes.c_int32),
                ("newton_max_iter", ctypes.c_int32), ("integrator", ctypes.c_int32),
                ("boost", ctypes.c_int32), ("gcl", ctypes.c_int32), ("plain_launches", ctypes.c_int32),
                ("beta_P", ctypes.c_double), ("beta_J", ctypes.c_double), ("T_ref", ctypes.c_double),
                ("float_quartic", ctypes.c_int32), ("hydro", ctypes.c_int32)]


_lib = None


def lib_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load librt_gb300.so (building it first if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library {path} is missing; run paper_2002_08377_gb300.build")
        _build.build()
    L = ctypes.CDLL(path)
    vp, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    pd = ctypes.POINTER(ctypes.c_double)
    sig = {
        "rt_create": ([ctypes.POINTER(MeshDesc), ctypes.POINTER(Params), vp, ctypes.POINTER(vp)], i32),
        "rt_set_gas": ([vp] * 7, i32),
        "rt_set_gas_energy": ([vp, vp, vp, i32], i32),
        "rt_set_cells": ([vp, vp, vp, vp, vp, vp, i64, vp], i32),
        "rt_set_intensity": ([vp, vp, i32], i32),
        "rt_get_intensity": ([vp, vp, i32], i32),
        "rt_get_gas": ([vp, vp, vp, vp, i32], i32),
        "rt_dt_limits": ([vp, pd, pd], i32),
        "rt_step": ([vp, d, pd], i32),
        "rt_step_io": ([vp, d, vp, vp], i32),
        "rt_run": ([vp, i32, d, pd], i32),
        "rt_launch": ([vp, i32, d, pd], i32),
        "rt_moments": ([vp, vp, vp, vp, i32], i32),
        "rt_totals": ([vp, vp], i32),
        "rt_totals_noalloc": ([vp, vp], i32),
        "rt_sync": ([vp], i32),
        "rt_hydro_step": ([vp, d, i32], i32),
        "rt_hydro_dt": ([vp, d, pd], i32),
        "rt_radhydro_step": ([vp, d, i32, i32, pd], i32),
        "rt_get_density": ([vp, vp, i32], i32),
        "rt_adjoint_step": ([vp, d] + [vp] * 11 + [i32], i32),
        "rt_get_state": ([vp, vp, ctypes.POINTER(ctypes.c_size_t)], i32),
        "rt_set_state": ([vp, vp, ctypes.c_size_t], i32),
        "rt_device_bytes": ([vp, ctypes.POINTER(ctypes.c_size_t)], i32),
        "rt_launch_count": ([vp], i64),
        "rt_last_error": ([vp], ctypes.c_char_p),
        "rt_destroy": ([vp], None),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def check(state, code):
    if code != RT_OK:
        msg = load().rt_last_error(state).decode() if state else ""
        raise RTError(code, msg)
    return code
