"""ctypes binding of libsplatloam (include/splatloam.h), argument marshalling only.

Every function here has the name of the C entry point it calls and forwards raw device pointers,
sizes and the stream handle.  Loading fails loudly when the library has not been built: there is
no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

_P = ctypes.c_void_p
_I = ctypes.c_int
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64


class splat_lidar_intrinsics(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int32), ("cols", ctypes.c_int32),
                ("elev_min", ctypes.c_float), ("elev_max", ctypes.c_float)]


class splat_gaussians(ctypes.Structure):
    _fields_ = [("pos_logit", _P), ("quat_wxyz", _P), ("log_scale", _P), ("n", _I64)]


class splat_render_config(ctypes.Structure):
    _fields_ = [("alpha_min", ctypes.c_float), ("alpha_max", ctypes.c_float),
                ("t_min", ctypes.c_float), ("sigma_cut", ctypes.c_float),
                ("tile_h", ctypes.c_int32), ("tile_w", ctypes.c_int32),
                ("work_cap", ctypes.c_int32), ("flip_normals", ctypes.c_int32)]


class splat_capacity(ctypes.Structure):
    _fields_ = [("max_gaussians", _I64), ("max_views", ctypes.c_int32), ("max_pixels", _I64),
                ("max_pairs", _I64), ("max_tiles", _I64)]


class splat_loss_config(ctypes.Structure):
    _fields_ = [("lambda_n", ctypes.c_float), ("lambda_o", ctypes.c_float),
                ("o_eps", ctypes.c_float), ("lambda_s", ctypes.c_float),
                ("tau_s", ctypes.c_float), ("normal_mode", ctypes.c_int32),
                ("rho_exp", ctypes.c_float)]


class splat_densify_config(ctypes.Structure):
    _fields_ = [("refine", ctypes.c_int32), ("lambda_do", ctypes.c_float),
                ("lambda_de", ctypes.c_float), ("w0", ctypes.c_float), ("w_cap", ctypes.c_float),
                ("scale_k", ctypes.c_float), ("opacity", ctypes.c_float),
                ("seed", ctypes.c_uint64)]


class splat_adam_config(ctypes.Structure):
    _fields_ = [("lr_pos", ctypes.c_float), ("lr_opacity", ctypes.c_float),
                ("lr_rot", ctypes.c_float), ("lr_scale", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float)]


class splat_stats(ctypes.Structure):
    _fields_ = [("n_pairs", _I64), ("fwd_evals", _I64), ("bwd_evals", _I64),
                ("n_pixels", _I64), ("n_tiles", _I64), ("kernel_launches", _I64),
                ("n_touching", _I64)]


SPLAT_OK = 0
SPLAT_STATUS_CAPACITY = 1
SPLAT_STATUS_NONFINITE = 2
SPLAT_STATUS_TIMEOUT = 4

# every symbol the header declares, with its ctypes signature
SIGNATURES = {
    "splat_version": ([], _I),
    "splat_error_string": ([_I], ctypes.c_char_p),
    "splat_last_cuda_error": ([], ctypes.c_char_p),
    "splat_default_config": ([ctypes.POINTER(splat_render_config)], None),
    "splat_ctx_create": ([ctypes.POINTER(splat_render_config), ctypes.POINTER(splat_capacity),
                          ctypes.POINTER(_P)], _I),
    "splat_ctx_destroy": ([_P], None),
    "splat_set_views": ([_P, _I32, _P, ctypes.POINTER(splat_lidar_intrinsics)], _I),
    "splat_view_pixel_offset": ([_P, _I32], _I64),
    "splat_render_views": ([_P, ctypes.POINTER(splat_gaussians), _P, _P, _P, _P], _I),
    "splat_render_views_backward": ([_P, ctypes.POINTER(splat_gaussians), _P, _P, _P, _P, _P, _P,
                                     _I, _P], _I),
    "splat_render": ([_P, ctypes.POINTER(splat_gaussians), _P,
                      ctypes.POINTER(splat_lidar_intrinsics), _P, _P, _P, _P], _I),
    "splat_render_backward": ([_P, ctypes.POINTER(splat_gaussians), _P, _P, _P, _P, _P, _P, _I,
                               _P], _I),
    "splat_loss": ([_P, _P, _P, _P, _P, _I64, ctypes.POINTER(splat_loss_config), _P, _P, _P, _P,
                    _P], _I),
    "splat_photometric": ([_P, _I32, _P, _P, _P, _P, ctypes.c_float, ctypes.c_float, _P, _P,
                           _P], _I),
    "splat_densify": ([_P] * 4 + [ctypes.POINTER(splat_densify_config), _I64] + [_P] * 3
                      + [_I64, _I64, _P], _I),
    "splat_view_loss": ([_P] * 6 + [ctypes.POINTER(splat_loss_config)] + [_P] * 5, _I),
    "splat_adam_step": ([_P] * 13 + [_I64, ctypes.POINTER(splat_adam_config), _P], _I),
    "splat_refine_step": ([_P, _P, _P, _P, _I64, _P, _P, ctypes.POINTER(splat_loss_config),
                           ctypes.POINTER(splat_adam_config)] + [_P] * 9, _I),
    "splat_backproject": ([_P, _P, _P, ctypes.c_float, _P, _P], _I),
    "splat_set_view_sampling": ([_P, _I, ctypes.c_double, ctypes.c_uint64], _I),
    "splat_get_active_views": ([_P, _P], _I),
    "splat_set_pose_gradient": ([_P, _I], _I),
    "splat_pose_gradient": ([_P, _P, _P], _I),
    "splat_get_status": ([_P, ctypes.POINTER(ctypes.c_uint32)], _I),
    "splat_get_stats": ([_P, ctypes.POINTER(splat_stats)], _I),
    "splat_debug_copy": ([_P, _I32, _P, _I64], _I64),
    "splat_stage_times": ([_P, _P], _I),
    "splat_set_profiling": ([_P, _I], _I),
    "splat_render_noalloc": ([ctypes.POINTER(splat_gaussians), _P,
                              ctypes.POINTER(splat_lidar_intrinsics),
                              ctypes.POINTER(splat_render_config), _P, _P, _P, _P], _I),
    "splat_kernel_times": ([_P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)],
                           _I),
}

_lib = None


class SplatError(RuntimeError):
    pass


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libsplatloam.so (building it first if it is missing and nvcc is present)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise SplatError(f"libsplatloam.so not built ({path}); run paper_2503_17491_gb300.build")
        _build.build()
    lib = ctypes.CDLL(path)
    for name, (args, res) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def check(code: int, what: str = ""):
    if code != SPLAT_OK:
        lib = load()
        msg = lib.splat_error_string(code).decode()
        if code == 2:
            msg += ": " + lib.splat_last_cuda_error().decode()
        raise SplatError(f"{what or 'splat call'} failed ({code}): {msg}")


def __getattr__(name):
    # splat_* names resolve to the raw C entry points
    if name.startswith("splat_") and name in SIGNATURES:
        return getattr(load(), name)
    raise AttributeError(name)
