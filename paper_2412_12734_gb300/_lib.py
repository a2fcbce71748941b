"""ctypes binding of ``libgbill.so`` (C ABI declared in include/gbill.h).

Argument marshalling only: every step of the rasterizer runs in the CUDA
library.  Loading fails loudly if the shared object is missing; there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
import re

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
LIB_PATH = os.path.join(PKG, "libgbill.so")
HEADER = os.path.join(ROOT, "include", "gbill.h")

GB_OK = 0
STATUS = {0: "GB_OK", 1: "GB_ERR_INVALID_ARG", 2: "GB_ERR_UNSUPPORTED", 3: "GB_ERR_CUDA",
          4: "GB_ERR_CAPACITY", 5: "GB_ERR_TIMEOUT", 6: "GB_ERR_NONFINITE"}
GB_F32, GB_F16, GB_BF16 = 0, 1, 2
GB_FLAG_NO_SYNC = 1
GB_FLAG_PERSISTENT = 2
GB_FLAG_TIMING = 4
PHASES = ("preprocess", "depth_sort", "count_scan", "emit", "tile_sort", "ranges", "render_fwd",
          "bwd_setup", "render_bwd", "preprocess_bwd")
MAX_CAMERAS = 64
MAX_SCENES = 16


class gb_camera(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32),
                ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("world_to_cam", C.c_float * 12), ("near_plane", C.c_float), ("scene", C.c_int32)]


class gb_scene(C.Structure):
    _fields_ = [("num_splats", C.c_int64),
                ("means", C.c_void_p), ("quats", C.c_void_p), ("scales", C.c_void_p),
                ("opacities", C.c_void_p), ("sh", C.c_void_p), ("textures", C.c_void_p),
                ("sh_degree", C.c_int32), ("sh_dtype", C.c_int32),
                ("tex_n", C.c_int32), ("tex_dtype", C.c_int32),
                ("sigma", C.c_float), ("mip_level", C.c_int32), ("tex_sh_degree", C.c_int32),
                ("reserved", C.c_int32), ("splat_tex_n", C.c_void_p)]


class gb_grads(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in
                ("d_means", "d_quats", "d_scales", "d_opacities", "d_sh", "d_textures")]


class gb_options(C.Structure):
    _fields_ = [("tile_size", C.c_int32), ("batch_depth", C.c_int32), ("flags", C.c_uint32),
                ("pixels_per_thread", C.c_int32), ("background", C.c_float * 3), ("batch_depth_fwd", C.c_int32),
                ("bwd_kernel", C.c_int32)]


class gb_adam_tensor(C.Structure):
    _fields_ = [("param", C.c_void_p), ("grad", C.c_void_p), ("m", C.c_void_p), ("v", C.c_void_p),
                ("shadow", C.c_void_p), ("shadow_dtype", C.c_int32), ("reserved", C.c_int32), ("n", C.c_int64)]


class gb_adam_config(C.Structure):
    _fields_ = [("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("step", C.c_int32), ("reserved", C.c_int32)]


class gb_stats(C.Structure):
    _fields_ = [("records", C.c_int64), ("visible", C.c_int64), ("instances", C.c_int64),
                ("tiles", C.c_int64), ("pixels", C.c_int64), ("capacity", C.c_int64),
                ("overflow", C.c_int32), ("error_flags", C.c_int32),
                ("pairs_fwd", C.c_int64), ("pairs_bwd", C.c_int64),
                ("blended_fwd", C.c_int64), ("contributing_bwd", C.c_int64)]


_lib = None


class GbillError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


def declared_symbols() -> list[str]:
    """Names of the functions declared in include/gbill.h."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(gb_\w+)\s*\(", text, re.M)))


_bound: tuple = ()


def signatures() -> tuple:
    """Names of the C entry points bound (with argument and result types) by load()."""
    load()
    return _bound


def load() -> C.CDLL:
    """Loads the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                           "(there is no CPU fallback)")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    sig = {
        "gb_context_create": (C.c_int, [i32, C.POINTER(vp)]),
        "gb_context_destroy": (C.c_int, [vp]),
        "gb_last_error": (C.c_char_p, [vp]),
        "gb_status_string": (C.c_char_p, [C.c_int]),
        "gb_saved_create": (C.c_int, [vp, C.POINTER(vp)]),
        "gb_saved_destroy": (C.c_int, [vp]),
        "gb_saved_reserve": (C.c_int, [vp, i64, i64, i64, i64]),
        "gb_saved_stats": (C.c_int, [vp, C.POINTER(gb_stats)]),
        "gb_saved_check": (C.c_int, [vp]),
        "gb_saved_phase_times": (C.c_int, [vp, C.POINTER(C.c_float), i32]),
        "gb_kernel_launches": (C.c_uint64, []),
        "gb_saved_export_keys": (C.c_int, [vp, vp, vp, vp, i64, C.POINTER(i64)]),
        "gb_saved_export_records": (C.c_int, [vp, vp, vp, vp, i64, C.POINTER(i64)]),
        "gb_render_forward": (C.c_int, [vp, vp, C.POINTER(gb_scene), i32, C.POINTER(gb_camera), i32,
                                        C.POINTER(gb_options), vp, vp, vp, vp]),
        "gb_render_backward": (C.c_int, [vp, vp, vp, vp, vp, C.POINTER(gb_grads), i32, vp]),
        "gb_adam_step": (C.c_int, [vp, C.POINTER(gb_adam_tensor), i32, C.POINTER(gb_adam_config), vp]),
        "gb_render_forward_noalloc": (C.c_int, [vp, C.POINTER(gb_scene), i32, C.POINTER(gb_camera), i32,
                                                C.POINTER(gb_options), vp, vp, vp, vp]),
        "gb_fit_params": (C.c_int, [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]),
        "gb_fit_params_backward": (C.c_int, [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]),
        "gb_mse_loss": (C.c_int, [vp, vp, vp, i64, vp, vp, vp]),
        "gb_autotune": (C.c_int, [vp, vp, C.POINTER(gb_scene), i32, C.POINTER(gb_camera), i32,
                                  C.POINTER(gb_options), i32, C.POINTER(gb_options), vp, vp, vp, vp, i32,
                                  C.POINTER(i32)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    global _bound
    _bound = tuple(sig)
    _lib = L
    return L


def check(status: int, ctx=None) -> None:
    if status != GB_OK:
        msg = load().gb_last_error(ctx).decode() if ctx else ""
        raise GbillError(status, msg)
