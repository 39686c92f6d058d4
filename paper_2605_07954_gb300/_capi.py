"""ctypes declarations of include/stencil.h (argument marshalling only).

Every function here has the name and argument list of the C entry point it
wraps.  Loading fails loudly if the CUDA library has not been built: there is
no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libstencil_gb300.so")

STENCIL_OK = 0
STENCIL_ERR_INVALID_ARG = 1
STENCIL_ERR_UNSUPPORTED = 2
STENCIL_ERR_CUDA = 3
STENCIL_ERR_OOM = 4
STENCIL_ERR_TIMEOUT = 5
STENCIL_ERR_DEVICE_CHECK = 6

STENCIL_F32, STENCIL_BF16, STENCIL_F16 = 0, 1, 2
STENCIL_BOUNDARY_ZERO, STENCIL_BOUNDARY_PERIODIC = 0, 1
STENCIL_COMPUTE_AUTO, STENCIL_COMPUTE_FP32, STENCIL_COMPUTE_TC_TF32, STENCIL_COMPUTE_TC_BF16 = 0, 1, 2, 3
STENCIL_KERNEL_AUTO, STENCIL_KERNEL_NAIVE, STENCIL_KERNEL_STREAM = 0, 1, 2


class stencil_options_t(ctypes.Structure):
    _fields_ = [("compute", ctypes.c_int), ("kernel", ctypes.c_int), ("tb_depth", ctypes.c_int),
                ("threads", ctypes.c_int), ("tile_rows", ctypes.c_int), ("autotune", ctypes.c_int),
                ("mma_n", ctypes.c_int), ("timeout_ms", ctypes.c_int), ("debug_withhold", ctypes.c_int),
                ("load", ctypes.c_int), ("rank", ctypes.c_int)]


class stencil_plan_info_t(ctypes.Structure):
    _fields_ = [("ny", ctypes.c_int64), ("nx", ctypes.c_int64), ("radius", ctypes.c_int),
                ("shape", ctypes.c_int), ("dtype", ctypes.c_int), ("boundary", ctypes.c_int),
                ("compute", ctypes.c_int), ("kernel", ctypes.c_int), ("tb_depth", ctypes.c_int),
                ("threads", ctypes.c_int), ("halo_cols", ctypes.c_int), ("tile_cols", ctypes.c_int),
                ("tile_rows", ctypes.c_int), ("ctas", ctypes.c_int), ("smem_bytes", ctypes.c_int),
                ("workspace_bytes", ctypes.c_int64), ("mma_n", ctypes.c_int), ("load", ctypes.c_int),
                ("rank", ctypes.c_int)]


class stencil_grid_desc_t(ctypes.Structure):
    _fields_ = [("ny", ctypes.c_int64), ("nx", ctypes.c_int64), ("radius", ctypes.c_int),
                ("weights", ctypes.POINTER(ctypes.c_float)), ("boundary", ctypes.c_int),
                ("T", ctypes.c_int64), ("in_", ctypes.c_void_p), ("out", ctypes.c_void_p)]


class stencil_batch_options_t(ctypes.Structure):
    _fields_ = [("tb_depth", ctypes.c_int), ("threads", ctypes.c_int), ("tile_rows", ctypes.c_int),
                ("autotune", ctypes.c_int), ("timeout_ms", ctypes.c_int),
                ("debug_withhold_item", ctypes.c_int)]


class stencil_batch_info_t(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("tb_depth", ctypes.c_int), ("threads", ctypes.c_int),
                ("tiles", ctypes.c_int), ("items", ctypes.c_int64), ("launches", ctypes.c_int),
                ("ctas", ctypes.c_int), ("point_steps", ctypes.c_int64)]


class stencil_slab_info_t(ctypes.Structure):
    _fields_ = [("ny", ctypes.c_int64), ("nx", ctypes.c_int64), ("y0", ctypes.c_int64),
                ("y1", ctypes.c_int64), ("radius", ctypes.c_int), ("boundary", ctypes.c_int),
                ("steps_per_exchange", ctypes.c_int64), ("ghost_depth", ctypes.c_int64),
                ("ghost_above", ctypes.c_int64), ("ghost_below", ctypes.c_int64),
                ("buffer_rows", ctypes.c_int64), ("send_above_row", ctypes.c_int64),
                ("send_below_row", ctypes.c_int64), ("recv_above_row", ctypes.c_int64),
                ("recv_below_row", ctypes.c_int64)]


_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int
_PROTOS = {
    "stencil_plan_create": (_i32, [ctypes.POINTER(_vp), _i64, _i64, _i32,
                                   ctypes.POINTER(ctypes.c_float), _i32, _i32,
                                   ctypes.POINTER(stencil_options_t)]),
    "stencil_plan_destroy": (None, [_vp]),
    "stencil_plan_info": (_i32, [_vp, ctypes.POINTER(stencil_plan_info_t)]),
    "stencil_plan_set_weights": (_i32, [_vp, ctypes.POINTER(ctypes.c_float)]),
    "stencil_run": (_i32, [_vp, _vp, _vp, _i64, _vp]),
    "stencil_run_host": (_i32, [_vp, _vp, _vp, _i64, _vp]),
    "stencil_run_host_async": (_i32, [_vp, _vp, _vp, _i64, _vp]),
    "stencil_run_launches": (_i64, [_vp, _i64]),
    "stencil_plan_status": (_i32, [_vp]),
    "stencil_status_string": (ctypes.c_char_p, [_i32]),
    "stencil_last_error": (ctypes.c_char_p, []),
    "stencil_version": (_i32, []),
    "stencil_run_residual": (_i32, [_vp, _vp, _vp, _i64, _i64, _vp, _vp]),
    "stencil_residual_last_error": (ctypes.c_char_p, []),
    "stencil_adjoint": (_i32, [_vp, _vp, _vp, _i64, _vp, _vp, _i64, _vp]),
    "stencil_adjoint_launches": (_i64, [_vp, _i64, _i64]),
    "stencil_adjoint_last_error": (ctypes.c_char_p, []),
    "stencil_batch_create": (_i32, [ctypes.POINTER(_vp), _i32, ctypes.POINTER(stencil_grid_desc_t),
                                    _i32, ctypes.POINTER(stencil_batch_options_t)]),
    "stencil_run_batched": (_i32, [_vp, _vp]),
    "stencil_batch_status": (_i32, [_vp]),
    "stencil_batch_info": (_i32, [_vp, ctypes.POINTER(stencil_batch_info_t)]),
    "stencil_batch_destroy": (None, [_vp]),
    "stencil_batch_last_error": (ctypes.c_char_p, []),
    "stencil_run_noalloc": (_i32, [_i64, _i64, _i32, ctypes.POINTER(ctypes.c_float), _i32, _i32,
                                   _vp, _vp, _i64, _vp]),
    "stencil_noalloc_last_error": (ctypes.c_char_p, []),
    "stencil_slab_geometry": (_i32, [_i64, _i64, _i64, _i64, _i32, _i32, _i64,
                                     ctypes.POINTER(stencil_slab_info_t)]),
    "stencil_slab_create": (_i32, [ctypes.POINTER(_vp), _i64, _i64, _i64, _i64, _i32,
                                   ctypes.POINTER(ctypes.c_float), _i32, _i32, _i64,
                                   ctypes.POINTER(stencil_options_t)]),
    "stencil_slab_destroy": (None, [_vp]),
    "stencil_slab_info": (_i32, [_vp, ctypes.POINTER(stencil_slab_info_t)]),
    "stencil_slab_plan": (_vp, [_vp]),
    "stencil_slab_step": (_i32, [_vp, _vp, _i64, _vp]),
    "stencil_slab_last_error": (ctypes.c_char_p, []),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()'). "
            "There is no CPU fallback.")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _PROTOS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def declared_symbols(header: str | None = None) -> list[str]:
    """Function names declared in include/stencil.h."""
    import re
    header = header or os.path.join(os.path.dirname(HERE), "include", "stencil.h")
    text = open(header).read()
    decl = re.compile(r"^[A-Za-z_][A-Za-z0-9_ *]*?\b(stencil_[a-z0-9_]+)\s*\(", re.M)
    return sorted(set(decl.findall(text)))


class StencilError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load()
        name = lib.stencil_status_string(status).decode()
        if "residual" in where:
            msg = lib.stencil_residual_last_error().decode()
        elif "adjoint" in where:
            msg = lib.stencil_adjoint_last_error().decode()
        elif "batch" in where:
            msg = lib.stencil_batch_last_error().decode()
        elif "noalloc" in where:
            msg = lib.stencil_noalloc_last_error().decode()
        elif "slab" in where:
            msg = lib.stencil_slab_last_error().decode()
        else:
            msg = lib.stencil_last_error().decode()
        super().__init__(f"{where}: {name}: {msg}")
        self.status = status


def check(status: int, where: str):
    if status != STENCIL_OK:
        raise StencilError(status, where)


def __getattr__(name):
    if name in _PROTOS:
        return getattr(load(), name)
    raise AttributeError(name)
