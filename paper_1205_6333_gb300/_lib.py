"""ctypes declarations of the C ABI in include/sd.h (libsd_gb300.so).

Loading fails loudly when the shared library is missing or was built for
another machine: there is no CPU fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# SD_LIBRARY selects another build of the library, e.g. the debug build
# libsd_gb300_debug.so (device-side index checks) that the tests load in a subprocess.
LIB_PATH = os.environ.get("SD_LIBRARY") or os.path.join(HERE, "libsd_gb300.so")

c_int32, c_int64, c_double, c_void_p, c_char_p = (ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                                                  ctypes.c_void_p, ctypes.c_char_p)

ALLOC_FN = ctypes.CFUNCTYPE(c_void_p, ctypes.c_size_t, c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, c_void_p, c_void_p)

# sd_status
SD_OK, SD_ERR_ARG, SD_ERR_CUDA, SD_ERR_OOM, SD_ERR_COINCIDENT, SD_ERR_NONFINITE, SD_ERR_TIMEOUT, \
    SD_ERR_STATE, SD_ERR_UNSUPPORTED, SD_ERR_INTERNAL = range(10)
STATUS_NAMES = ["SD_OK", "SD_ERR_ARG", "SD_ERR_CUDA", "SD_ERR_OOM", "SD_ERR_COINCIDENT", "SD_ERR_NONFINITE",
                "SD_ERR_TIMEOUT", "SD_ERR_STATE", "SD_ERR_UNSUPPORTED", "SD_ERR_INTERNAL"]
SD_TENSOR_RPY, SD_TENSOR_RP, SD_TENSOR_OSEEN = 0, 1, 2
SD_PREC_FP32C, SD_PREC_FP64, SD_PREC_FP32 = 0, 1, 2
SD_DTYPE_F32, SD_DTYPE_F64 = 0, 1
SD_DENSE_AUTO, SD_DENSE_DIRECTED, SD_DENSE_SYMMETRIC = 0, 1, 2
SD_KERNEL_DENSE, SD_KERNEL_EPILOGUE, SD_KERNEL_CELLS, SD_KERNEL_FORCES, SD_KERNEL_BATCHED, SD_KERNEL_VJP, \
    SD_KERNEL_NEAR = range(7)


class sd_config(ctypes.Structure):
    _fields_ = [
        ("n", c_int32),
        ("a", c_double),
        ("eta", c_double),
        ("tensor", c_int32),
        ("prec", c_int32),
        ("box", c_double * 3),
        ("r_near", c_double),
        ("rep_eps", c_double),
        ("rep_rc", c_double),
        ("gravity", c_double * 3),
        ("device", c_int32),
        ("stream", c_void_p),
        ("alloc", ALLOC_FN),
        ("free", FREE_FN),
        ("alloc_ctx", c_void_p),
        ("dense_kernel", c_int32),
        ("lubrication", c_int32),
        ("verlet_skin", c_double),
    ]


# name -> (restype, argtypes); every symbol include/sd.h declares
PROTOTYPES = {
    "sd_config_init": (None, [ctypes.POINTER(sd_config)]),
    "sd_create": (c_int32, [ctypes.POINTER(sd_config), ctypes.POINTER(c_void_p)]),
    "sd_destroy": (None, [c_void_p]),
    "sd_set_positions": (c_int32, [c_void_p, c_void_p, c_int32]),
    "sd_get_positions": (c_int32, [c_void_p, c_void_p, c_int32]),
    "sd_set_forces": (c_int32, [c_void_p, c_void_p, c_int32]),
    "sd_mobility_apply": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int32]),
    "sd_step": (c_int32, [c_void_p, c_double, c_int64]),
    "sd_synchronize": (c_int32, [c_void_p]),
    "sd_mobility_vjp": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_int32]),
    "sd_adjoint": (c_int32, [c_void_p, c_double, c_int64, c_int32, c_void_p, c_void_p, c_void_p, c_int32]),
    "sd_batch_create": (c_int32, [ctypes.POINTER(sd_config), c_void_p, c_int32, ctypes.POINTER(c_void_p)]),
    "sd_batch_destroy": (None, [c_void_p]),
    "sd_batch_set_positions": (c_int32, [c_void_p, c_void_p, c_int32]),
    "sd_batch_get_positions": (c_int32, [c_void_p, c_void_p, c_int32]),
    "sd_batch_set_forces": (c_int32, [c_void_p, c_void_p, c_int32]),
    "sd_step_batched": (c_int32, [c_void_p, c_double, c_int64]),
    "sd_batch_autotune": (c_int32, [c_void_p, ctypes.POINTER(c_int32)]),
    "sd_batch_synchronize": (c_int32, [c_void_p]),
    "sd_batch_shape_count": (c_int32, [c_void_p]),
    "sd_batch_shape_info": (c_int32, [c_void_p, c_int32, ctypes.POINTER(c_int32), ctypes.POINTER(c_int32),
                                      ctypes.POINTER(c_int32)]),
    "sd_batch_set_shape": (c_int32, [c_void_p, c_int32]),
    "sd_profile": (c_int32, [c_void_p, c_int32]),
    "sd_batch_profile": (c_int32, [c_void_p, c_int32]),
    "sd_profile_read": (c_int32, [c_void_p, c_int32, ctypes.POINTER(c_double), ctypes.POINTER(c_int64)]),
    "sd_batch_profile_read": (c_int32, [c_void_p, c_int32, ctypes.POINTER(c_double), ctypes.POINTER(c_int64)]),
    "sd_launch_count": (c_int64, [c_void_p]),
    "sd_dense_kernel_used": (c_int32, [c_void_p]),
    "sd_mobility_apply_rows": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32]),
    "sd_step_rows": (c_int32, [c_void_p, c_double, c_int32, c_int32]),
    "sd_mobility_apply_part": (c_int32, [c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32, c_void_p]),
    "sd_mobility_apply_combine": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_int32, c_int32]),
    "sd_step_part": (c_int32, [c_void_p, c_int32, c_int32, c_void_p]),
    "sd_step_combine": (c_int32, [c_void_p, c_double, c_void_p, c_int32]),
    "sd_batch_launch_count": (c_int64, [c_void_p]),
    "sd_set_watchdog": (c_int32, [c_void_p, c_int64]),
    "sd_inject_stall": (c_int32, [c_void_p, c_int32]),
    "sd_mobility_apply_noalloc": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_double, c_double, c_int32,
                                            c_void_p]),
    "sd_access_run": (c_int32, [c_int32, c_int32, c_int32, c_int32, c_int32, c_void_p, c_void_p, c_void_p]),
    "sd_access_status": (c_int32, []),
    "sd_last_error": (c_char_p, []),
    "sd_version": (c_char_p, []),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libsd_gb300.so (building it first if the toolkit is present and it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        from . import build as _build
        _build.build()
    if not os.path.exists(path):
        raise ImportError("libsd_gb300.so is missing; run paper_1205_6333_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
