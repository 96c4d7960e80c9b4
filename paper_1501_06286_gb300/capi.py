"""ctypes declarations of the C ABI in include/qmc.h (argument marshalling only).

The shared library is built in-tree by ``paper_1501_06286_gb300.build``.
Loading fails loudly when it is missing: there is no CPU fallback.
"""

from __future__ import annotations

import ctypes as C
import os

from . import build as _build

QMC_OK = 0
STATUS = {0: "QMC_OK", 1: "QMC_ERR_INVALID", 2: "QMC_ERR_NOT_PRIME", 3: "QMC_ERR_NOT_PRIMITIVE",
          4: "QMC_ERR_GENERATOR", 5: "QMC_ERR_SHAPE", 6: "QMC_ERR_UNSUPPORTED", 7: "QMC_ERR_ALLOC",
          8: "QMC_ERR_CUDA", 9: "QMC_ERR_TIMEOUT", 10: "QMC_ERR_DEVICE", 11: "QMC_ERR_SCRATCH",
          12: "QMC_ERR_NONFINITE", 13: "QMC_ERR_BOUNDS"}

KIND = {"prime": 0, "f2": 1, "pset": 2, "fb": 3}
MAP = {"identity": 0, "centred": 1, "phi_inv": 2, "tent": 3}
ROW0 = {"auto": 0, "include": 1, "exclude": 2}
ORDER = {"conventional": 0, "circulant": 1}
PREC = {"fp32": 0, "fp32_split": 1}
DTYPE_F32, DTYPE_F64 = 0, 1
TABLE = {"pow": 0, "log": 1, "exponents": 2, "out_row": 3, "zeta": 4, "spectrum64": 5,
         "row_ptr": 6, "jlist": 7}

EXPORTS = ["qmc_plan_create", "qmc_plan_destroy", "qmc_plan_info", "qmc_plan_exponents",
           "qmc_plan_copy_table", "qmc_plan_reserve", "qmc_plan_sync_status", "qmc_matmul",
           "qmc_matmul_backward", "qmc_generate_points", "qmc_batch_create", "qmc_batch_matmul",
           "qmc_batch_destroy", "qmc_status_string", "qmc_version", "qmc_plan_set_profiling",
           "qmc_plan_read_profile", "qmc_kernel_launches", "qmc_plan_set_option", "qmc_matmul_noalloc", "qmc_matmul_affine", "qmc_batch_set_option",
           "qmc_batch_sync_status", "qmc_fe_work_bytes", "qmc_fe_solve_mean"]
BATCH_OPT = {"mode": 0, "branches": 1, "wait_limit_us": 2, "test_block_item": 3}
BATCH_MODE = {"graph": 0, "persistent": 1}
OPT_PASS_KERNEL = 0
OPT_ROW_MEAN = 1
OPT_FIRST_PASS = 2
OPT_FFT_SPLIT = 3
ROW_MEAN = {"linear": 0, "fused": 1}
FIRST_PASS = {"auto": 0, "transform": 1, "sparse": 2}
FE_KIND = {"tridiag": 0, "midpoint": 1}
KERNEL = {"auto": 0, "generic": 1, "register": 2, "pipelined": 3}
NUM_STAGES = 14
STAGES = ["row0", "fwd_scatter", "fwd_spectral", "fwd_unpermute", "fwd_fused", "bwd_gather",
          "bwd_spectral", "bwd_scatter", "bwd_fused", "batch", "row_mean", "dense_scatter",
          "sparse_pack", "fwd_sparse"]


class QmcDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("N", C.c_int64), ("modulus_P", C.c_uint64), ("g", C.c_int64),
                ("s", C.c_int32), ("gen_host", C.POINTER(C.c_int64)),
                ("gen_is_exponent", C.c_int32), ("map", C.c_int32), ("row0", C.c_int32),
                ("order", C.c_int32), ("prec", C.c_int32), ("shift", C.c_double), ("base", C.c_int32)]


class QmcInfo(C.Structure):
    _fields_ = [("N", C.c_int64), ("L", C.c_int64), ("g", C.c_int64), ("modulus_P", C.c_uint64),
                ("s", C.c_int32), ("n_distinct", C.c_int32), ("collision_adds", C.c_int32),
                ("row0_adds", C.c_int32), ("out_rows", C.c_int64), ("phi0", C.c_double),
                ("L1", C.c_int32), ("L2", C.c_int32), ("has_row0", C.c_int32), ("base", C.c_int32)]


class QmcError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)} ({status_string(code)})")


_LIB = None


def lib_path() -> str:
    return _build.lib_path()


def load(path: str | None = None):
    """Loads libqmcfft.so (raises if it has not been built).  The
    environment variable QMC_LIBRARY names another build of the same ABI to
    load instead (the bounds-checked libqmcfft_checked.so)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or os.environ.get("QMC_LIBRARY") or lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libqmcfft.so not built ({path}); run __graft_entry__.build()")
    lib = C.CDLL(path)
    vp, i32, i64, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
    pvp = C.POINTER(C.c_void_p)
    sig = {
        "qmc_plan_create": (C.c_int, [pvp, C.POINTER(QmcDesc), vp]),
        "qmc_plan_destroy": (C.c_int, [vp]),
        "qmc_plan_info": (C.c_int, [vp, C.POINTER(QmcInfo)]),
        "qmc_plan_exponents": (C.c_int, [vp, C.POINTER(C.c_int32)]),
        "qmc_plan_copy_table": (C.c_int, [vp, i32, vp, i64]),
        "qmc_plan_reserve": (C.c_int, [vp, i32]),
        "qmc_plan_sync_status": (C.c_int, [vp, vp]),
        "qmc_matmul": (C.c_int, [vp, vp, i64, i32, i32, vp, i64, vp, vp, vp]),
        "qmc_matmul_backward": (C.c_int, [vp, vp, i64, i32, i32, vp, i64, vp]),
        "qmc_generate_points": (C.c_int, [vp, vp, i64, vp]),
        "qmc_batch_create": (C.c_int, [pvp, pvp, C.POINTER(C.c_int32), i32, vp]),
        "qmc_batch_matmul": (C.c_int, [vp, pvp, C.POINTER(C.c_int64), pvp, C.POINTER(C.c_int64), vp]),
        "qmc_batch_destroy": (C.c_int, [vp]),
        "qmc_status_string": (C.c_char_p, [C.c_int]),
        "qmc_version": (C.c_int, []),
        "qmc_plan_set_profiling": (C.c_int, [vp, i32]),
        "qmc_plan_read_profile": (C.c_int, [vp, C.POINTER(C.c_double), C.POINTER(C.c_int32)]),
        "qmc_kernel_launches": (C.c_int64, []),
        "qmc_plan_set_option": (C.c_int, [vp, i32, i64]),
        "qmc_matmul_noalloc": (C.c_int, [vp, vp, i64, i32, i32, vp, i64, vp]),
        "qmc_matmul_affine": (C.c_int, [vp, vp, i64, i32, i32, vp, i32, vp, i64, vp]),
        "qmc_batch_set_option": (C.c_int, [vp, i32, i64]),
        "qmc_batch_sync_status": (C.c_int, [vp, vp]),
        "qmc_fe_work_bytes": (C.c_int64, [i64, i32]),
        "qmc_fe_solve_mean": (C.c_int, [vp, i64, i64, i32, i32, vp, vp, i64, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if hasattr(lib, "qmc_debug_poke_table"):  # bounds-checked builds only (qmc_debug.h)
        lib.qmc_debug_poke_table.restype = C.c_int
        lib.qmc_debug_poke_table.argtypes = [vp, i32, i64, i32, C.POINTER(C.c_int32)]
    _LIB = lib
    return lib


def status_string(code: int) -> str:
    try:
        return load().qmc_status_string(code).decode()
    except Exception:
        return STATUS.get(code, str(code))


def check(code: int, where: str) -> None:
    if code != QMC_OK:
        raise QmcError(code, where)
