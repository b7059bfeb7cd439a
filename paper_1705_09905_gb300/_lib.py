"""ctypes loader and signatures for libfcoo.so (the C ABI in include/fcoo.h).

The library is the only compute path: if it is missing, importing this module
raises, there is no CPU fallback.  Build it with ``python
paper_1705_09905_gb300/build.py`` or ``__graft_entry__.build()``.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libfcoo.so")

FCOO_OK = 0
STATUS = {
    0: "FCOO_OK", -1: "FCOO_ERR_INVALID_ARG", -2: "FCOO_ERR_INDEX_RANGE", -3: "FCOO_ERR_DUPLICATE",
    -4: "FCOO_ERR_NOMEM", -5: "FCOO_ERR_CUDA", -6: "FCOO_ERR_NOT_PD", -7: "FCOO_ERR_NONFINITE",
    -8: "FCOO_ERR_TIMEOUT", -9: "FCOO_ERR_UNSUPPORTED",
}
FCOO_ERR_INVALID_ARG = -1
FCOO_ERR_UNSUPPORTED = -9
MAX_MODES = 8
MAX_RANK = 256
NOALLOC_MAX_RANK = 128  # FCOO_NOALLOC_MAX_RANK


class FcooError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.message = message


class FcooInfo(ctypes.Structure):
    _fields_ = [
        ("nmodes", ctypes.c_int), ("mode", ctypes.c_int), ("op", ctypes.c_int), ("threadlen", ctypes.c_int),
        ("nnz", ctypes.c_int64), ("nseg", ctypes.c_int64), ("nfib", ctypes.c_int64),
        ("dims", ctypes.c_uint32 * MAX_MODES),
        ("nprod", ctypes.c_int), ("prod_modes", ctypes.c_int * MAX_MODES),
        ("nidx", ctypes.c_int), ("idx_modes", ctypes.c_int * MAX_MODES),
        ("bytes_val", ctypes.c_int64), ("bytes_pidx", ctypes.c_int64), ("bytes_bf", ctypes.c_int64),
        ("bytes_sf", ctypes.c_int64), ("bytes_table2", ctypes.c_int64), ("bytes_segmap", ctypes.c_int64),
        ("bytes_aux", ctypes.c_int64), ("bytes_scratch", ctypes.c_int64), ("bytes_pidx16", ctypes.c_int64),
    ]


class FcooView(ctypes.Structure):
    """fcoo_view_t: an SpMTTKRP F-COO layout in caller-owned device buffers."""

    _fields_ = [
        ("nmodes", ctypes.c_int), ("mode", ctypes.c_int), ("threadlen", ctypes.c_int),
        ("nnz", ctypes.c_int64), ("nseg", ctypes.c_int64),
        ("dims", ctypes.c_uint32 * MAX_MODES),
        ("pidx", ctypes.c_void_p * (MAX_MODES - 1)),
        ("val", ctypes.c_void_p), ("bf", ctypes.c_void_p), ("sf", ctypes.c_void_p),
        ("segrow", ctypes.c_void_p), ("hcount", ctypes.c_void_p),
    ]


_vp = ctypes.c_void_p
_i = ctypes.c_int
_i64 = ctypes.c_int64
_vpp = ctypes.POINTER(ctypes.c_void_p)

# name: (restype, argtypes)
SIGNATURES = {
    "fcoo_last_error": (ctypes.c_char_p, []),
    "fcoo_status_string": (ctypes.c_char_p, [_i]),
    "fcoo_version": (_i, []),
    "fcoo_table2_bytes": (_i64, [_i, _i64, _i]),
    "fcoo_table2_bytes_ex": (_i64, [_i, _i64, _i, _i]),
    "fcoo_compress_indices": (_i, [_vp, _vp]),
    "fcoo_build": (_i, [_i, _vp, _i64, _vpp, _vp, _i, _i, _i, _vp, ctypes.POINTER(_vp)]),
    "fcoo_destroy": (_i, [_vp]),
    "fcoo_info": (_i, [_vp, ctypes.POINTER(FcooInfo)]),
    "fcoo_copy_layout": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "fcoo_fibre_indices": (_i, [_vp, _vp, _vp]),
    "spmttkrp": (_i, [_vp, _vpp, _i, _i, _vp, _vp]),
    "spttm": (_i, [_vp, _vp, _i, _i, _vp, _vp]),
    "spttmc": (_i, [_vp, _vpp, _i, _i, _vp, _vp]),
    "spttmc_plan_create": (_i, [_vp, _i, _i, _i, ctypes.POINTER(_vp), _vp]),
    "spttmc_plan_run": (_i, [_vp, _vpp, _i, _vp, _vp]),
    "spttmc_plan_info": (_i, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "spttmc_plan_destroy": (_i, [_vp]),
    "spmttkrp_noalloc": (_i, [ctypes.POINTER(FcooView), _vpp, _i, _i, _vp, _vp]),
    "spmttkrp_gather_bound": (_i, [_vp, _vpp, _i, _i, _vp, _vp]),
    "cp_state_create": (_i, [_i, _vp, _i, _i, _vpp, _vp, ctypes.POINTER(_vp)]),
    "tucker_state_create": (_i, [_i, _vp, _i, _vpp, _vp, ctypes.POINTER(_vp)]),
    "tucker_state_destroy": (_i, [_vp]),
    "tucker_hooi_iter": (_i, [_vpp, _vp, _vp]),
    "tucker_state_stats": (_i, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "tucker_state_copy_factor": (_i, [_vp, _i, _vp, _vp]),
    "cp_state_destroy": (_i, [_vp]),
    "cp_als_iter": (_i, [_vpp, _vp, _vp]),
    "cp_state_stats": (_i, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "cp_state_copy_factor": (_i, [_vp, _i, _vp, _vp]),
    "cp_state_set_dtype": (_i, [_vp, _i, _vp]),
    "cp_state_use_fibres": (_i, [_vp, _vp, _i, _vp]),
    "cp_state_blob_size": (_i64, [_vp]),
    "cp_state_save": (_i, [_vp, _vp, _i64, _vp]),
    "cp_state_load": (_i, [_vp, _vp, _i64, _vp]),
    "spmttkrp_backward": (_i, [_vpp, _vpp, _i, _i, _vp, _i, _i, _vpp, _vp, _vp, _vp]),
    "sparse_cp_loss": (_i, [_vp, _vpp, _i, _i, _vp, _vp]),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libfcoo.so not found at {LIB_PATH}; build it with "
                          "`python -m paper_1705_09905_gb300.build` (needs nvcc); there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name, None)
        if fn is None:
            continue
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def exported(name: str) -> bool:
    return hasattr(lib, name)


def check(status: int) -> int:
    if status != FCOO_OK:
        msg = lib.fcoo_last_error()
        raise FcooError(int(status), msg.decode() if msg else "")
    return status


def ptr_array(ptrs):
    arr = (ctypes.c_void_p * len(ptrs))(*[(int(p) if p else None) for p in ptrs])
    return ctypes.cast(arr, _vpp), arr
