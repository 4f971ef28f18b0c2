"""ctypes declarations of the libgcdf C ABI (include/gcdf.h).

Loading fails loudly when the shared library is missing: there is no other
implementation of these calls in this package.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgcdf.so")

GCDF_OK, GCDF_EINVAL, GCDF_ENOMEM, GCDF_ECUDA, GCDF_EUNSUPPORTED = 0, 1, 2, 3, 4
GCDF_FP32, GCDF_BF16, GCDF_FP16 = 0, 1, 2
GCDF_RED_MIN, GCDF_RED_SOFTMIN, GCDF_RED_HINGE = 0, 1, 2

# Every function the header declares, with (restype, argtypes).
_vp = ctypes.c_void_p
_i = ctypes.c_int
_f = ctypes.c_float


class NetDesc(ctypes.Structure):
    _fields_ = [("n_dof", _i), ("hidden", _i), ("n_hidden_layers", _i), ("precision", _i)]


SIGNATURES = {
    "gcdf_weight_count": (ctypes.c_size_t, [ctypes.POINTER(NetDesc)]),
    "gcdf_create_net": (_i, [ctypes.POINTER(NetDesc), _vp, ctypes.c_size_t, ctypes.POINTER(_vp)]),
    "gcdf_destroy_net": (_i, [_vp]),
    "gcdf_query": (_i, [_vp, _vp, _i, _vp, _i, _vp, _vp, _i, _vp, _vp, _vp, _vp]),
    "gcdf_collision_cost": (_i, [_vp, _vp, _i, _vp, _i, _vp, _vp, _i, _vp, _i, _f, _vp, _vp, _vp, _vp]),
    "gcdf_collision_cost_noalloc": (_i, [_vp, _vp, _i, _vp, _i, _vp, _vp, _i, _vp, _i, _f, _vp, _vp, _vp, _vp]),
    "gcdf_device_status": (_i, [_vp, ctypes.POINTER(_i)]),
    "gcdf_set_profile_events": (_i, [_vp, _vp, _vp]),
    "gcdf_last_error": (ctypes.c_char_p, []),
}

_lib = None


def load() -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"libgcdf.so is not built ({LIB_PATH} missing); run "
            "`python -m paper_2601_18548_gb300.build` or __graft_entry__.build() first")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class GcdfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libgcdf error {code}: {msg}")
        self.code = code


def check(rc: int):
    if rc != GCDF_OK:
        msg = load().gcdf_last_error()
        raise GcdfError(rc, msg.decode() if msg else "")
