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
GCDF_EAGAIN, GCDF_PENDING, GCDF_ETIMEOUT = 5, 6, 7
GCDF_FP32, GCDF_BF16, GCDF_FP16, GCDF_FP8 = 0, 1, 2, 3
GCDF_RED_MIN, GCDF_RED_SOFTMIN, GCDF_RED_HINGE = 0, 1, 2

# Every function the header declares, with (restype, argtypes).
_vp = ctypes.c_void_p
_i = ctypes.c_int
_f = ctypes.c_float


class NetDesc(ctypes.Structure):
    _fields_ = [("n_dof", _i), ("hidden", _i), ("n_hidden_layers", _i), ("precision", _i)]


class FitDesc(ctypes.Structure):
    _fields_ = [("n_dof", _i), ("hidden", _i), ("n_hidden_layers", _i), ("precision", _i)]


class PlanParams(ctypes.Structure):
    _fields_ = [("dt", _f), ("w_trans", _f), ("w_rot", _f), ("w_goal", _f), ("mu", _f), ("delta", _f),
                ("lambda0", _f), ("lambda_min", _f), ("lambda_max", _f), ("iterations", _i),
                ("partition_radius", _f)]


class PlanProblem(ctypes.Structure):
    _fields_ = [("n_waypoints", _i), ("q_start", _vp), ("q_goal", _vp), ("q_init", _vp),
                ("points", _vp), ("n_points", _i)]


class ServerDesc(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_active", _i), ("max_queued", _i),
                ("params", PlanParams)]


class PlanRequest(ctypes.Structure):
    _fields_ = [("net", _vp), ("n_waypoints", _i), ("q_start", _vp), ("q_goal", _vp),
                ("points", _vp), ("n_points", _i)]


class PlanResult(ctypes.Structure):
    _fields_ = [("q", _vp), ("merit", ctypes.c_double), ("accepted_steps", _i),
                ("submit_s", ctypes.c_double), ("admit_s", ctypes.c_double), ("done_s", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_uint64), ("step_device_s", ctypes.c_double), ("step_host_s", ctypes.c_double),
                ("pass_s", ctypes.c_double), ("active_sum", ctypes.c_uint64)]


SIGNATURES = {
    "gcdf_weight_count": (ctypes.c_size_t, [ctypes.POINTER(NetDesc)]),
    "gcdf_create_net": (_i, [ctypes.POINTER(NetDesc), _vp, ctypes.c_size_t, ctypes.POINTER(_vp)]),
    "gcdf_destroy_net": (_i, [_vp]),
    "gcdf_query": (_i, [_vp, _vp, _i, _vp, _i, _vp, _vp, _i, _vp, _vp, _vp, _vp]),
    "gcdf_collision_cost": (_i, [_vp, _vp, _i, _vp, _i, _vp, _vp, _i, _vp, _i, _f, _vp, _vp, _vp, _vp]),
    "gcdf_collision_cost_noalloc": (_i, [_vp, _vp, _i, _vp, _i, _vp, _vp, _i, _vp, _i, _f, _vp, _vp, _vp, _vp]),
    "gcdf_device_status": (_i, [_vp, ctypes.POINTER(_i)]),
    "gcdf_set_profile_events": (_i, [_vp, _vp, _vp]),
    "gcdf_set_active_set": (_i, [_vp, _i]),
    "gcdf_selftest_wait_expiry": (_i, [_vp, ctypes.c_longlong, ctypes.POINTER(_i)]),
    "gcdf_diag_fp32_fma": (ctypes.c_longlong, [_i, _i, _i, _vp, _vp]),
    "gcdf_project": (_i, [_vp, _vp, _i, _vp, _i, _vp, _vp, _i, _vp, _vp, _vp, _vp]),
    "gcdf_partition_offsets": (_i, [_vp, _i, _vp, _i, _f, _vp, _vp]),
    "gcdf_partition_indices": (_i, [_vp, _i, _vp, _i, _f, _vp, _vp, _vp]),
    "gcdf_jacobian_scatter": (_i, [_vp, _i, _i, _vp, _i, _i, _vp, _vp, _vp, _vp]),
    "gcdf_fit_device_status": (_i, [ctypes.POINTER(_i)]),
    "gcdf_fit_forward": (_i, [ctypes.POINTER(FitDesc), _vp, _vp, _vp, _i, _vp, _vp]),
    "gcdf_fit_vjp": (_i, [ctypes.POINTER(FitDesc), _vp, _vp, _vp, _i, _vp, _vp, _vp, _vp]),
    "gcdf_fit_value_grad": (_i, [ctypes.POINTER(FitDesc), _vp, _vp, _vp, _i, _vp, _vp, _vp]),
    "gcdf_fit_vjp2": (_i, [ctypes.POINTER(FitDesc), _vp, _vp, _vp, _i, _vp, _vp, _vp, _vp]),
    "gcdf_fit_tape_bytes": (_i, [ctypes.POINTER(FitDesc), _i, ctypes.POINTER(ctypes.c_size_t)]),
    "gcdf_fit_forward_tape": (_i, [ctypes.POINTER(FitDesc), _vp, _vp, _vp, _i, _vp, _vp, ctypes.c_size_t, _vp]),
    "gcdf_fit_vjp_tape": (_i, [ctypes.POINTER(FitDesc), _vp, _vp, _vp, _i, _vp, _vp, ctypes.c_size_t, _vp, _vp,
                               _vp]),
    "gcdf_plan_solve": (_i, [_vp, ctypes.POINTER(PlanProblem), _i, ctypes.POINTER(PlanParams), _vp, _vp, _vp, _vp]),
    "gcdf_server_create": (_i, [ctypes.POINTER(ServerDesc), ctypes.POINTER(_vp)]),
    "gcdf_plan_submit": (_i, [_vp, ctypes.POINTER(PlanRequest), ctypes.POINTER(ctypes.c_uint64)]),
    "gcdf_plan_poll": (_i, [_vp, ctypes.c_uint64, ctypes.POINTER(PlanResult)]),
    "gcdf_server_clock": (ctypes.c_double, [_vp]),
    "gcdf_server_stats_get": (_i, [_vp, ctypes.POINTER(ServerStats)]),
    "gcdf_plan_request_bytes": (ctypes.c_size_t, [_vp, _i, _i]),
    "gcdf_server_destroy": (_i, [_vp]),
    "gcdf_release_cached_memory": (_i, []),
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
