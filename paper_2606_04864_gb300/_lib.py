"""ctypes view of the C ABI declared in include/ams.h.

Loads ``libams.so`` from this package directory.  There is no fallback: if
the library is missing or fails to load, :func:`lib` raises, so nothing can
run on a silent CPU path.
"""

from __future__ import annotations

import ctypes as C
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
# AMS_LIBRARY=debug selects the checking build (device-side index checks;
# see _build.py), anything else the release build
LIB_PATH = os.path.join(_PKG, "libams_debug.so" if os.environ.get("AMS_LIBRARY") == "debug" else "libams.so")

AMS_OK = 0
STATUS_NAMES = {
    0: "AMS_OK", 1: "AMS_ERR_INVALID_ARG", 2: "AMS_ERR_NOT_SPD", 3: "AMS_ERR_BREAKDOWN",
    4: "AMS_ERR_NOT_CONVERGED", 5: "AMS_ERR_DEVICE_TIMEOUT", 6: "AMS_ERR_CUDA", 7: "AMS_ERR_OOM",
}
PREC = {"fp64": 0, "fp32": 1, "fp32_bf16": 2}
# AMS_KERNEL_* indices of ams_time_kernel / ams_profile_solve, in launch order
KERNEL_NAMES = ["spmv_direction", "local_solve_restrict", "coarse_solve", "prolong_update"]
AMS_NUM_KERNELS = len(KERNEL_NAMES)
CG = {"auto": -1, "pcg": 0, "fcg": 1}


class ams_options(C.Structure):
    _fields_ = [
        ("precision", C.c_int32),
        ("cg_variant", C.c_int32),
        ("maxit", C.c_int32),
        ("device_ptrs", C.c_int32),
        ("autotune", C.c_int32),
        ("coarse", C.c_int32),
        ("eig_shift", C.c_double),
        ("eig_maxit", C.c_int32),
        ("eig_tol", C.c_double),
        ("spin_budget_cycles", C.c_int64),
        ("eig_threshold", C.c_double),
        ("two_grid_omega", C.c_double),
        ("timeout_probe", C.c_int32),
        ("warm_start", C.c_int32),
    ]


class ams_system_desc(C.Structure):
    _fields_ = [
        ("n", C.c_int64),
        ("rowptr", C.c_void_p),
        ("colind", C.c_void_p),
        ("vals", C.c_void_p),
        ("part", C.c_void_p),
        ("nparts", C.c_int32),
        ("m", C.c_int32),
    ]


class ams_info(C.Structure):
    _fields_ = [
        ("n", C.c_int64),
        ("nnz", C.c_int64),
        ("nparts", C.c_int32),
        ("nsys", C.c_int32),
        ("ncoarse", C.c_int64),
        ("max_band_tiles", C.c_int32),
        ("precision", C.c_int32),
        ("cg_variant", C.c_int32),
        ("setup_seconds", C.c_double),
        ("eig_seconds", C.c_double),
        ("coarse_seconds", C.c_double),
        ("eig_iterations", C.c_int32),
        ("eig_max_residual", C.c_double),
        ("local_factor_bytes", C.c_int64),
        ("coarse_inverse_bytes", C.c_int64),
        ("basis_bytes", C.c_int64),
        ("spmv_variant", C.c_int32),
        ("kernel_launches", C.c_int64),
        ("two_grid_omega", C.c_double),
        ("local_lambda_max", C.c_double),
        ("coarse_factor_seconds", C.c_double),
        ("coarse_factor_gflop", C.c_double),
    ]


# exported symbol -> (restype, argtypes)
SIGNATURES = {
    "ams_options_default": (None, [C.POINTER(ams_options)]),
    "ams_setup": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                            C.c_int32, C.POINTER(ams_options), C.c_void_p, C.POINTER(C.c_void_p)]),
    "ams_setup_batched": (C.c_int, [C.c_int32, C.POINTER(ams_system_desc), C.POINTER(ams_options),
                                    C.c_void_p, C.POINTER(C.c_void_p)]),
    "ams_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_double, C.c_void_p, C.c_void_p,
                            C.c_void_p]),
    "ams_solve_adjoint": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_double, C.c_void_p,
                                    C.c_void_p, C.c_void_p, C.c_void_p]),
    "ams_destroy": (C.c_int, [C.c_void_p]),
    "ams_set_matrix_values": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ams_status_string": (C.c_char_p, [C.c_int]),
    "ams_last_error": (C.c_char_p, []),
    "ams_get_info": (C.c_int, [C.c_void_p, C.POINTER(ams_info)]),
    "ams_get_index_maps": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "ams_get_launch_shape": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
    "ams_partition": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_int32, C.c_double, C.c_uint64,
                                C.c_void_p, C.c_void_p]),
    "ams_set_launch_shape": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
    "ams_get_coarse_basis": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ams_get_coarse_matrix": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ams_get_coarse_factor_inverse": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "ams_debug_selftest": (C.c_int, [C.c_void_p]),
    "ams_apply_preconditioner": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "ams_spmv": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "ams_time_kernel": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_double),
                                  C.POINTER(C.c_double)]),
    "ams_profile_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_double, C.c_void_p,
                                    C.c_void_p, C.c_void_p]),
    "ams_csr_spmv_dot_noalloc": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                           C.c_void_p, C.c_void_p, C.c_void_p]),
    "ams_check_conversions": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
}

_lock = threading.Lock()
_lib = None


def lib() -> C.CDLL:
    """The loaded library (raises if it is missing: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{os.path.basename(LIB_PATH)} not found at {LIB_PATH}; build it with "
                    "`python -m paper_2606_04864_gb300._build` (add --debug for the checking build)")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
        return _lib


class AmsError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().ams_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")


def check(status: int, where: str, allow=()):
    if status != AMS_OK and status not in allow:
        raise AmsError(status, where)
    return status
