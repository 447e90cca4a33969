"""ctypes binding of liblbm.so: same entry-point names as include/lbm.h, argument marshalling only.

The shared object is built in-tree by ``paper_1110_5004_gb300.build``.  If it is missing the
import fails loudly: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbm.so")

LBM_PERIODIC, LBM_WALL = 0, 1
LBM_FP32, LBM_FP16_DEV, LBM_BF16_DEV = 0, 1, 2
LBM_KERNEL_AUTO, LBM_KERNEL_ROWS, LBM_KERNEL_TILES, LBM_KERNEL_RESIDENT = 0, 1, 2, 3
LBM_OK = 0
LBM_ERR_INVALID_ARG, LBM_ERR_OOM, LBM_ERR_BUDGET, LBM_ERR_DIVERGED, LBM_ERR_TIMEOUT, LBM_ERR_CUDA = \
    -1, -2, -3, -4, -5, -6

# Every function the C ABI (include/lbm.h) declares.
EXPORTS = (
    "lbm_params_from_sigma_W", "lbm_tau_from_nu", "lbm_device_bytes", "lbm_create", "lbm_init_fields",
    "lbm_step", "lbm_moments", "lbm_interfacial_force", "lbm_diagnostics", "lbm_destroy", "lbm_step_count", "lbm_set_stream",
    "lbm_set_tile", "lbm_launch_count", "lbm_strerror", "lbm_last_error", "lbm_batch_create",
    "lbm_batch_add", "lbm_batch_remove", "lbm_batch_step", "lbm_batch_size", "lbm_batch_bytes",
    "lbm_batch_destroy", "lbm_diagnostics_fields_noalloc", "lbm_batch_set_tile", "lbm_checkpoint_bytes",
    "lbm_checkpoint", "lbm_restore", "lbm_sim_device_bytes", "lbm_init_fields_packed", "lbm_moments_packed",
    "lbm_set_kernel", "lbm_set_wait_limit", "lbm_step_status", "lbm_active_kernel",
)


class lbm_params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "beta", "kappa", "phi_star", "theta_M", "tau_f", "tau_g_A", "tau_g_B", "rho_A", "rho_B",
        "gravity")] + [(n, ctypes.c_int) for n in ("bc_x", "bc_y", "remove_Fa", "storage", "ch_conservative", "fs_form", "s_form", "f_form")]


class lbm_diag(ctypes.Structure):
    _fields_ = [("step", ctypes.c_longlong)] + [(n, ctypes.c_double) for n in (
        "sum_phi", "liquid_area", "centroid_x", "centroid_y", "vel_x", "vel_y", "spread_radius",
        "max_u", "p_liquid", "p_gas")] + [("finite", ctypes.c_int), ("pad", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class LBMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (_strerror(code), code, msg))
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load liblbm.so and declare the signatures.  Raises if the library was not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("liblbm.so not built at %s: run paper_1110_5004_gb300.build.build()" % path)
    L = ctypes.CDLL(path)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
    fp = ctypes.c_void_p   # float* (host or device address)
    sig = {
        "lbm_params_from_sigma_W": (ip, [ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp]),
        "lbm_tau_from_nu": (ctypes.c_double, [ctypes.c_double]),
        "lbm_device_bytes": (ctypes.c_size_t, [ip, ip, ip]),
        "lbm_create": (ip, [ip, ip, ctypes.POINTER(lbm_params), vp, ctypes.POINTER(vp)]),
        "lbm_init_fields": (ip, [vp, fp, fp, fp, fp]),
        "lbm_step": (ip, [vp, ip]),
        "lbm_moments": (ip, [vp, fp, fp, fp, fp, fp]),
        "lbm_init_fields_packed": (ip, [vp, fp]),
        "lbm_moments_packed": (ip, [vp, fp]),
        "lbm_interfacial_force": (ip, [vp, fp, fp]),
        "lbm_diagnostics": (ip, [vp, ctypes.POINTER(lbm_diag)]),
        "lbm_destroy": (ip, [vp]),
        "lbm_step_count": (ctypes.c_longlong, [vp]),
        "lbm_checkpoint_bytes": (ctypes.c_size_t, [vp]),
        "lbm_sim_device_bytes": (ctypes.c_size_t, [vp]),
        "lbm_checkpoint": (ip, [vp, vp, ctypes.c_size_t]),
        "lbm_restore": (ip, [vp, vp, ctypes.c_size_t]),
        "lbm_set_stream": (ip, [vp, vp]),
        "lbm_set_tile": (ip, [vp, ip, ip]),
        "lbm_set_kernel": (ip, [vp, ip]),
        "lbm_set_wait_limit": (ip, [vp, ctypes.c_longlong, ip]),
        "lbm_step_status": (ip, [vp]),
        "lbm_active_kernel": (ip, [vp]),
        "lbm_launch_count": (ctypes.c_longlong, [vp]),
        "lbm_strerror": (ctypes.c_char_p, [ip]),
        "lbm_last_error": (ctypes.c_char_p, []),
        "lbm_batch_create": (ip, [ctypes.c_size_t, vp, ctypes.POINTER(vp)]),
        "lbm_batch_add": (ip, [vp, vp, ctypes.POINTER(ip)]),
        "lbm_batch_remove": (ip, [vp, ip]),
        "lbm_batch_step": (ip, [vp, ip]),
        "lbm_batch_set_tile": (ip, [vp, ip, ip]),
        "lbm_batch_size": (ip, [vp]),
        "lbm_batch_bytes": (ctypes.c_size_t, [vp]),
        "lbm_batch_destroy": (ip, [vp]),
        "lbm_diagnostics_fields_noalloc": (ip, [fp, fp, fp, fp, ip, ip, ctypes.c_double, ctypes.c_longlong, vp,
                                                ctypes.POINTER(lbm_diag)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _strerror(code):
    try:
        return load().lbm_strerror(code).decode()
    except Exception:   # pragma: no cover - message only
        return "error"


def check(rc):
    if rc != LBM_OK:
        raise LBMError(rc, load().lbm_last_error().decode())
    return rc


def check_value(rc):
    """For calls that return a non-negative value or a negative LBM_ERR_* code."""
    if rc < 0:
        raise LBMError(rc, load().lbm_last_error().decode())
    return rc
