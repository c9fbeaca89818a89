"""ctypes declarations of the C interface in include/gsm.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgsm.so")

KERNELS = {"coulomb3d": 0, "coulomb2d": 1, "poisson2d": 2, "dipolar3d": 3, "ds2d": 4, "power3d": 5, "power2d": 6}
KERNEL_DIM = {"coulomb3d": 3, "coulomb2d": 2, "poisson2d": 2, "dipolar3d": 3, "ds2d": 2, "power3d": 3,
              "power2d": 2}
PRECISIONS = {"fp64": 0, "fp32": 1, "fp32x2": 2}
STATUS = {0: "GSM_OK", 1: "GSM_ERR_INVALID_ARG", 2: "GSM_ERR_UNSUPPORTED_SIZE", 3: "GSM_ERR_OOM",
          4: "GSM_ERR_CUDA", 5: "GSM_ERR_ACCURACY", 6: "GSM_ERR_TIMEOUT", 7: "GSM_ERR_BAD_PLAN"}

# Every function declared in include/gsm.h
EXPORTS = ["gsm_default_options", "gsm_plan", "gsm_apply", "gsm_apply_pass", "gsm_plan_autotune", "gsm_apply_host", "gsm_apply_batched",
           "gsm_hartree", "gsm_plan_info", "gsm_plan_destroy", "gsm_status_string", "gsm_last_error",
           "gsm_plan_gs_terms", "gsm_plan_kernel_tensor", "gsm_plan_factors", "gsm_fft_lines",
           "gsm_fft_lines_noalloc", "gsm_batch_create", "gsm_batch_launch", "gsm_batch_destroy",
           "gsm_plan_save", "gsm_plan_load", "gsm_debug_fail_alloc", "gsm_debug_alloc_stats",
           "gsm_batch_wait", "gsm_debug_batch_wait", "gsm_plan_set_schedule", "gsm_dft32_tc"]


class Options(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_double), ("S", ctypes.c_int), ("precision", ctypes.c_int),
                ("dip_n", ctypes.c_double * 3), ("dip_m", ctypes.c_double * 3), ("debug", ctypes.c_int),
                ("box", ctypes.c_double * 3), ("beta", ctypes.c_double), ("host_zero_copy", ctypes.c_int)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("d", ctypes.c_int), ("n", ctypes.c_int * 3), ("M", ctypes.c_int * 3),
                ("L", ctypes.c_double), ("delta", ctypes.c_double), ("S", ctypes.c_int), ("nterms", ctypes.c_int),
                ("gs_err", ctypes.c_double), ("c0", ctypes.c_double), ("c2", ctypes.c_double),
                ("precision", ctypes.c_int), ("bytes_multiplier", ctypes.c_size_t),
                ("bytes_workspace", ctypes.c_size_t), ("npasses", ctypes.c_int),
                ("launch_nl", ctypes.c_int * 5), ("launch_threads", ctypes.c_int * 5),
                ("launch_emax", ctypes.c_int * 5), ("box", ctypes.c_double * 3), ("beta", ctypes.c_double),
                ("radix_fwd", (ctypes.c_int * 12) * 3), ("radix_inv", (ctypes.c_int * 12) * 3)]


class GSMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None

_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def load(path: str = LIB_PATH):
    """Load libgsm.so; raises if it has not been built (no fallback exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"GSM CUDA library not found at {path}; build it with "
                               "`python -m paper_1501_04438_gb300.build` (there is no CPU fallback)")
        L = ctypes.CDLL(path)
        L.gsm_default_options.argtypes = [ctypes.POINTER(Options)]
        L.gsm_default_options.restype = None
        L.gsm_plan.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, ctypes.c_double, _ip,
                               ctypes.c_double, ctypes.POINTER(Options), _vp]
        L.gsm_apply.argtypes = [_vp, _vp, _vp, _vp]
        L.gsm_apply_host.argtypes = [_vp, _vp, _vp, _vp]
        L.gsm_apply_pass.argtypes = [_vp, ctypes.c_int, _vp, _vp, _vp]
        L.gsm_plan_autotune.argtypes = [_vp, _vp, ctypes.c_char_p, ctypes.c_size_t]
        L.gsm_plan_set_schedule.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _ip, ctypes.c_int, _vp]
        L.gsm_apply_batched.argtypes = [ctypes.c_int, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                        ctypes.POINTER(_vp), _vp]
        L.gsm_batch_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                       ctypes.POINTER(_vp), _vp]
        L.gsm_batch_launch.argtypes = [_vp, _vp]
        L.gsm_batch_destroy.argtypes = [_vp]
        L.gsm_batch_wait.argtypes = [_vp, _vp]
        L.gsm_debug_batch_wait.argtypes = [ctypes.c_longlong, ctypes.c_int]
        L.gsm_hartree.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
        L.gsm_plan_info.argtypes = [_vp, ctypes.POINTER(PlanInfo)]
        L.gsm_plan_destroy.argtypes = [_vp]
        L.gsm_plan_save.argtypes = [_vp, _vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
        L.gsm_plan_load.argtypes = [ctypes.POINTER(_vp), _vp, ctypes.c_size_t, ctypes.c_int, _vp]
        L.gsm_status_string.argtypes = [ctypes.c_int]
        L.gsm_status_string.restype = ctypes.c_char_p
        L.gsm_last_error.argtypes = []
        L.gsm_last_error.restype = ctypes.c_char_p
        L.gsm_plan_gs_terms.argtypes = [_vp, _dp, _dp, ctypes.c_int, _ip]
        L.gsm_plan_kernel_tensor.argtypes = [_vp, _dp, ctypes.c_size_t]
        L.gsm_plan_factors.argtypes = [_vp, ctypes.c_int, _dp, ctypes.c_size_t]
        L.gsm_fft_lines.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp]
        L.gsm_fft_lines_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp]
        L.gsm_dft32_tc.argtypes = [ctypes.c_int, ctypes.c_int, _vp, _vp, _vp]
        L.gsm_debug_fail_alloc.argtypes = [ctypes.c_int]
        L.gsm_debug_alloc_stats.argtypes = [ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]
        for name in EXPORTS:
            if name not in ("gsm_default_options", "gsm_status_string", "gsm_last_error"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
        return _lib


def check(status: int):
    if status != 0:
        msg = load().gsm_last_error().decode(errors="replace")
        raise GSMError(status, msg)
