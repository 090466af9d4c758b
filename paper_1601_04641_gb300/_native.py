"""ctypes declarations of the C ABI in include/gp.h (libgpcn.so).

Argument marshalling only.  Loading fails loudly when the library has not
been built: there is no CPU fallback for any of these calls.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgpcn.so")

GP_OK, GP_ERR_ARG, GP_ERR_CUDA, GP_ERR_NOMEM, GP_ERR_NONFINITE, GP_ERR_TIMEOUT, GP_ERR_STATE, GP_ERR_IO = range(8)
STATUS_NAMES = {0: "GP_OK", 1: "GP_ERR_ARG", 2: "GP_ERR_CUDA", 3: "GP_ERR_NOMEM",
                4: "GP_ERR_NONFINITE", 5: "GP_ERR_TIMEOUT", 6: "GP_ERR_STATE", 7: "GP_ERR_IO"}
GP_OUT_PSI, GP_OUT_DENSITY = 0, 1
GP_F64, GP_F32, GP_F16 = 0, 1, 2
GP_COMPLEX, GP_REAL = 0, 1


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double)]


class Obs(ctypes.Structure):
    _fields_ = [("norm", ctypes.c_double), ("mu", ctypes.c_double), ("energy", ctypes.c_double),
                ("rms_x", ctypes.c_double), ("rms_y", ctypes.c_double), ("rms_z", ctypes.c_double),
                ("step", ctypes.c_longlong), ("t", ctypes.c_double)]


Handle = ctypes.c_void_p
_vp = ctypes.c_void_p
_d = ctypes.c_double
_i = ctypes.c_int

# name -> (restype, argtypes), in the order of include/gp.h
SIGNATURES = {
    "gp_create": (_i, [ctypes.POINTER(Handle), Grid, _d, _d, _d, _d, _d, _i, _i, _vp]),
    "gp_create_ext": (_i, [ctypes.POINTER(Handle), Grid, _d, _d, _d, _d, _d, _i, _i, _vp, _vp,
                           ctypes.c_size_t]),
    "gp_destroy": (None, [Handle]),
    "gp_init_gaussian": (_i, [Handle]),
    "gp_set_psi": (_i, [Handle, _vp, _i]),
    "gp_get_psi": (_i, [Handle, _vp, _i]),
    "gp_set_g": (_i, [Handle, _d]),
    "gp_set_dt": (_i, [Handle, _d]),
    "gp_step_imag": (_i, [Handle, _i]),
    "gp_step_real": (_i, [Handle, _i]),
    "gp_run_imag_until": (_i, [Handle, _d, _i, _i, ctypes.POINTER(_i)]),
    "gp_observables": (_i, [Handle, ctypes.POINTER(Obs)]),
    "gp_set_tracking": (_i, [Handle, _i, _i]),
    "gp_get_tracking": (_i, [Handle, ctypes.POINTER(Obs), _i, ctypes.POINTER(_i)]),
    "gp_step_stage": (_i, [Handle, _i, _i]),
    "gp_set_stream": (_i, [Handle, _vp]),
    "gp_sync": (_i, [Handle]),
    "gp_get_window": (_i, [Handle, _i, ctypes.POINTER(_i)]),
    "gp_set_window": (_i, [Handle, _i]),
    "gp_set_axis_window": (_i, [Handle, _i, _i]),
    "gp_set_pair_lines": (_i, [Handle, _i]),
    "gp_set_lines_per_thread": (_i, [Handle, _i, _i]),
    "gp_get_lines_per_thread": (_i, [Handle, _i, ctypes.POINTER(_i)]),
    "gp_set_tma": (_i, [Handle, _i]),
    "gp_set_tma_lines": (_i, [Handle, _i]),
    "gp_get_tma_lines": (_i, [Handle, ctypes.POINTER(_i)]),
    "gp_set_stop_rule": (_i, [Handle, _i]),
    "gp_set_splitting": (_i, [Handle, _i]),
    "gp_selftest_bounded_wait": (_i, [ctypes.c_longlong, _vp, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "gp_debug_fail_alloc": (None, [_i]),
    "gp_debug_raise_status": (_i, [Handle, ctypes.c_uint]),
    "gp_run_imag_schedule": (_i, [Handle, _i, ctypes.POINTER(_d), ctypes.POINTER(_d), _i, _i,
                                  ctypes.POINTER(_i)]),
    "gp_get_tma": (_i, [Handle, ctypes.POINTER(_i)]),
    "gp_set_threads": (_i, [Handle, _i, _i]),
    "gp_set_segments": (_i, [Handle, _i, _i]),
    "gp_get_segments": (_i, [Handle, _i, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "gp_autotune": (_i, [Handle, _i, _i, ctypes.c_char_p]),
    "gp_set_graph_block": (_i, [Handle, _i]),
    "gp_psi_device_ptr": (_i, [Handle, ctypes.POINTER(_vp), ctypes.POINTER(_i)]),
    "gp_pending_scale": (_i, [Handle, ctypes.POINTER(_d)]),
    "gp_density_profiles": (_i, [Handle, ctypes.POINTER(_d), ctypes.POINTER(_d), ctypes.POINTER(_d)]),
    "gp_write_wavefunction": (_i, [Handle, ctypes.c_char_p, _i]),
    "gp_observables_noalloc": (_i, [_vp, Grid, _i, _i, _d, _d, _d, _d, _d, _vp, _vp]),
    "gp_batch_create": (_i, [ctypes.POINTER(Handle), _i, ctypes.POINTER(Grid), ctypes.POINTER(_d),
                             ctypes.POINTER(_d), ctypes.POINTER(_d), ctypes.POINTER(_d), ctypes.POINTER(_d),
                             _i, _i, _vp]),
    "gp_batch_destroy": (None, [Handle]),
    "gp_axial_create": (_i, [ctypes.POINTER(Handle), _i, _i, _d, _d, _d, _d, _d, _d, _i, _i, _vp]),
    "gp_axial_destroy": (None, [Handle]),
    "gp_axial_last_error": (ctypes.c_char_p, [Handle]),
    "gp_axial_init_gaussian": (_i, [Handle]),
    "gp_axial_set_psi": (_i, [Handle, _vp, _i]),
    "gp_axial_get_psi": (_i, [Handle, _vp, _i]),
    "gp_axial_step_imag": (_i, [Handle, _i]),
    "gp_axial_step_real": (_i, [Handle, _i]),
    "gp_axial_observables": (_i, [Handle, ctypes.POINTER(Obs)]),
    "gp_axial_run_imag_until": (_i, [Handle, _d, _i, _i, ctypes.POINTER(_i)]),
    "gp_batch_init_gaussian": (_i, [Handle]),
    "gp_batch_set_psi": (_i, [Handle, _i, _vp, _i]),
    "gp_batch_get_psi": (_i, [Handle, _i, _vp, _i]),
    "gp_batch_step_imag": (_i, [Handle, _i]),
    "gp_batch_observables": (_i, [Handle, ctypes.POINTER(Obs)]),
    "gp_batch_run_imag_until": (_i, [Handle, _d, _i, _i, ctypes.POINTER(_i)]),
    "gp_batch_get_window": (_i, [Handle, ctypes.POINTER(_i)]),
    "gp_batch_get_segments": (_i, [Handle, _i, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "gp_batch_set_segments": (_i, [Handle, _i]),
    "gp_batch_set_streams": (_i, [Handle, _i]),
    "gp_batch_set_graph_block": (_i, [Handle, _i]),
    "gp_batch_set_tma": (_i, [Handle, _i]),
    "gp_batch_get_tma": (_i, [Handle, ctypes.POINTER(_i)]),
    "gp_batch_set_stop_rule": (_i, [Handle, _i]),
    "gp_batch_set_dt_scale": (_i, [Handle, _d]),
    "gp_batch_run_imag_schedule": (_i, [Handle, _i, ctypes.POINTER(_d), ctypes.POINTER(_d), _i, _i,
                                        ctypes.POINTER(_i)]),
    "gp_batch_last_error": (ctypes.c_char_p, [Handle]),
    "gp_nn_param_count": (_i, []),
    "gp_nn_create": (_i, [ctypes.POINTER(Handle), ctypes.c_ulonglong, _vp]),
    "gp_nn_destroy": (None, [Handle]),
    "gp_nn_set_params": (_i, [Handle, ctypes.POINTER(ctypes.c_float), _i]),
    "gp_nn_get_params": (_i, [Handle, ctypes.POINTER(ctypes.c_float), _i]),
    "gp_nn_set_data": (_i, [Handle, _i, ctypes.POINTER(Grid), ctypes.POINTER(_d), ctypes.POINTER(_d),
                            ctypes.POINTER(_d), ctypes.POINTER(_d), _vp, ctypes.POINTER(ctypes.c_longlong),
                            ctypes.POINTER(ctypes.c_float)]),
    "gp_nn_train": (_i, [Handle, _i, _i, ctypes.c_float, ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_float)]),
    "gp_nn_loss_grad": (_i, [Handle, _i, ctypes.POINTER(_i), ctypes.POINTER(ctypes.c_longlong),
                             ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]),
    "gp_nn_predict": (_i, [Handle, Handle]),
    "gp_nn_predict_batch": (_i, [Handle, Handle]),
    "gp_nn_last_error": (ctypes.c_char_p, [Handle]),
    "gp_last_error": (ctypes.c_char_p, [Handle]),
    "gp_version": (ctypes.c_char_p, []),
}

_lock = threading.Lock()
_lib = None


class GPError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


def load():
    """Load libgpcn.so (built by paper_1601_04641_gb300.build)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libgpcn.so is not built (run paper_1601_04641_gb300.build.build()); "
                                   "the CUDA path has no fallback")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def check(status, handle=None, batch=False, nn=False, axial=False):
    if status != GP_OK:
        lib = load()
        if axial:
            msg = lib.gp_axial_last_error(handle)
        elif nn:
            msg = lib.gp_nn_last_error(handle)
        elif batch:
            msg = lib.gp_batch_last_error(handle)
        else:
            msg = lib.gp_last_error(handle)
        raise GPError(status, msg.decode() if msg else "")
