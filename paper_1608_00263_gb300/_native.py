"""ctypes binding of the C ABI in include/qs.h (argument marshalling only).

Every computation happens in ``libqs.so``; this module converts Python
arguments to pointers and sizes and raises ``QSError`` on a non-zero status.
The library must be built (``paper_1608_00263_gb300.build.build()``); there
is no fallback path: a missing library raises at import of the functions.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# QS_CHECKED=1 selects the checked build (device-side index checks)
CHECKED = os.environ.get("QS_CHECKED") == "1"
LIB_PATH = os.path.join(_PKG, "libqs_checked.so" if CHECKED else "libqs.so")

QS_OK, QS_ERR_INVALID_ARG, QS_ERR_OOM, QS_ERR_CUDA, QS_ERR_TIMEOUT, QS_ERR_UNSUPPORTED = range(6)
QS_C64, QS_C128 = 0, 1
(QS_H, QS_X_HALF, QS_Y_HALF, QS_T, QS_CZ, QS_RX, QS_RY, QS_RZ, QS_CPHASE) = range(9)
QS_MODE_PLAIN, QS_MODE_FUSED, QS_MODE_FUSED_TC = 0, 1, 2
(QS_PREC_DEFAULT, QS_PREC_FP16X3, QS_PREC_BF16X3, QS_PREC_BF16X6, QS_PREC_TF32X3,
 QS_PREC_TF32) = range(6)
QS_BATCH_PERSISTENT, QS_BATCH_ROUNDS = 0, 1

GATE_DTYPE = np.dtype([("kind", np.uint8), ("q0", np.uint8), ("q1", np.uint8),
                       ("pad", np.uint8), ("cycle", np.uint32), ("theta", np.float64)])

STATUS_NAMES = {0: "QS_OK", 1: "QS_ERR_INVALID_ARG", 2: "QS_ERR_OOM", 3: "QS_ERR_CUDA",
                4: "QS_ERR_TIMEOUT", 5: "QS_ERR_UNSUPPORTED"}


class QSError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


class qs_opts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("precision", ctypes.c_int), ("k", ctypes.c_int),
                ("tile_log2", ctypes.c_int), ("autotune", ctypes.c_int)]


class qs_plan_stats(ctypes.Structure):
    _fields_ = [("passes", ctypes.c_int), ("phases", ctypes.c_int), ("ops", ctypes.c_int),
                ("tile_log2", ctypes.c_int), ("reg_log2", ctypes.c_int), ("gates", ctypes.c_int),
                ("bytes", ctypes.c_double)]


# Every function the header declares, with its ctypes signature.
P = ctypes.c_void_p
D = ctypes.c_double
U64 = ctypes.c_uint64
PD = ctypes.POINTER(ctypes.c_double)
SIGNATURES = {
    "qs_version": (ctypes.c_char_p, []),
    "qs_batch_correlation": (ctypes.c_int, [P, P, P]),
    "qs_batch_apply": (ctypes.c_int, [P, P, P]),
    "qs_single_error_circuit": (ctypes.c_int, [P, ctypes.c_size_t, ctypes.c_int, ctypes.c_uint32, ctypes.c_int,
                                               ctypes.c_int, P, ctypes.POINTER(ctypes.c_size_t)]),
    "qs_batch_mean_probabilities": (ctypes.c_int, [P, P]),
    "qs_batch_sample": (ctypes.c_int, [P, U64, U64, D, P]),
    "qs_noisy_circuit": (ctypes.c_int, [P, ctypes.c_size_t, ctypes.c_int, D, D, D, U64, P,
                                        ctypes.POINTER(ctypes.c_size_t)]),
    "qs_circuit_generate_dense": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, U64, P,
                                                 ctypes.POINTER(ctypes.c_size_t)]),
    "qs_pt_convergence": (ctypes.c_int, [P, ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
    "qs_last_error": (ctypes.c_char_p, []),
    "qs_state_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, P, ctypes.POINTER(P)]),
    "qs_state_attach": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, P, P, ctypes.POINTER(P)]),
    "qs_state_destroy": (ctypes.c_int, [P]),
    "qs_state_amplitudes": (ctypes.c_int, [P, ctypes.POINTER(P)]),
    "qs_state_reset": (ctypes.c_int, [P]),
    "qs_apply_circuit": (ctypes.c_int, [P, P, ctypes.c_size_t, ctypes.POINTER(qs_opts)]),
    "qs_prepare_circuit": (ctypes.c_int, [P, P, ctypes.c_size_t, ctypes.POINTER(qs_opts)]),
    "qs_plan_circuit": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, P, ctypes.c_size_t,
                                       ctypes.POINTER(qs_opts), ctypes.POINTER(qs_plan_stats)]),
    "qs_probabilities": (ctypes.c_int, [P, P, ctypes.c_int]),
    "qs_probabilities_async": (ctypes.c_int, [P, P, ctypes.c_int]),
    "qs_state_sync": (ctypes.c_int, [P]),
    "qs_readout_share": (ctypes.c_int, [P, ctypes.c_double, P]),
    "qs_sample": (ctypes.c_int, [P, U64, U64, P]),
    "qs_sample_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, P, P, U64, U64, P]),
    "qs_cross_entropy": (ctypes.c_int, [P, P, U64, PD, PD]),
    "qs_pt_moments": (ctypes.c_int, [P, ctypes.c_int, PD, PD, PD, PD]),
    "qs_adjoint_gradient": (ctypes.c_int, [P, P, ctypes.c_size_t, P, U64, ctypes.POINTER(qs_opts), PD, P]),
    "qs_cycle_statistics": (ctypes.c_int, [P, P, ctypes.c_size_t, ctypes.POINTER(qs_opts), ctypes.c_int, P,
                                           ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "qs_batch_create": (ctypes.c_int, [ctypes.c_int, P, P, ctypes.POINTER(P)]),
    "qs_batch_run": (ctypes.c_int, [P, P, P, ctypes.c_int, P]),
    "qs_batch_state": (ctypes.c_int, [P, ctypes.c_int, ctypes.POINTER(P)]),
    "qs_batch_destroy": (ctypes.c_int, [P]),
    "qs_state_copy_out": (ctypes.c_int, [P, P]),
    "qs_state_copy_in": (ctypes.c_int, [P, P]),
    "qs_circuit_generate": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, P, ctypes.c_int, U64, P,
                                           ctypes.POINTER(ctypes.c_size_t)]),
    "qs_alu_rate": (ctypes.c_int, [ctypes.c_int, P, PD]),
    "qs_build_flags": (ctypes.c_int, []),
    "qs_check_probe": (ctypes.c_int, []),
    "qs_batch_set_options": (ctypes.c_int, [P, ctypes.POINTER(qs_opts)]),
    "qs_batch_plan_info": (ctypes.c_int, [P, P, PD]),
    "qs_batch_set_engine": (ctypes.c_int, [P, ctypes.c_int]),
}

_lib = None


def lib():
    """Loads libqs.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError("%s is not built: run paper_1608_00263_gb300.build.build(%s)"
                          % (os.path.basename(LIB_PATH), "checked=True" if CHECKED else ""))
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(status):
    if status != QS_OK:
        msg = lib().qs_last_error()
        raise QSError(status, msg.decode() if msg else "")
