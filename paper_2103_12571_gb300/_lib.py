"""ctypes binding of the C ABI declared in include/alphacirc.h.

Argument marshalling only: every numerical step runs in the CUDA library.
Loading fails loudly if the library has not been built (there is no
fallback implementation).
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libalphacirc.so")

AC_OK = 0
AC_ERR_INVALID_ARG = -1
AC_ERR_NOT_DIAGONALIZABLE = -2
AC_ERR_NO_CONVERGENCE = -3
AC_ERR_INNER_BREAKDOWN = -4
AC_ERR_CUDA = -5
AC_ERR_NOT_FINITE = -6

AC_C128, AC_C64 = 0, 1
AC_INNER_FFT, AC_INNER_BICGSTAB, AC_INNER_GMRES = 0, 1, 2
AC_ALPHA_FIXED, AC_ALPHA_PAPER, AC_ALPHA_MIXED = 0, 1, 2
AC_STOP_RESIDUAL, AC_STOP_PAPER = 0, 1
AC_FORM_CORRECTION, AC_FORM_PAPER = 0, 1
AC_UPDATE_PLAIN, AC_UPDATE_TMA = 0, 1
AC_MAX_STATS = 128


class Problem(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("nu", ctypes.c_double),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double), ("order", ctypes.c_int),
                ("upwind", ctypes.c_int)]


class Schedule(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("alpha0", ctypes.c_double), ("m0", ctypes.c_double),
                ("tau", ctypes.c_double), ("max_iter", ctypes.c_int), ("stop_rule", ctypes.c_int),
                ("inner_max_iter", ctypes.c_int), ("form", ctypes.c_int), ("inner_restart", ctypes.c_int),
                ("update_kernel", ctypes.c_int), ("space_cluster", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int),
                ("res_rel", ctypes.c_double * AC_MAX_STATS), ("alpha", ctypes.c_double * AC_MAX_STATS),
                ("m", ctypes.c_double * AC_MAX_STATS), ("diff_last", ctypes.c_double * AC_MAX_STATS),
                ("inner_iters", ctypes.c_int * AC_MAX_STATS), ("inner_failed", ctypes.c_int * AC_MAX_STATS),
                ("w_norm2", ctypes.c_double),
                ("w_inf", ctypes.c_double)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("M", ctypes.c_int), ("L", ctypes.c_int), ("F", ctypes.c_int),
                ("tile_fwd", ctypes.c_int), ("tile_upd", ctypes.c_int), ("spatial_path", ctypes.c_int),
                ("workspace_bytes", ctypes.c_longlong), ("launches", ctypes.c_longlong),
                ("update_kernel", ctypes.c_int), ("update_tile_tma", ctypes.c_int),
                ("space_cluster", ctypes.c_int)]


_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_PROTOS = {
    "ac_setup": (_I, [ctypes.POINTER(Problem), _I, _I, _D, ctypes.POINTER(Schedule), _I, _I,
                      ctypes.POINTER(_P)]),
    "ac_destroy": (None, [_P]),
    "ac_plan_get_info": (_I, [_P, ctypes.POINTER(PlanInfo)]),
    "ac_apply_C": (_I, [_P, _P, _P, _P]),
    "ac_apply_CT": (_I, [_P, _P, _P, _P]),
    "ac_precond_solve": (_I, [_P, _D, _P, _P, _P]),
    "ac_collocation_rhs": (_I, [_P, _P, _P, _P]),
    "ac_richardson_step": (_I, [_P, _D, _P, _P, _P, ctypes.POINTER(_D), _P]),
    "ac_richardson_step_host": (_I, [_P, _D, _P, _P, _P, _I, ctypes.POINTER(_D), _P]),
    "ac_plan_shape": (_I, [ctypes.POINTER(Problem), _I, _I, _I, _I, ctypes.POINTER(Schedule), ctypes.POINTER(PlanInfo)]),
    "ac_richardson_solve": (_I, [_P, _P, _P, _P, _I, _D, ctypes.POINTER(Stats), _P]),
    "ac_adjoint_solve": (_I, [_P, _P, _P, _D, ctypes.POINTER(Stats), _P]),
    "ac_window_solve": (_I, [_P, _P, _I, _P, _P, _D, ctypes.POINTER(Stats), ctypes.POINTER(_I), _P]),
    "ac_grad_params": (_I, [_P, _P, _P, _P, _P, _P]),
    "ac_precond_solve_noalloc": (_I, [ctypes.POINTER(Problem), _I, _I, _D, _D, _I, _P, _P, _P]),
    "ac_sequential_solve": (_I, [_P, _P, _P, _P, _P]),
    "ac_krylov_solve": (_I, [_P, _P, _P, _P, _I, _D, _I, _P, _P]),
    "ac_radau_nodes": (_I, [_I, _P]),
    "ac_stencil_taps": (_I, [ctypes.POINTER(Problem), _P, _P, _P]),
    "ac_collocation_matrix": (_I, [_I, _P]),
    "ac_freq_tables": (_I, [_I, _I, _D, _I, _P, _P, _P, _P]),
    "ac_alpha_sequence": (_I, [_D, _D, _I, _P, _P]),
    "ac_profile_enable": (_I, [_P, _I]),
    "ac_measure_fp64_fma_rate": (_I, [_P, _P]),
    "ac_profile_read": (_I, [_P, _I, ctypes.POINTER(ctypes.c_char_p), _P, _P]),
    "ac_status_string": (ctypes.c_char_p, [_I]),
    "ac_last_error": (ctypes.c_char_p, []),
}

_lib = None


def lib():
    """The loaded library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                "libalphacirc.so is not built (expected at %s); run "
                "`python -m paper_2103_12571_gb300.build` (nvcc, sm_103a)" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _PROTOS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class ACError(RuntimeError):
    def __init__(self, code, where):
        L = lib()
        msg = "%s: %s (%d): %s" % (where, L.ac_status_string(code).decode(), code,
                                   L.ac_last_error().decode())
        super().__init__(msg)
        self.code = code


def check(code, where):
    if code != AC_OK:
        raise ACError(code, where)
    return code
