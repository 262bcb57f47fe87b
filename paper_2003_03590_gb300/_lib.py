"""ctypes view of libgpqt.so (declarations mirror include/gp.h)."""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgpqt.so")

GP_OK = 0
STATUS = {0: "GP_OK", 1: "GP_ERR_INVALID_ARG", 2: "GP_ERR_UNSUPPORTED_SIZE", 3: "GP_ERR_OOM",
          4: "GP_ERR_CUDA", 5: "GP_ERR_TIMEOUT", 6: "GP_ERR_NONFINITE"}
GP_FP32, GP_FP64 = 0, 1
GP_SPLIT_NKN, GP_SPLIT_KNK = 0, 1
# sweep kinds (axis, op) and kernel variants of gp_plan_sweep_variant / gp_plan_set_sweep_variant
OP_FWD, OP_INV, OP_INV_N_FWD, OP_N_FWD, OP_INV_N, OP_FWD_K_INV, OP_PLANE = 1, 2, 3, 4, 5, 6, 7
VARIANT_TMA, VARIANT_TMA_ONE, VARIANT_PLAIN, VARIANT_TMA_2STAGE, VARIANT_TMA_GROUPS = 0, 1, 2, 3, 4
GP_FLOW_NONE, GP_FLOW_TG, GP_FLOW_ABC = 0, 1, 2
SUPPORTED_N = (8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 512, 1024)


class FieldParams(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("xi", ctypes.c_double), ("alpha", ctypes.c_double),
                ("beta", ctypes.c_double), ("dt", ctypes.c_double), ("precision", ctypes.c_int),
                ("split", ctypes.c_int), ("nonlin_minus_one", ctypes.c_int)]


DIAG_NAMES = ("N", "E", "E_kin", "E_kin_i", "E_kin_c", "E_q", "E_int", "P_x", "P_y", "P_z", "M_max", "M_rms")


class Diag(ctypes.Structure):
    _fields_ = [(name, ctypes.c_double) for name in DIAG_NAMES]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_PP = ctypes.POINTER(ctypes.c_void_p)

# name -> (restype, argtypes)
SIGNATURES = {
    "gp_plan_create": (_I, [ctypes.POINTER(FieldParams), _I, _P, ctypes.POINTER(_P)]),
    "gp_plan_destroy": (_I, [_P]),
    "gp_plan_nbins": (_I, [_P, _I]),
    "gp_plan_coefficients": (_I, [_P, _I, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "gp_init_srp": (_I, [_P, _I, _P, ctypes.c_uint64, _I, _D, _D]),
    "gp_init_rvr": (_I, [_P, _I, _P, ctypes.c_uint64, _I, _I, _D, _D]),
    "gp_psi_from_phase": (_I, [_P, _I, _P, _P]),
    "gp_step": (_I, [_P, _PP, _I]),
    "gp_step_host": (_I, [_P, _PP, _I]),
    "gp_diagnostics": (_I, [_P, _I, _P, ctypes.POINTER(Diag), ctypes.POINTER(_D), _I]),
    "gp_adjoint_step": (_I, [_P, _I, _P, _P, _I]),
    "gp_ekin_i_grad": (_I, [_P, _I, _P, _P, _D, ctypes.POINTER(_D)]),
    "gp_phase_grad": (_I, [_P, _I, _P, _P, _P]),
    "gp_diagnostics_noalloc": (_I, [_I, _D, _D, _P, ctypes.POINTER(Diag), ctypes.POINTER(_D), _I, _P]),
    "gp_structure_function": (_I, [_P, _I, _P, _I, ctypes.POINTER(_D), _I]),
    "gp_helicity": (_I, [_P, _I, _P, ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_D), _I]),
    "gp_plan_autotune": (_I, [_P, ctypes.c_char_p]),
    "gp_plan_sweep_variant": (_I, [_P, _I, _I, _I]),
    "gp_plan_set_sweep_variant": (_I, [_P, _I, _I, _I, _I]),
    "gp_plan_set_fused_batch": (_I, [_P, _I]),
    "gp_plan_sync": (_I, [_P]),
    "gp_init_tg": (_I, [_P, _I, _P]),
    "gp_init_abc": (_I, [_P, _I, _P, _P]),
    "gp_argle": (_I, [_P, _I, _P, _I, _P, ctypes.c_double, _I, _I, _P]),
    "gp_argle_converge": (_I, [_P, _I, _P, _I, _P, ctypes.c_double, _I, _I, ctypes.c_double, _I,
                               ctypes.POINTER(_I), ctypes.POINTER(_D), ctypes.POINTER(_D), _P]),
    "gp_plan_test_timeout": (_I, [_P, _I]),
    "gp_profile": (_I, [_P, _I]),
    "gp_profile_read": (_I, [_P, _I, ctypes.c_char_p, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_D)]),
    "gp_launch_count": (ctypes.c_longlong, [_P]),
    "gp_last_error": (ctypes.c_char_p, [_P]),
    "gp_status_string": (ctypes.c_char_p, [_I]),
}

_lib = None


def load():
    """Load the CUDA library; raises if it has not been built (there is no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libgpqt.so not found at {LIB_PATH}: run paper_2003_03590_gb300.build.build() first")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class GPError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
