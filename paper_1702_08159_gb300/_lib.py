"""ctypes loader for libmck.so (the C ABI declared in include/mck.h).

The library is built in-tree by ``paper_1702_08159_gb300.build``. Loading
fails loudly when it is missing: there is no fallback implementation.
"""

import ctypes
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libmck.so")

MCK_OK = 0
MCK_EINVAL = -1
MCK_ENOMEM = -2
MCK_ECUDA = -3
MCK_ETIMEOUT = -4
MCK_EUNSUPPORTED = -5

MCK_RBF = 0
MCK_MATERN = 1
MCK_LAPLACE = 2
MCK_FP32 = 0
MCK_BF16 = 1
MCK_FP16 = 2
MCK_BF16_SPLIT = 3
MCK_FP16_SPLIT = 4
PRECISIONS = {"fp32": 0, "bf16": 1, "fp16": 2, "bf16_split": 3, "fp16_split": 4}
FWHT_REGIMES = {"auto": 0, "cluster_2_15": 1, "cluster_2_14": 2, "two_pass": 3}

MAX_LOG2_D = 20
MAX_LOG2_D_MATERN = 15
MAX_LOG2_D_FWHT = 20
MAX_CLASSES = 16

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_U64 = ctypes.c_uint64
_D = ctypes.c_double
_ST = ctypes.c_int

# name -> (restype, argtypes); the same list as include/mck.h.
SIGNATURES = {
    "mck_plan": (_ST, [ctypes.POINTER(_P), _I64, _I32, _I32, _D, _U64]),
    "mck_plan_ex": (_ST, [ctypes.POINTER(_P), _I64, _I32, _I32, _D, _I32, _U64, _I32]),
    "mck_plan_destroy": (None, [_P]),
    "mck_plan_info": (_ST, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                            ctypes.POINTER(_D), ctypes.POINTER(_I32), ctypes.POINTER(_U64),
                            ctypes.POINTER(_I32)]),
    "mck_plan_tables": (_ST, [_P, _P, _P, _P, _P]),
    "mck_plan_set_signs": (_ST, [_P, _P, _P]),
    "mck_fwht": (_ST, [_P, _I64, _I64, _I32, _P]),
    "mck_fwht_ex": (_ST, [_P, _I64, _I64, _I32, _I32, _P]),
    "mck_plan_set_launch": (_ST, [_P, _I32, _I32]),
    "mck_host_pipe_create": (_ST, [ctypes.POINTER(_P), _P, _I64, _I64, _I32]),
    "mck_features_host": (_ST, [_P, _P, _I64, _I64, _P, _P, _P, _P]),
    "mck_host_pipe_destroy": (None, [_P]),
    "mck_plan_get_launch": (_ST, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    "mck_features": (_ST, [_P, _P, _I64, _I64, _I64, _P, _P, _P, _P]),
    "mck_features_ex": (_ST, [_P, _P, _I64, _I64, _I64, _P, _P, _P, _I32, _P]),
    "mck_features_backward": (_ST, [_P, _P, _I64, _I64, _I64, _P, _P, _P, _P, _P, _P, _P]),
    "mck_features_backward_ex": (_ST, [_P, _P, _I64, _I64, _I64, _P, _P, _P, _P, _P, _P, _P,
                                       _P]),
    "mck_fused_logits": (_ST, [_P, _P, _I64, _I64, _I64, _P, _P, _P, _P, _I32, _P, _P]),
    "mck_fused_logits_ex": (_ST, [_P, _P, _I64, _I64, _I64, _P, _P, _P, _P, _I32, _P, _I32, _P]),
    "mck_fused_logits_noalloc": (_ST, [_P, _P, _I64, _I64, _I64, _P, _P, _P, _P, _I32, _P, _P]),
    "mck_fused_logits_backward": (_ST, [_P, _P, _I64, _I64, _I64, _P, _P, _P, _I32, _P, _P, _P,
                                        _P, _P, _P, _P]),
    "mck_fused_logits_backward_ex": (_ST, [_P, _P, _I64, _I64, _I64, _P, _P, _P, _I32, _P, _P,
                                           _P, _P, _P, _P, _P, _P]),
    "mck_softmax_xent": (_ST, [_P, _P, _I64, _I32, _P, _P, _P]),
    "mck_group_create": (_ST, [ctypes.POINTER(_P), _P, _I32, _P, _I64, _I64, _I64, _I32]),
    "mck_group_set_grain": (_ST, [_P, _I32]),
    "mck_group_info": (_ST, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                             ctypes.POINTER(_I32)]),
    "mck_group_features": (_ST, [_P, _P, _P, _P]),
    "mck_group_destroy": (None, [_P]),
    "mck_status_string": (ctypes.c_char_p, [_ST]),
    "mck_last_error": (ctypes.c_char_p, []),
}



class GroupItem(ctypes.Structure):
    """mck_group_item_t."""
    _fields_ = [("plan", _I32), ("E", _I32), ("in_dim", _I64), ("x_offset", _I64),
                ("phi_offset", _I64)]


_lib = None


class MckError(RuntimeError):
    """A libmck call returned a status other than MCK_OK."""

    def __init__(self, status, where, detail):
        self.status = status
        super().__init__(f"{where}: {detail} [status {status}]")


def load():
    """Load libmck.so once and attach argument types; raises if it is not built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with `python -m paper_1702_08159_gb300.build` "
                "(or __graft_entry__.build()); there is no fallback path")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(status, where):
    if status != MCK_OK:
        lib = load()
        detail = lib.mck_last_error().decode(errors="replace")
        name = lib.mck_status_string(status).decode()
        raise MckError(status, where, f"{name}; {detail}")
