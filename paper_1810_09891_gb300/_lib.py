"""ctypes loader for ``libgbnfft.so`` (the C ABI declared in ``include/gbnfft.h``).

Only argument marshalling lives here. The library must have been built
(``python -m paper_1810_09891_gb300.build_lib`` or ``__graft_entry__.build()``); if it is
missing, loading raises immediately: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgbnfft.so")

NFFT_FP32 = 0
NFFT_FP64 = 1

STATUS = {
    0: "NFFT_OK",
    1: "NFFT_EINVAL",
    2: "NFFT_ENOMEM",
    3: "NFFT_ECUDA",
    4: "NFFT_ENOTREADY",
    5: "NFFT_EBADNODE",
    6: "NFFT_ETIMEOUT",
    7: "NFFT_EUNSUPPORTED",
    8: "NFFT_ESCRATCH",
}

# Every symbol include/gbnfft.h declares, with (argtypes, restype).
_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_PI64 = ctypes.POINTER(ctypes.c_int64)
_PSZ = ctypes.POINTER(ctypes.c_size_t)


class NfftInfo(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int),
        ("m", ctypes.c_int),
        ("dtype", ctypes.c_int),
        ("M", ctypes.c_int64),
        ("N", ctypes.c_int64 * 3),
        ("n", ctypes.c_int64 * 3),
        ("bin", ctypes.c_int64 * 3),
        ("workspace_bytes", ctypes.c_size_t),
        ("window", ctypes.c_int),
        ("window_table", ctypes.c_int),
    ]


SIGNATURES = {
    "nfft_plan_create": ([ctypes.POINTER(_P), _I, _PI64, _I64, _PI64, _I, _I], _I),
    "nfft_destroy": ([_P], _I),
    "nfft_set_stream": ([_P, _P], _I),
    "nfft_workspace_size": ([_P, _PSZ], _I),
    "nfft_set_workspace": ([_P, _P, ctypes.c_size_t], _I),
    "nfft_set_nodes": ([_P, _P], _I),
    "nfft_trafo": ([_P, _P, _P], _I),
    "nfft_adjoint": ([_P, _P, _P], _I),
    "nfft_grad_x": ([_P, _P, _P, _P], _I),
    "nfft_set_nodes_host": ([_P, _P], _I),
    "nfft_trafo_host": ([_P, _P, _P], _I),
    "nfft_adjoint_host": ([_P, _P, _P], _I),
    "nfft_status": ([_P], _I),
    "nfft_get_info": ([_P, ctypes.POINTER(NfftInfo)], _I),
    "nfft_strerror": ([_I], ctypes.c_char_p),
    "nfft_use_device": ([_I], _I),
    "nfft_set_option": ([_P, _I, _I64], _I),
    "nfft_profile": ([_P, _I], _I),
    "nfft_profile_read": ([_P, ctypes.POINTER(ctypes.c_double), _PI64, _I], _I),
    "nfft_trafo_1d_noalloc": ([_I64, _I64, _PI64, _I, _P, _P, _P, _P], _I),
    # batches: pointer arrays are passed as the address of a ctypes array of c_void_p
    "nfft_batch_create": ([ctypes.POINTER(_P), _P, _I, _I], _I),
    "nfft_batch_destroy": ([_P], _I),
    "nfft_batch_set_stream": ([_P, _P], _I),
    "nfft_batch_size": ([_P, ctypes.POINTER(_I), ctypes.POINTER(_I)], _I),
    "nfft_batch_lane": ([_P, _I], _I),
    "nfft_batch_trafo": ([_P, _P, _P], _I),
    "nfft_batch_adjoint": ([_P, _P, _P], _I),
    "nfft_batch_grad_x": ([_P, _P, _P, _P], _I),
    "nfft_batch_set_fused": ([_P, _I], _I),
    "nfft_batch_get_fused": ([_P, ctypes.POINTER(_I)], _I),
}

OPT_SPREAD_METHOD = 1
OPT_BIN = (2, 3, 4)
OPT_INTERP_METHOD = 5
OPT_WINDOW = 6
OPT_SUBPROBLEM = 7
OPT_WINDOW_TABLE = 8
OPT_STRIPE_ITEM = 9
WINDOWS = {"kaiser_bessel": 0, "gaussian": 1, "bspline": 2, "sinc": 3}
INTERP_METHODS = {"auto": 0, "thread": 1, "warp": 2, "tile": 3, "octet": 4}
SPREAD_METHODS = {"auto": 0, "thread": 1, "warp_atomic": 2, "warp_private": 3, "octet": 4,
                  "half": 5, "plane": 6, "stripe": 7, "rows": 8}

STAGES = ["set_nodes", "fft_forward", "interp", "zero_grid", "spread", "fft_adjoint", "grad"]

_lock = threading.Lock()
_lib = None


class NfftError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        name = STATUS.get(code, str(code))
        msg = ""
        try:
            msg = lib().nfft_strerror(code).decode()
        except Exception:  # pragma: no cover - strerror is always exported
            pass
        super().__init__(f"{where}: {name} ({msg})")


def lib():
    """Load the shared library (once); raise if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"libgbnfft.so not found at {LIB_PATH}: build it with "
                "`python -m paper_1810_09891_gb300.build_lib` (needs nvcc); there is no CPU path")
        h = ctypes.CDLL(LIB_PATH)
        for name, (argt, rest) in SIGNATURES.items():
            fn = getattr(h, name)
            fn.argtypes = argt
            fn.restype = rest
        _lib = h
        return h


def check(code: int, where: str) -> None:
    if code != 0:
        raise NfftError(code, where)
