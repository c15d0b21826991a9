"""ctypes declarations of the libgbs C ABI (include/gbs.h).  Marshalling only."""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(_PKG, "libgbs.so")

GBS_OK, GBS_E_INVALID, GBS_E_CUDA, GBS_E_NOMEM, GBS_E_NONPOSITIVE, GBS_E_NOT_SPD, GBS_E_TIMEOUT, \
    GBS_E_FIT, GBS_E_RANGE, GBS_E_FLOOR = range(10)
GBS_FP64, GBS_FP32_SPLIT, GBS_DD, GBS_FX, GBS_FF, GBS_AUTO, GBS_FX192 = 0, 1, 2, 3, 4, 5, 6
STATUS_NAMES = {0: "ok", 1: "invalid", 2: "cuda", 3: "nomem", 4: "nonpositive", 5: "not_spd",
                6: "timeout", 7: "fit", 8: "range", 9: "floor"}

_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double
_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32

# name -> (restype, argtypes); the same names as include/gbs.h
SIGNATURES = {
    "gbs_create": (_i, [ctypes.POINTER(_vp), _i, _vp]),
    "gbs_destroy": (_i, [_vp]),
    "gbs_set_stream": (_i, [_vp, _vp]),
    "gbs_last_error": (ctypes.c_char_p, [_vp]),
    "gbs_version": (_i, []),
    "gbs_reserve": (_i, [_vp, _i, _i]),
    "gbs_click_distribution": (_i, [_vp, _i, _vp, _vp, _vp, _vp]),
    "gbs_sector_distribution": (_i, [_vp, _i, _vp, _vp, _i, _d, _i, _i, _i, _vp]),
    "gbs_approx_sector_curves": (_i, [_vp, _i, _vp, _vp, _vp, _i, _i, _i, _i, _vp, _vp, _vp]),
    "gbs_autotune": (_i, [_vp, _i, _vp, _vp, _vp, _i, _i, ctypes.POINTER(_i), ctypes.POINTER(_d)]),
    "gbs_build_state": (_i, [_vp, _i, _vp, _vp, _d, _vp, _vp, _vp, _vp]),
    "gbs_prob": (_i, [_vp, _i, _vp, _vp, _vp, _i, _i, _i, _vp, _vp, _vp, _vp]),
    "gbs_run_host": (_i, [_vp, _i, _vp, _vp, _d, _vp, _i, _i, _i, _vp, _vp, _vp, _vp]),
    "gbs_prob_noalloc": (_i, [_vp, _i, _vp, _vp, _vp, _i, _i, _i, _vp, _vp, _vp, _vp]),
    "gbs_prob_partial": (_i, [_vp, _i, _vp, _vp, _i, _i, _i, _i, _vp, _vp]),
    "gbs_prob_combine": (_i, [_vp, _vp, _vp, _i, _i, _i, _vp, _vp, _vp, _vp, _vp, _vp]),
    "gbs_gen_patterns": (_i, [_vp, _u64, _u32, _i, _i, _i, _i, _vp]),
    "gbs_grad": (_i, [_vp, _i, _vp, _vp, _vp, _i, _vp, _vp, _vp, _vp]),
    "gbs_grad_approx": (_i, [_vp, _i, _vp, _vp, _vp, _i, _i, _vp, _vp, _vp, _vp]),
    "gbs_grad_params": (_i, [_vp, _i, _vp, _vp, _d, _vp, _vp, _vp, _vp]),
    "gbs_clements_unitary": (_i, [_vp, _i, _vp, _vp, _vp]),
    "gbs_clements_grad": (_i, [_vp, _i, _vp, _vp, _vp, _vp, _vp, _vp]),
    "gbs_peak_flops": (_i, [_vp, _i, ctypes.POINTER(_d)]),
    "gbs_set_pair_from": (_i, [_vp, _i]),
    "gbs_timing_enable": (_i, [_vp, _i]),
    "gbs_timing_read": (_i, [_vp, _i, ctypes.POINTER(_d), ctypes.POINTER(ctypes.c_longlong)]),
}

_lock = threading.Lock()
_lib = None


def load(path: str = SO_PATH) -> ctypes.CDLL:
    """Load libgbs.so.  There is no fallback: a missing library is an error."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise ImportError("libgbs.so is not built (run `python -m paper_2106_01445_gb300.build`)")
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


class GbsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("libgbs error %d (%s): %s" % (code, STATUS_NAMES.get(code, "?"), msg))
        self.code = code
