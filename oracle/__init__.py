"""FP64 CPU oracle for threshold-detector click-pattern probabilities.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The CUDA library never
imports, links or runs anything here, and nothing here uses the library.

* ``oracle.c``   -- state build and the exact signed subset sum, one Cholesky
  per subset, Sum2 compensated accumulation (C, OpenMP over patterns); a
  double-double variant for sums that cancel beyond FP64 precision.
* ``approx.py``  -- the paper's moment approximation, step by step, with
  exact power series of every minor's generating function (numpy).
* ``grad.py``    -- gradients of log P from the trace formula, per subset in
  double-double (C), chained to (r, eta, U) and the mesh phases (numpy).
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into _liboracle.so (gcc, OpenMP, no fast-math)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + ".%d.tmp" % os.getpid()
        # fused multiply-add in hardware where the ISA has it as an option (the
        # result of fma() is the same correctly rounded value either way)
        isa = ["-mfma"] if platform.machine() in ("x86_64", "AMD64") else []
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-fno-fast-math", "-ffp-contract=off", *isa, src, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            up = ctypes.POINTER(ctypes.c_uint64)
            L.orc_build_state.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, dp, dp, dp, dp, dp]
            L.orc_subset_sum.argtypes = [ctypes.c_int, dp, ip, ctypes.c_int, ctypes.c_uint64,
                                         ctypes.c_uint64, dp]
            L.orc_subset_sum_parallel.argtypes = [ctypes.c_int, dp, ip, ctypes.c_int, ctypes.c_int,
                                                  ctypes.c_int, dp]
            L.orc_prob_exact.argtypes = [ctypes.c_int, dp, ctypes.c_double, up, ctypes.c_int, dp, dp,
                                         dp, ip, ctypes.c_int, ctypes.c_int]
            L.orc_subset_sum_dd.argtypes = L.orc_subset_sum.argtypes
            L.orc_subset_sum_dd_parallel.argtypes = L.orc_subset_sum_parallel.argtypes
            L.orc_grad_subsets_dd.argtypes = [ctypes.c_int, dp, ip, ctypes.c_int, dp, dp, dp]
            L.orc_max_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _p(a, t=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(t))


class State:
    """sigma, sigma_Q, A = sigma_Q^{-1}, O = I - A (2M x 2M, xp order) and log det sigma_Q."""

    def __init__(self, M, sigma, sigmaQ, A, O, logdet):
        self.M, self.sigma, self.sigmaQ, self.A, self.O, self.logdet = M, sigma, sigmaQ, A, O, logdet


def build_state(U: np.ndarray, r: np.ndarray, eta: float) -> State:
    U = np.ascontiguousarray(U, dtype=np.complex128)
    M = U.shape[0]
    Ui = np.ascontiguousarray(U.view(np.float64).reshape(M, 2 * M))
    r = np.ascontiguousarray(r, dtype=np.float64)
    mats = [np.zeros((2 * M, 2 * M)) for _ in range(4)]
    ld = np.zeros(1)
    st = lib().orc_build_state(M, _p(Ui), _p(r), float(eta), *[_p(m) for m in mats], _p(ld))
    if st:
        raise ValueError("oracle state build failed with status %d" % st)
    return State(M, *mats, float(ld[0]))


def subset_sum(A: np.ndarray, M: int, modes, z_begin: int = 0, z_end: int | None = None,
               nchunk: int = 0, nthreads: int = 0, dd: bool = False):
    """(T_hi, T_lo, sum|tau|) of the signed subset sum over the given mask range
    (dd=True: double-double subset determinants and sum)."""
    modes = np.ascontiguousarray(modes, dtype=np.int32)
    n = modes.size
    A = np.ascontiguousarray(A, dtype=np.float64)
    out = np.zeros(3)
    if nchunk:
        f = lib().orc_subset_sum_dd_parallel if dd else lib().orc_subset_sum_parallel
        st = f(M, _p(A), _p(modes, ctypes.c_int), n, nchunk, nthreads, _p(out))
    else:
        z_end = (1 << n) if z_end is None else z_end
        f = lib().orc_subset_sum_dd if dd else lib().orc_subset_sum
        st = f(M, _p(A), _p(modes, ctypes.c_int), n, z_begin, z_end, _p(out))
    if st:
        raise ValueError("oracle subset sum failed with status %d" % st)
    return out


def prob_exact(state: State, patterns: np.ndarray, nthreads: int = 0, dd: bool = False):
    """Exact log P per pattern (dd=True: double-double arithmetic).
    Returns dict(logP, T(hi,lo), sumabs, kappa, status)."""
    pats = np.ascontiguousarray(patterns, dtype=np.uint64).reshape(-1, 2)
    n_pat = pats.shape[0]
    logP, T, sabs = np.zeros(n_pat), np.zeros((n_pat, 2)), np.zeros(n_pat)
    status = np.zeros(n_pat, dtype=np.int32)
    lib().orc_prob_exact(state.M, _p(np.ascontiguousarray(state.A)), state.logdet,
                         _p(pats, ctypes.c_uint64), n_pat, _p(logP), _p(T), _p(sabs),
                         _p(status, ctypes.c_int), nthreads, 1 if dd else 0)
    t = T[:, 0] + T[:, 1]
    with np.errstate(divide="ignore", invalid="ignore"):
        kappa = sabs / np.abs(t)
    return dict(logP=logP, T=T, sumabs=sabs, kappa=kappa, status=status)


def max_threads() -> int:
    return int(lib().orc_max_threads())
