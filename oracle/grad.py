"""Oracle gradients of L = sum_p w_p log P_p (test infrastructure only).

Not in the paper.  From the signed subset sum (Methods, "Probability of any
sample"): log P = -1/2 log det sigma_Q + log T(A_S), A = sigma_Q^{-1}, and
    dT = tr(Gbar dA_S),  Gbar = sum_Z (-1)^{n-|Z|} (-1/2) tau_Z A_Z^{-1}   (per subset, double-double),
    dA = -A dsigma_Q A
  => dL/dsigma_Q = -1/2 (sum_p w_p) A - A H A,   H = sum_p (w_p / T_p) embed(Gbar_p).
Chain to the physical parameters with sigma_Q = eta R diag(d) R^T + (1 - eta/2) I,
d = (e^{-2r}/2 on x, e^{2r}/2 on p), R the xp form of U, and through the
rectangular mesh U = T_last ... T_1 of cells T(theta, phi) on modes (m, m+1).
The same chain carries the gradient of the moment approximation (grad_sigmaQ_approx).
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import _p, lib


def gbar_subsets(A: np.ndarray, M: int, modes):
    """(Gbar as a 2n x 2n float array from hi + lo, T as (hi, lo))."""
    modes_a = np.ascontiguousarray(modes, dtype=np.int32)
    n = modes_a.size
    gh = np.zeros((2 * n, 2 * n))
    gl = np.zeros((2 * n, 2 * n))
    T = np.zeros(2)
    st = lib().orc_grad_subsets_dd(M, _p(np.ascontiguousarray(A)), _p(modes_a, ctypes.c_int), n,
                                   _p(gh), _p(gl), _p(T))
    if st:
        raise ValueError("oracle gradient failed with status %d" % st)
    return gh, gl, T


def grad_sigmaQ(state, patterns, w) -> np.ndarray:
    """dL/dsigma_Q (2M x 2M, symmetric) for L = sum_p w_p log P_p."""
    from gbs_inputs import pattern_modes
    M = state.M
    H = np.zeros((2 * M, 2 * M))
    for p, wp in zip(patterns, w):
        modes = pattern_modes(p)
        gh, gl, T = gbar_subsets(state.A, M, modes)
        # Gbar / T: the cancellation of both is resolved by the double-double sums
        scale = wp / (T[0] + T[1])
        G = (gh + gl) * scale
        rows = []
        for m in modes:
            rows += [m, m + M]
        H[np.ix_(rows, rows)] += G
    return -0.5 * float(np.sum(w)) * state.A - state.A @ H @ state.A


def grad_sigmaQ_approx(state, patterns, w, order: int):
    """dL/dsigma_Q for L = sum_p w_p log P_p with the order-j approximation of every P_p
    (oracle/approx.py: approx_logprob_grad); the same chain as grad_sigmaQ.  Returns
    (dL/dsigma_Q, log P per pattern)."""
    from gbs_inputs import pattern_modes
    from .approx import approx_logprob_grad, sub_rows
    M = state.M
    H = np.zeros((2 * M, 2 * M))
    logP = []
    for p, wp in zip(patterns, w):
        modes = pattern_modes(p)
        lp, g = approx_logprob_grad(state.O, state.logdet, M, modes, order)
        logP.append(lp)
        rows = sub_rows(modes, M)
        H[np.ix_(rows, rows)] += wp * g
    return -0.5 * float(np.sum(w)) * state.A - state.A @ H @ state.A, np.array(logP)


def xp_form(U: np.ndarray) -> np.ndarray:
    return np.block([[U.real, -U.imag], [U.imag, U.real]])


def chain_params(U: np.ndarray, r: np.ndarray, eta: float, dsq: np.ndarray):
    """dL/dU (complex: d/dRe U + i d/dIm U), dL/dr, dL/deta from dL/dsigma_Q."""
    M = U.shape[0]
    R = xp_form(U)
    W = 0.5 * (dsq + dsq.T)
    dx, dp = 0.5 * np.exp(-2 * r), 0.5 * np.exp(2 * r)
    d = np.concatenate([dx, dp])
    RWR = R.T @ W @ R
    dr = eta * (-2 * dx * np.diag(RWR)[:M] + 2 * dp * np.diag(RWR)[M:])
    deta = float(np.sum(d * np.diag(RWR)) - 0.5 * np.trace(W))
    dR = 2 * eta * W @ R @ np.diag(d)
    dU = (dR[:M, :M] + dR[M:, M:]) + 1j * (-dR[:M, M:] + dR[M:, :M])
    return dU, dr, deta


def chain_clements(M: int, theta: np.ndarray, phi: np.ndarray, dU: np.ndarray):
    """dL/dtheta, dL/dphi of the mesh U = T_last ... T_1, from dL/dU (complex)."""
    from gbs_inputs import clements_cells
    cells = clements_cells(M)
    # forward pass keeping the rows each cell read
    U = np.eye(M, dtype=complex)
    saved = []
    for c, m in enumerate(cells):
        rows = U[[m, m + 1], :].copy()
        saved.append(rows)
        ct, st, e = math.cos(theta[c]), math.sin(theta[c]), complex(math.cos(phi[c]), math.sin(phi[c]))
        U[m, :] = e * ct * rows[0] - st * rows[1]
        U[m + 1, :] = e * st * rows[0] + ct * rows[1]
    G = dU.copy()                                   # dL/dU, Wirtinger-style: Re/Im parts
    dth = np.zeros(len(cells))
    dph = np.zeros(len(cells))
    for c in range(len(cells) - 1, -1, -1):
        m = cells[c]
        a, b = saved[c]
        ct, st, e = math.cos(theta[c]), math.sin(theta[c]), complex(math.cos(phi[c]), math.sin(phi[c]))
        g0, g1 = G[m, :].copy(), G[m + 1, :].copy()
        # outputs o0 = e ct a - st b, o1 = e st a + ct b; dL = Re sum conj(g) do
        do0_dth, do1_dth = -e * st * a - ct * b, e * ct * a - st * b
        do0_dph, do1_dph = 1j * e * ct * a, 1j * e * st * a
        dth[c] = np.real(np.sum(np.conj(g0) * do0_dth + np.conj(g1) * do1_dth))
        dph[c] = np.real(np.sum(np.conj(g0) * do0_dph + np.conj(g1) * do1_dph))
        # adjoint of the inputs: dL/da = conj(e) ct g0 + conj(e) st g1, dL/db = -st g0 + ct g1
        G[m, :] = np.conj(e) * ct * g0 + np.conj(e) * st * g1
        G[m + 1, :] = -st * g0 + ct * g1
    return dth, dph
