"""Fock-space brute force for small Gaussian boson samplers (test helper).

Independent of every determinant formula: the output state is expanded as a
polynomial in the output creation operators.  A squeezed vacuum on input j is
exp(-tanh(r_j)/2 a_j^dag^2)|0> / sqrt(cosh r_j), and the interferometer maps
a_j^dag to sum_i V_ij b_i^dag, so the output state is the truncated product of
the series exp(-t_j/2 (sum_i V_ij y_i)^2) in the variables y_i = b_i^dag.
Loss eta is a dilation: V = [sqrt(eta) U ; sqrt(1 - eta) U] on M system plus M
environment modes (the environment is summed over).  Passive optics conserve
the photon number, so truncating at total degree N gives the exact projection
of the state onto <= N photons; the missing norm is reported as ``tail``.
"""
from __future__ import annotations

import math
from itertools import product

import numpy as np


def _mul_linear(poly: np.ndarray, coef: np.ndarray, N: int, deg: np.ndarray) -> np.ndarray:
    """poly * sum_i coef[i] y_i, truncated at total degree N."""
    out = np.zeros_like(poly)
    K = poly.ndim
    for i in range(K):
        if coef[i] == 0:
            continue
        src = [slice(None)] * K
        dst = [slice(None)] * K
        src[i] = slice(0, N)
        dst[i] = slice(1, N + 1)
        out[tuple(dst)] += coef[i] * poly[tuple(src)]
    out[deg > N] = 0
    return out


def output_state(U: np.ndarray, r: np.ndarray, eta: float, N: int):
    """Amplitude array psi[n_1..n_K] (K = M, or 2M with loss) and the tail mass."""
    M = U.shape[0]
    V = U if eta == 1.0 else np.vstack([math.sqrt(eta) * U, math.sqrt(1.0 - eta) * U])
    K = V.shape[0]
    shape = (N + 1,) * K
    deg = np.indices(shape).sum(axis=0)
    poly = np.zeros(shape, dtype=np.complex128)
    poly[(0,) * K] = 1.0
    norm = 1.0
    for j in range(M):
        if r[j] == 0.0:
            continue
        t = math.tanh(r[j])
        norm /= math.sqrt(math.cosh(r[j]))
        acc = poly.copy()
        term = poly
        for l in range(1, N // 2 + 1):
            term = _mul_linear(_mul_linear(term, V[:, j], N, deg), V[:, j], N, deg)
            term = term * (-0.5 * t / l)
            acc = acc + term
        poly = acc
    fact = np.zeros(shape)
    idx = np.indices(shape)
    lf = np.zeros(shape)
    for i in range(K):
        lf += np.array([math.lgamma(k + 1) for k in range(N + 1)])[idx[i]]
    fact = np.exp(0.5 * lf)
    psi = poly * fact * norm
    psi[deg > N] = 0
    tail = 1.0 - float(np.sum(np.abs(psi) ** 2))
    return psi, tail


def click_probs(U: np.ndarray, r: np.ndarray, eta: float, N: int):
    """P(S) for all 2^M click patterns (index = bitmask) and the truncation tail."""
    M = U.shape[0]
    psi, tail = output_state(U, r, eta, N)
    p2 = np.abs(psi) ** 2
    K = psi.ndim
    if K > M:  # sum over the environment modes
        p2 = p2.sum(axis=tuple(range(M, K)))
    clicked = (np.indices(p2.shape) > 0)
    out = np.zeros(1 << M)
    mask = np.zeros(p2.shape, dtype=np.int64)
    for i in range(M):
        mask |= clicked[i].astype(np.int64) << i
    np.add.at(out, mask.reshape(-1), p2.reshape(-1))
    return out, tail


def sector_probs(U: np.ndarray, r: np.ndarray, eta: float, N: int, Z, kmax: int):
    """P(exactly k photons in the modes Z, vacuum on the other detected modes), k <= kmax."""
    M = U.shape[0]
    psi, tail = output_state(U, r, eta, N)
    p2 = np.abs(psi) ** 2
    if psi.ndim > M:
        p2 = p2.sum(axis=tuple(range(M, psi.ndim)))
    idx = np.indices(p2.shape)
    ok = np.ones(p2.shape, dtype=bool)
    for i in range(M):
        if i not in Z:
            ok &= idx[i] == 0
    tot = sum(idx[i] for i in Z) if len(Z) else np.zeros(p2.shape, dtype=np.int64)
    out = np.zeros(kmax + 1)
    for k in range(kmax + 1):
        out[k] = p2[ok & (tot == k)].sum()
    return out, tail
