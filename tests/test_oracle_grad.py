"""Pins of the oracle gradient: closed forms for one mode, and central finite
differences (h = 1e-6) of the double-double oracle's log P through the state
build and the interferometer mesh."""
import math

import numpy as np
import pytest

import gbs_inputs as g
import oracle
from oracle import grad as og


def logp(U, r, eta, pats):
    st = oracle.build_state(U, r, eta)
    return oracle.prob_exact(st, pats, dd=True)["logP"]


def analytic(U, r, eta, pats, w):
    st = oracle.build_state(U, r, eta)
    dsq = og.grad_sigmaQ(st, pats, w)
    return og.chain_params(U, r, eta, dsq)


def test_single_mode_closed_forms():
    # P0 = (1 + eta(2-eta) sinh^2 r)^{-1/2}: d log P0 / dr and d log P0 / d eta
    for r0, eta in ((0.7, 1.0), (1.1, 0.4)):
        U = np.eye(1, dtype=complex)
        r = np.array([r0])
        pats = np.zeros((1, 2), dtype=np.uint64)
        dU, dr, deta = analytic(U, r, eta, pats, [1.0])
        a = eta * (2 - eta) * math.sinh(r0) ** 2
        assert abs(dr[0] + eta * (2 - eta) * math.sinh(r0) * math.cosh(r0) / (1 + a)) < 1e-13
        assert abs(deta + (1 - eta) * math.sinh(r0) ** 2 / (1 + a)) < 1e-13
        # the clicked pattern: log(1 - P0)
        pats1 = np.array([[1, 0]], dtype=np.uint64)
        _, dr1, deta1 = analytic(U, r, eta, pats1, [1.0])
        P0 = (1 + a) ** -0.5
        dP0dr = -eta * (2 - eta) * math.sinh(r0) * math.cosh(r0) * (1 + a) ** -1.5
        assert abs(dr1[0] - (-dP0dr / (1 - P0))) < 1e-12


def test_finite_differences_through_mesh():
    M = 5
    th, ph = g.clements_phases(M, 17)
    r = g.squeezing(M, 3, 0.5, 1.0, 17)
    eta = 0.65
    pats = np.stack([g.modes_to_pattern(m) for m in ([0, 2], [1, 3, 4], [0, 1, 2, 3], [4])])
    w = np.array([1.0, 0.5, -0.7, 2.0])
    U = g.clements_unitary(M, th, ph)
    dU, dr, deta = analytic(U, r, eta, pats, w)
    dth, dph = og.chain_clements(M, th, ph, dU)
    L = lambda U_, r_, e_: float(np.dot(w, logp(U_, r_, e_, pats)))
    h = 1e-6
    for j in range(M):
        e = np.zeros(M); e[j] = h
        fd = (L(U, r + e, eta) - L(U, r - e, eta)) / (2 * h)
        assert abs(fd - dr[j]) < 1e-6 * max(1, abs(fd)), j
    fd = (L(U, r, eta + h) - L(U, r, eta - h)) / (2 * h)
    assert abs(fd - deta) < 1e-6 * max(1, abs(fd))
    for c in (0, 3, 7, 9):
        e = np.zeros(len(th)); e[c] = h
        fd = (L(g.clements_unitary(M, th + e, ph), r, eta) - L(g.clements_unitary(M, th - e, ph), r, eta)) / (2 * h)
        assert abs(fd - dth[c]) < 1e-6 * max(1, abs(fd)), c
        fd = (L(g.clements_unitary(M, th, ph + e), r, eta) - L(g.clements_unitary(M, th, ph - e), r, eta)) / (2 * h)
        assert abs(fd - dph[c]) < 1e-6 * max(1, abs(fd)), c


def test_gradient_of_highly_cancelling_pattern():
    # a pattern whose signed sum cancels by ~1e12: the double-double adjoint still
    # matches finite differences of the double-double log P
    M = 10
    U = g.haar_unitary(M, 123)
    r = g.squeezing(M, 10, 0.3, 0.6, 123)
    eta = 0.3
    pats = g.modes_to_pattern(list(range(10)))[None]
    st = oracle.build_state(U, r, eta)
    assert oracle.prob_exact(st, pats)["kappa"][0] > 1e11
    dU, dr, deta = analytic(U, r, eta, pats, [1.0])
    h = 1e-6
    for j in (0, 5):
        e = np.zeros(M); e[j] = h
        fd = (logp(U, r + e, eta, pats)[0] - logp(U, r - e, eta, pats)[0]) / (2 * h)
        assert abs(fd - dr[j]) < 1e-5 * max(1, abs(fd))
