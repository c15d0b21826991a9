"""The oracle's whole-device sectors p_k(n) (the probability of n clicks with k photons),
pinned by quantities it does not compute itself: the click-number distribution from the
determinant oracle (sum over k), and the total photon-number distribution, which for a
passive interferometer with uniform loss is the convolution over the inputs of each
squeezed vacuum's photon distribution thinned binomially by eta (sum over n)."""
import math

import numpy as np
import pytest

import gbs_inputs as g
import oracle
from oracle import approx as ap


def photon_distribution(r, eta, K):
    """P(N = k), k = 0..K: single-mode squeezed vacuum P(2j) = tanh(r)^(2j) (2j)! /
    (4^j j!^2) / cosh(r), thinned by eta (each photon kept with probability eta),
    convolved over the modes."""
    Kb = 8 * K  # the input photon numbers that thin down to <= K (tail below 1e-20 here)
    tot = np.zeros(K + 1)
    tot[0] = 1.0
    for rr in r:
        p = np.zeros(Kb + 1)
        th = math.tanh(rr)
        for j in range(Kb // 2 + 1):
            p[2 * j] = th ** (2 * j) * math.comb(2 * j, j) / 4.0 ** j / math.cosh(rr)
        q = np.array([sum(p[n] * math.comb(n, m) * eta ** m * (1 - eta) ** (n - m) for n in range(m, Kb + 1))
                      for m in range(K + 1)])
        tot = np.convolve(tot, q)[:K + 1]
    return tot


@pytest.mark.parametrize("eta", [1.0, 0.6])
def test_sectors_sum_to_click_distribution(eta):
    M = 6
    U, r = g.haar_unitary(M, 11), g.squeezing(M, 3, 0.7, 0.9, 11)
    st = oracle.build_state(U, r, eta)
    pkn = ap.sector_distribution(st.O, st.logdet, M, 90)
    pats = g.all_patterns(M)
    lp = oracle.prob_exact(st, pats, dd=True)["logP"]
    n = np.array([bin(int(p[0])).count("1") for p in pats])
    pn = np.array([np.exp(lp[n == k]).sum() for k in range(M + 1)])
    assert np.allclose(pkn.sum(axis=0), pn, rtol=1e-9, atol=1e-13)


@pytest.mark.parametrize("eta", [1.0, 0.6])
def test_sectors_sum_to_photon_distribution(eta):
    M = 6
    U, r = g.haar_unitary(M, 12), g.squeezing(M, 4, 0.5, 1.0, 12)
    st = oracle.build_state(U, r, eta)
    K = 40
    pkn = ap.sector_distribution(st.O, st.logdet, M, K)
    assert np.allclose(pkn.sum(axis=1), photon_distribution(r, eta, K), rtol=1e-9, atol=1e-14)


def test_sector_support():
    """No more clicks than photons; a lossless state holds photon pairs only."""
    M = 6
    U, r = g.haar_unitary(M, 13), g.squeezing(M, 3, 0.8, 0.8, 13)
    st = oracle.build_state(U, r, 1.0)
    pkn = ap.sector_distribution(st.O, st.logdet, M, 30)
    k, n = np.meshgrid(np.arange(31), np.arange(M + 1), indexing="ij")
    assert np.abs(pkn[k < n]).max() < 1e-14
    assert np.abs(pkn[1::2]).max() < 1e-14
    assert abs(pkn[0, 0] - math.exp(-0.5 * st.logdet)) < 1e-15


@pytest.mark.parametrize("M,eta", [(4, 1.0), (5, 0.6)])
def test_curves_at_full_order_are_the_exact_sectors(M, eta):
    """With order >= the support size - 1 the fit reproduces the moments' distribution
    exactly, so the whole-device curves of S = all modes are the sectors p_k(c)."""
    U, r = g.haar_unitary(M, 14), g.squeezing(M, M // 2 + 1, 0.6, 0.9, 14)
    st = oracle.build_state(U, r, eta)
    K = 30
    got = ap.approx_sector_curves(st.O, st.logdet, M, range(M), 4, K)
    ref = ap.sector_distribution(st.O, st.logdet, M, K)
    assert np.abs(got - ref).max() < 1e-12


def test_curve_matches_the_sector_moments():
    """A fitted sector distribution reproduces its factorial moments D_0..D_j."""
    M, n, j = 10, 8, 3
    U, r = g.haar_unitary(M, 15), g.squeezing(M, 5, 0.8, 1.0, 15)
    st = oracle.build_state(U, r, 0.7)
    modes = list(range(n))
    D = ap.factorial_moment_tables(st.O, M, modes, j, 40)
    for k in (8, 12, 20):
        q, flag = ap.sector_curve(D[:, k], n, k, j)
        assert flag == 0
        v = np.arange(n + 1)
        for w in range(j + 1):
            fm = (q * np.array([math.comb(int(x), w) for x in v])).sum()
            assert abs(fm - D[w, k]) <= 1e-9 * D[w, k]
