"""Pins of the oracle's moment approximation (Methods, "Partition function",
"Moments calculation", "Approximation method")."""
import math
import numpy as np
import pytest

import fock
import gbs_inputs as g
import oracle
from oracle import approx as ap


def test_sector_series_matches_fock():
    # c_k[Z] det(sigma_Q)^{-1/2} = P(k photons in Z, vacuum on the other detectors):
    # the paper's sector decomposition, extended to loss, against the brute force.
    M = 2
    U = g.haar_unitary(M, 12)
    r = np.array([0.4, 0.35])
    for eta in (1.0, 0.7):
        st = oracle.build_state(U, r, eta)
        for Z in ([0], [1], [0, 1], []):
            pf, tail = fock.sector_probs(U, r, eta, 30, Z, 10)
            rows = ap.sub_rows(Z, M)
            c = ap.series_coeffs(st.O[np.ix_(rows, rows)], 10) * math.exp(-0.5 * st.logdet)
            assert np.abs(c - pf).max() <= tail + 1e-15


def test_lossless_odd_sectors_vanish():
    # Methods, "Model": squeezed light holds photon pairs, so odd sectors are empty.
    M = 5
    st = oracle.build_state(g.haar_unitary(M, 3), g.squeezing(M, 5, 0.5, 1.0, 3), 1.0)
    c = ap.series_coeffs(st.O, 30)
    assert np.abs(c[1::2]).max() < 1e-14 * c.max()


def _exact_vacuum_distribution(O, M, modes, K):
    """q_k(v): exact by inclusion-exclusion over every vacuum set V inside S."""
    n = len(modes)
    q = np.zeros((n + 1, K + 1))
    cache = {}

    def coeff(Z):
        key = tuple(Z)
        if key not in cache:
            rows = ap.sub_rows(Z, M)
            cache[key] = ap.series_coeffs(O[np.ix_(rows, rows)], K)
        return cache[key]

    for vmask in range(1 << n):
        C = [modes[a] for a in range(n) if not vmask >> a & 1]    # clicked set
        tot = np.zeros(K + 1)
        for z in range(1 << len(C)):
            Z = [C[b] for b in range(len(C)) if z >> b & 1]
            tot += (-1) ** (len(C) - len(Z)) * coeff(Z)
        q[bin(vmask).count("1")] += tot
    return q


@pytest.mark.parametrize("eta", [1.0, 0.5])
def test_minor_moments_equal_enumerated_moments(eta):
    # D_w^(k) from minors == sum_v C(v, w) q_k(v) with q_k(v) enumerated exactly.
    M = 9
    st = oracle.build_state(g.haar_unitary(M, 71), g.squeezing(M, 5, 0.6, 1.2, 71), eta)
    modes = [0, 2, 3, 5, 6, 8]
    K = 40
    D = ap.factorial_moment_tables(st.O, M, modes, 4, K)
    q = _exact_vacuum_distribution(st.O, M, modes, K)
    scale = D[0].max()
    for w in range(5):
        ref = sum(math.comb(v, w) * q[v] for v in range(len(modes) + 1))
        assert np.abs(D[w] - ref).max() <= 1e-12 * scale * math.comb(len(modes), w)
    # the all-clicked point summed over sectors is the exact probability
    T = oracle.subset_sum(st.A, M, modes)
    Kfull = ap.choose_kmax(st.O, M, modes)
    last = ap.exact_sector_last_points(st.O, M, modes, Kfull)
    assert abs(last.sum() - (T[0] + T[1])) <= 1e-12 * T[2]


def test_maxent_fit_recovers_exponential_family():
    x = np.arange(3, 12) / 12.0
    a_true = np.array([0.3, -2.0, 5.0, -1.5, 0.7])
    q = np.exp(-np.vander(x, 5, increasing=True) @ a_true)
    q /= q.sum()
    m = np.vander(x, 5, increasing=True).T @ q
    a, ok = ap.maxent_fit(x, m)
    assert ok
    qf = np.exp(-np.vander(x, 5, increasing=True) @ a)
    assert np.abs(qf - q).max() < 1e-11


@pytest.mark.parametrize("eta", [1.0, 0.6])
def test_order_at_least_support_is_exact(eta):
    # With n <= j + 1 every sector's support has at most j + 1 points, the
    # fitted family is the whole simplex and the approximation is exact.
    M = 6
    st = oracle.build_state(g.haar_unitary(M, 81), g.squeezing(M, 4, 0.6, 1.3, 81), eta)
    for modes in ([0], [1, 4], [0, 2, 5], [0, 1, 3, 5], [0, 1, 2, 3, 4]):
        ex = oracle.prob_exact(st, g.modes_to_pattern(modes)[None])["logP"][0]
        lp, info = ap.approx_logprob(st.O, st.logdet, M, modes, 4)
        assert info["flag"] == 0
        assert abs(lp - ex) < 1e-10


def test_tilted_contour_keeps_exactness_for_improbable_patterns():
    # weak squeezing, strong loss: all-clicked patterns are improbable and the
    # contour radius moves into the upper sector tail; with n <= j + 1 the
    # approximation must still be exact
    M = 10
    U = g.haar_unitary(M, 401)
    r = g.squeezing(M, 10, 0.2, 0.4, 401)
    for eta in (0.3, 0.9):
        st = oracle.build_state(U, r, eta)
        modes = [0, 1, 2, 3, 4]
        ex = oracle.prob_exact(st, g.modes_to_pattern(modes)[None], dd=True)["logP"][0]
        lp, info = ap.approx_logprob(st.O, st.logdet, M, modes, 4)
        assert info["rho"] > 1.0
        assert abs(lp - ex) < 1e-10


def test_order_two_is_a_discrete_gaussian():
    # Methods, "Approximation method": the second-order scheme is a Gaussian
    # c0 exp(-(v - c1)^2 / (2 c2^2)) matching moments 0, 1, 2.
    M = 8
    st = oracle.build_state(g.haar_unitary(M, 91), g.squeezing(M, 4, 0.8, 1.2, 91), 0.8)
    modes = [0, 1, 2, 4, 5, 7]
    n = len(modes)
    K = ap.choose_kmax(st.O, M, modes)
    D = ap.factorial_moment_tables(st.O, M, modes, 2, K)
    k = int(np.argmax(D[0])) + n
    mu = ap.raw_moments(D[:, k], 2)
    val, flag = ap.sector_last_point(D[:, k], n, k, 2)
    v = np.arange(max(0, n - k), n, dtype=float)
    # a Gaussian through those moments: the fitted log-weights are quadratic in v
    x = v / n
    m = np.array([mu[i] / n ** i for i in range(3)]) / mu[0]
    a, ok = ap.maxent_fit(x, m)
    q = np.exp(-np.vander(x, 3, increasing=True) @ a)
    assert ok and a[2] > 0                          # concave log-weights: a Gaussian bump
    assert abs(q @ v - mu[1] / mu[0]) < 1e-10 * n
    assert abs(val - mu[0] * math.exp(-a[0])) <= 1e-14 * mu[0]
