"""Pins of the FP64 oracle's exact path against things other than itself:
closed forms, the Fock-space brute force, two independent determinant
formulas, invariants (sum over all patterns, mean click number) and the
exactly solvable two-mode squeezed vacuum."""
import math
from itertools import combinations

import numpy as np
import pytest

import fock
import gbs_inputs as g
import oracle


def probs_all(U, r, eta):
    st = oracle.build_state(U, r, eta)
    res = oracle.prob_exact(st, g.all_patterns(U.shape[0]))
    assert (res["status"] == 0).all()
    return np.exp(res["logP"]), st


def p_vac_closed(r, eta):
    """P(no click) of one lossy squeezed mode: (1 + eta(2 - eta) sinh^2 r)^{-1/2}."""
    return (1.0 + eta * (2.0 - eta) * np.sinh(r) ** 2) ** -0.5


def test_single_mode_vacuum_closed_form():
    # Methods, "Model": <x|x> = (1 - tanh^2 r)^{-1/2} = cosh r, so P(no click) = 1/cosh r.
    for r in (0.1, 0.8, 1.6):
        p, _ = probs_all(np.eye(1, dtype=complex), np.array([r]), 1.0)
        assert abs(p[0] - 1.0 / math.cosh(r)) < 1e-15
        assert abs(p[1] - (1.0 - 1.0 / math.cosh(r))) < 1e-14
        for eta in (0.3, 0.6):
            p, _ = probs_all(np.eye(1, dtype=complex), np.array([r]), eta)
            assert abs(p[0] - p_vac_closed(r, eta)) < 1e-15


def test_no_click_any_interferometer():
    # Uniform loss commutes with U and the vacuum is U-invariant.
    M = 7
    r = g.squeezing(M, 5, 0.4, 1.3, seed=21)
    for eta in (1.0, 0.45):
        st = oracle.build_state(g.haar_unitary(M, 22), r, eta)
        lp = oracle.prob_exact(st, np.zeros((1, 2), dtype=np.uint64))["logP"][0]
        assert abs(math.exp(lp) - np.prod(p_vac_closed(r, eta))) < 1e-14


def test_identity_interferometer_factorises():
    M = 6
    r = g.squeezing(M, 6, 0.3, 1.5, seed=31)
    for eta in (1.0, 0.6):
        p, _ = probs_all(np.eye(M, dtype=complex), r, eta)
        p0 = p_vac_closed(r, eta)
        for mask in range(1 << M):
            ref = np.prod([(1 - p0[i]) if mask >> i & 1 else p0[i] for i in range(M)])
            assert abs(p[mask] - ref) <= 1e-14 + 1e-12 * ref


@pytest.mark.parametrize("eta", [1.0, 0.5])
def test_sum_over_all_patterns_is_one(eta):
    c = g.CONFIGS["m8_all"]
    p, _ = probs_all(c.unitary(), c.squeezing(), eta)
    assert abs(p.sum() - 1.0) < 1e-13
    assert (p > 0).all()


def test_two_mode_squeezed_vacuum():
    # U = [[1, i], [i, 1]]/sqrt2 on equal squeezing gives B = U tanh(r) U^T with
    # zero diagonal: photons come in pairs across the two modes.
    U = np.array([[1, 1j], [1j, 1]]) / math.sqrt(2)
    for r in (0.5, 1.2):
        st = oracle.build_state(U, np.array([r, r]), 1.0)
        res = oracle.prob_exact(st, g.all_patterns(2))
        # P(10), P(01) are zero: T is rounding noise there and log P undefined (status 4)
        p = math.exp(-0.5 * st.logdet) * res["T"].sum(axis=1)
        assert abs(p[0] - 1 / math.cosh(r) ** 2) < 1e-15
        assert abs(p[1]) < 1e-14 and abs(p[2]) < 1e-14
        assert abs(p[3] - math.tanh(r) ** 2) < 1e-14


@pytest.mark.parametrize("case", [
    dict(M=3, seed=11, r=[0.45, 0.40, 0.50], eta=1.0, N=34),
    dict(M=4, seed=13, r=[0.30, 0.25, 0.35, 0.0], eta=1.0, N=26),
    dict(M=2, seed=12, r=[0.35, 0.30], eta=0.6, N=28),
    dict(M=1, seed=0, r=[0.9], eta=0.3, N=80),
])
def test_fock_brute_force(case):
    M = case["M"]
    U = g.haar_unitary(M, case["seed"]) if M > 1 else np.eye(1, dtype=complex)
    r = np.array(case["r"])
    pf, tail = fock.click_probs(U, r, case["eta"], case["N"])
    assert 0 <= tail < 1e-11
    p, _ = probs_all(U, r, case["eta"])
    assert np.abs(p - pf).max() <= tail + 1e-13


def test_fock_detects_transposed_interferometer():
    # A plausible convention slip (U^T instead of U) must fail the brute-force pin.
    M = 3
    U = g.haar_unitary(M, 11)
    r = np.array([0.45, 0.40, 0.50])
    pf, tail = fock.click_probs(U, r, 1.0, 34)
    p_wrong, _ = probs_all(U.T, r, 1.0)
    assert np.abs(p_wrong - pf).max() > 1e3 * (tail + 1e-13)


def _marginal_form(sigmaQ, M, modes):
    """sum_{Z subset S} (-1)^{|S|-|Z|} P(vacuum outside Z), P(vac on W) = det(sigma_Q,WW)^{-1/2}."""
    n = len(modes)
    tot = 0.0
    for z in range(1 << n):
        Z = {modes[a] for a in range(n) if z >> a & 1}
        W = [i for i in range(M) if i not in Z]
        rows = W + [i + M for i in W]
        d = np.linalg.det(sigmaQ[np.ix_(rows, rows)]) if rows else 1.0
        tot += (-1) ** (n - len(Z)) * d ** -0.5
    return tot


def _b_form(U, r, modes):
    """Methods, Eq. for Z_X and Eq. (p(n)), lossless: B = U diag(tanh r) U^T,
    P(vac outside Z) = det(I - B_Z^dag B_Z)^{-1/2} / prod cosh r."""
    B = U @ np.diag(np.tanh(r)) @ U.T
    n = len(modes)
    tot = 0.0
    for z in range(1 << n):
        Z = [modes[a] for a in range(n) if z >> a & 1]
        Bz = B[np.ix_(Z, Z)]
        d = np.linalg.det(np.eye(len(Z)) - Bz.conj().T @ Bz).real if Z else 1.0
        tot += (-1) ** (n - len(Z)) * d ** -0.5
    return tot / np.prod(np.cosh(r))


def test_three_formulas_agree():
    M = 6
    U = g.haar_unitary(M, 41)
    r = g.squeezing(M, 4, 0.5, 1.2, seed=41)
    rng_pats = [[0, 2, 3], [1, 2, 4, 5], [0, 1, 2, 3, 4, 5], [5], []]
    for eta in (1.0, 0.7):
        st = oracle.build_state(U, r, eta)
        for modes in rng_pats:
            lp = oracle.prob_exact(st, g.modes_to_pattern(modes)[None])["logP"][0]
            p = math.exp(lp)
            assert abs(p - _marginal_form(st.sigmaQ, M, modes)) < 1e-13
            if eta == 1.0:
                assert abs(p - _b_form(U, r, modes)) < 1e-13


def test_mean_click_number():
    # Methods, "Moments calculation": n_bar = sum_l (1 - Z_{X_l}/Z_X) where
    # Z_{X_l}/Z_X is the probability that detector l stays dark.
    c = g.CONFIGS["m8_all"]
    for eta in (1.0, 0.55):
        p, st = probs_all(c.unitary(), c.squeezing(), eta)
        M = c.M
        nbar = sum(bin(m).count("1") * p[m] for m in range(1 << M))
        dark = [np.linalg.det(st.sigmaQ[np.ix_([l, l + M], [l, l + M])]) ** -0.5 for l in range(M)]
        assert abs(nbar - sum(1 - d for d in dark)) < 1e-12


def test_permutation_equivariance():
    M = 6
    U = g.haar_unitary(M, 51)
    r = g.squeezing(M, 6, 0.5, 1.0, seed=51)
    perm = np.array([3, 0, 5, 1, 4, 2])     # output i of the permuted device is output perm[i]
    p, _ = probs_all(U, r, 0.8)
    pp, _ = probs_all(U[perm], r, 0.8)
    for mask in range(1 << M):
        src = sum(1 << int(perm[i]) for i in range(M) if mask >> i & 1)
        assert abs(pp[mask] - p[src]) < 1e-14


def test_state_build_consistency():
    M = 5
    U = g.haar_unitary(M, 61)
    r = g.squeezing(M, 3, 0.5, 1.0, seed=61)
    st = oracle.build_state(U, r, 0.7)
    N = 2 * M
    assert np.allclose(st.sigmaQ, st.sigma + 0.5 * np.eye(N), atol=0)
    assert np.abs(st.A @ st.sigmaQ - np.eye(N)).max() < 1e-13
    assert np.abs(st.O - (np.eye(N) - st.A)).max() == 0
    assert abs(st.logdet - np.linalg.slogdet(st.sigmaQ)[1]) < 1e-13
    # the spectral radius of O is below one (used by the sector series)
    assert np.abs(np.linalg.eigvalsh(st.O)).max() < 1.0


def test_subset_sum_chunks_match():
    c = g.CONFIGS["m24_exact"]
    st = oracle.build_state(c.unitary(), c.squeezing(), c.eta)
    modes = g.pattern_modes(c.patterns()[0])[:14]
    whole = oracle.subset_sum(st.A, c.M, modes)
    parts = oracle.subset_sum(st.A, c.M, modes, nchunk=7, nthreads=2)
    assert abs((whole[0] + whole[1]) - (parts[0] + parts[1])) <= 1e-15 * whole[2]


def test_double_double_against_multiprecision():
    # Improbable patterns cancel by many orders of magnitude (kappa >> 1/u);
    # the double-double oracle is pinned by a 50-digit evaluation of the
    # independent marginal formula sum_Z +- det(sigma_Q,Z^c Z^c)^{-1/2}.
    mpmath = pytest.importorskip("mpmath")
    M = 10
    U = g.haar_unitary(M, 123)
    r = g.squeezing(M, 10, 0.3, 0.6, 123)
    st = oracle.build_state(U, r, 0.3)
    mpmath.mp.dps = 50
    worst64 = 0.0
    for modes in ([0, 1, 2, 3, 4, 5, 6, 7, 8, 9], [0, 2, 3, 4, 6, 7, 8, 9], [1, 3, 5, 7, 9]):
        pat = g.modes_to_pattern(modes)[None]
        n = len(modes)
        tot = mpmath.mpf(0)
        for z in range(1 << n):
            Z = {modes[i] for i in range(n) if z >> i & 1}
            W = [i for i in range(M) if i not in Z]
            rows = W + [i + M for i in W]
            d = mpmath.det(mpmath.matrix(st.sigmaQ[np.ix_(rows, rows)].tolist())) if rows else 1
            tot += (-1) ** (n - len(Z)) / mpmath.sqrt(d)
        ref = float(mpmath.log(tot))
        dd = oracle.prob_exact(st, pat, dd=True)
        f64 = oracle.prob_exact(st, pat)
        assert abs(dd["logP"][0] - ref) < 1e-13, (modes, dd["kappa"][0])
        worst64 = max(worst64, abs(f64["logP"][0] - ref) / (f64["kappa"][0] * 1.1e-16))
    # the FP64 oracle's error stays within its kappa-scaled bound
    assert worst64 < 4 * 24
