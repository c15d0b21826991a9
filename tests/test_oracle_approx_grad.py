"""Pins of the oracle gradient of the moment approximation (oracle/approx.py:
approx_logprob_grad, oracle/grad.py: grad_sigmaQ_approx):

* central differences in sigma_Q of the oracle's own order-j log P (the contour
  radius and the sector range held fixed, so that log P is a smooth function),
  at orders below the support size, where the fit is a genuine least-information
  extrapolation and its implicit derivative matters;
* orders j >= n - 1: the fit interpolates every sector exactly, the approximation
  is the exact probability (Methods, "Approximation method"), so its gradient is
  the exact gradient of the double-double subset-sum oracle, a separate code path
  (trace formula per subset in C)."""
import numpy as np
import pytest

import gbs_inputs as g
import oracle
from oracle import approx as oa
from oracle import grad as og


def _state(M, K, seed, eta):
    U = g.haar_unitary(M, seed)
    r = g.squeezing(M, K, 0.6, 1.1, seed)
    return oracle.build_state(U, r, eta)


@pytest.mark.parametrize("order", [2, 3])
def test_central_differences(order):
    M = 7
    st = _state(M, 4, 11, 0.6)
    modes = [0, 2, 3, 5, 6]
    pat = g.modes_to_pattern(modes)[None, :]
    _, info = oa.approx_logprob(st.O, st.logdet, M, modes, order)
    rho, K = info["rho"], info["K"]
    dsq, lp = og.grad_sigmaQ_approx(st, pat, [1.0], order)
    assert abs(lp[0] - oa.approx_logprob(st.O, st.logdet, M, modes, order)[0]) < 1e-14

    def L(sq):
        A = np.linalg.inv(sq)
        return oa.approx_logprob(np.eye(2 * M) - A, np.linalg.slogdet(sq)[1], M, modes, order,
                                 K=K, rho=rho)[0]

    h = 1e-5
    for i, k in [(0, 0), (0, 2), (2, 9), (5, 12), (3, 3), (10, 13), (1, 4), (7, 7)]:
        E = np.zeros((2 * M, 2 * M))
        E[i, k] += h
        if i != k:
            E[k, i] += h
        fd = (L(st.sigmaQ + E) - L(st.sigmaQ - E)) / (2 * h)
        an = dsq[i, k] + (dsq[k, i] if i != k else 0.0)
        # difference error ~h^2 plus the fits' convergence (1e-13) over h
        assert abs(fd - an) < 2e-8, (i, k, fd, an)


def test_exact_orders_match_exact_gradient():
    M = 8
    st = _state(M, 5, 3, 0.7)
    pats = np.stack([g.modes_to_pattern(m) for m in ([0, 1, 2], [1, 3, 4, 6], [0, 2, 5, 6, 7], [4])])
    w = np.array([1.0, -0.6, 0.8, 1.3])
    dA, lpa = og.grad_sigmaQ_approx(st, pats, w, 4)
    dE = og.grad_sigmaQ(st, pats, w)
    lpe = oracle.prob_exact(st, pats, dd=True)["logP"]
    assert np.max(np.abs(lpa - lpe)) < 1e-11
    assert np.max(np.abs(dA - dE)) < 1e-10 * np.max(np.abs(dE))


def test_empty_pattern_has_only_the_normalisation_term():
    M = 4
    st = _state(M, 2, 5, 0.8)
    pats = np.zeros((1, 2), dtype=np.uint64)
    dA, lp = og.grad_sigmaQ_approx(st, pats, [2.0], 3)
    assert abs(lp[0] + 0.5 * st.logdet) < 1e-14
    assert np.max(np.abs(dA + st.A)) < 1e-14       # -1/2 * 2 * A


def test_fit_adjoint_against_differences():
    # d part / d D_w of one fitted sector (order 3 on 6 support points) against central
    # differences of the fit itself
    M = 8
    st = _state(M, 4, 2, 0.7)
    modes = [0, 1, 3, 4, 6, 7]
    n, j = len(modes), 3
    rho = oa.choose_tilt(st.O, M, modes)
    K = oa.choose_kmax(st.O, M, modes, rho)
    D = oa.factorial_moment_tables(st.O, M, modes, j, K, rho)
    k = int(np.argmax(D[0, n:])) + n                     # the heaviest sector that is fitted
    val, flag, a, J = oa.sector_fit(D[:, k], n, k, j)
    assert flag == 0 and J == j
    beta = oa.fit_last_point_adjoint(n, a, J, j)
    for w in range(j + 1):
        h = 1e-6 * D[w, k]
        Dp, Dm = D[:, k].copy(), D[:, k].copy()
        Dp[w] += h
        Dm[w] -= h
        fd = (oa.sector_fit(Dp, n, k, j)[0] - oa.sector_fit(Dm, n, k, j)[0]) / (2 * h)
        assert abs(fd - beta[w]) < 1e-6 * max(abs(beta).max(), 1e-300), (w, fd, beta[w])


def test_series_adjoint_against_differences():
    # sum_k gam_k d c_k[X] / dX for a symmetric X against central differences
    rng = np.random.default_rng(5)
    B = rng.standard_normal((6, 6))
    X = 0.3 * (B + B.T) / np.abs(np.linalg.eigvalsh(B + B.T)).max()
    gam = rng.standard_normal(12)
    dX = oa.series_coeffs_adjoint(X, gam)
    h = 1e-6
    for i, k in [(0, 0), (1, 4), (5, 2), (3, 3)]:
        E = np.zeros_like(X)
        E[i, k] += h
        if i != k:
            E[k, i] += h
        fd = (gam @ oa.series_coeffs(X + E, 11) - gam @ oa.series_coeffs(X - E, 11)) / (2 * h)
        an = dX[i, k] + (dX[k, i] if i != k else 0.0)
        assert abs(fd - an) < 1e-8, (i, k, fd, an)
