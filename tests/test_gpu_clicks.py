"""The whole device's click-number distribution p(n) (gbs_click_distribution): one
double-double sweep over all 2^M subsets binned by size, then the binomial transform.
Pinned by the oracle summed over all patterns, by Sigma_n p(n) = 1, and by the
closed form of independent modes (identity interferometer)."""
import numpy as np
import pytest
import torch

import gbs_inputs as g
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(cuda_ok):
    from paper_2106_01445_gb300 import build
    build.build()
    from paper_2106_01445_gb300.api import Context
    return Context(0)


def gpu_pn(ctx, U, r, eta):
    st = ctx.build_state(U, r, eta)
    logp, kappa = ctx.click_distribution(st["O"], st["logdet"])
    torch.cuda.synchronize()
    return logp.cpu().numpy(), kappa.cpu().numpy()


def oracle_pn(U, r, eta):
    M = U.shape[0]
    pats = g.all_patterns(M)
    lp = oracle.prob_exact(oracle.build_state(U, r, eta), pats, dd=True)["logP"]
    n = np.array([bin(int(p[0])).count("1") for p in pats])
    return np.log(np.array([np.exp(lp[n == k]).sum() for k in range(M + 1)]))


@pytest.mark.parametrize("M,eta,seed", [(8, 1.0, 0), (8, 0.5, 0), (12, 0.6, 31)])
def test_matches_oracle_over_all_patterns(ctx, M, eta, seed):
    U = g.haar_unitary(M, seed)
    r = g.squeezing(M, M if M == 8 else 7, 0.8 if M == 8 else 0.5, 0.8 if M == 8 else 1.2, seed)
    got, kappa = gpu_pn(ctx, U, r, eta)
    ref = oracle_pn(U, r, eta)
    assert np.abs(got - ref).max() < 1e-10, (got - ref)
    assert np.isfinite(kappa).all()


def test_sums_to_one_on_the_24_mode_device(ctx):
    c = g.CONFIGS["m24_exact"]
    got, _ = gpu_pn(ctx, c.unitary(), c.squeezing(), c.eta)
    assert np.isfinite(got).all()
    assert abs(np.exp(got).sum() - 1.0) < 1e-12


def test_independent_modes_closed_form(ctx):
    # identity interferometer: modes are independent, p(n) = e_n(q_1..q_M) with the
    # single-mode click probability q = 1 - (1 + eta (2 - eta) sinh^2 r)^{-1/2}
    M, eta = 20, 0.7
    r = g.squeezing(M, 14, 0.3, 1.3, 5)
    q = 1.0 - (1.0 + eta * (2.0 - eta) * np.sinh(r) ** 2) ** -0.5
    e = np.zeros(M + 1)
    e[0] = 1.0
    for qi in q:
        e[1:] = e[1:] * (1.0 - qi) + e[:-1] * qi
        e[0] *= 1.0 - qi
    got, _ = gpu_pn(ctx, np.eye(M, dtype=complex), r, eta)
    ok = e > 1e-250
    assert np.abs(got[ok] - np.log(e[ok])).max() < 1e-10


def test_strong_squeezing_falls_back_to_double_double(ctx):
    """Squeezing beyond the fixed-point range (r = 4: pivot determinants below 2^-8) is
    flagged by the fixed-point pass and the distribution is taken in double-double; the
    closed form of independent modes checks it."""
    M, eta = 8, 1.0
    r = np.array([4.0, 3.5, 0.5, 0.6, 0.7, 0.8, 0.0, 0.0])
    q = 1.0 - (1.0 + eta * (2.0 - eta) * np.sinh(r) ** 2) ** -0.5
    e = np.zeros(M + 1)
    e[0] = 1.0
    for qi in q:
        e[1:] = e[1:] * (1.0 - qi) + e[:-1] * qi
        e[0] *= 1.0 - qi
    got, _ = gpu_pn(ctx, np.eye(M, dtype=complex), r, eta)
    ok = e > 1e-250
    assert np.abs(got[ok] - np.log(e[ok])).max() < 1e-10


@pytest.mark.parametrize("M", [3, 37])
def test_rejects_devices_out_of_range(ctx, M):
    from paper_2106_01445_gb300 import GbsError
    st = ctx.build_state(g.haar_unitary(M, 1), g.squeezing(M, 2, 0.5, 0.8, 1), 0.9)
    with pytest.raises(GbsError):
        ctx.click_distribution(st["O"], st["logdet"])
