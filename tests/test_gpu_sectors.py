"""Photon-number sectors of the whole device's click distribution (gbs_sector_distribution):
complex FP64 sweeps over all 2^M subsets at L points of a circle, binned by size, then the
DFT over the circle.  Checked against the oracle (all patterns, exact sector series), against
the click-number distribution of the double-double sweep (sum over k) and against the closed
form of the total photon-number distribution (sum over n)."""
import numpy as np
import pytest
import torch

import gbs_inputs as g
import oracle
from oracle import approx as ap

from test_oracle_sectors import photon_distribution

pytestmark = pytest.mark.gpu

# FP64 subset terms: absolute error ~ 1.1e-16 x the transform's cancellation (kappa <= 1e3 on
# these small devices) x the DFT's L terms (<= 256) ~ 3e-11; the bound below keeps a margin.
ATOL = 1e-10
# float-float subset terms: ~2^-46 per operation instead of 2^-53, the same argument
ATOL_FF = 3e-8


@pytest.fixture(scope="module")
def ctx(cuda_ok):
    from paper_2106_01445_gb300 import build
    build.build()
    from paper_2106_01445_gb300.api import Context
    return Context(0)


def gpu_pkn(ctx, U, r, eta, L, rho, K, even_only=False, precision="fp64"):
    st = ctx.build_state(U, r, eta)
    pkn = ctx.sector_distribution(st["O"], st["logdet"], L=L, rho=rho, K=K, even_only=even_only,
                                  precision=precision)
    torch.cuda.synchronize()
    return pkn.cpu().numpy(), st


@pytest.mark.parametrize("precision", ["fp64", "ff"])
@pytest.mark.parametrize("eta,rho", [(1.0, 1.0), (1.0, 0.9), (0.5, 1.0), (0.7, 0.8)])
def test_matches_oracle_over_all_patterns(ctx, eta, rho, precision):
    M, K = 8, 60
    U, r = g.haar_unitary(M, 21), g.squeezing(M, 4, 0.6, 1.0, 21)
    got, _ = gpu_pkn(ctx, U, r, eta, 128, rho, K, precision=precision)
    st = oracle.build_state(U, r, eta)
    ref = ap.sector_distribution(st.O, st.logdet, M, K)
    assert got.shape == (K + 1, M + 1)
    # the DFT divides sector k by rho^k: so does its error
    tol = (ATOL if precision == "fp64" else ATOL_FF) * rho ** -np.arange(K + 1.0)
    assert (np.abs(got - ref) < tol[:, None]).all()
    if eta == 1.0:
        even, _ = gpu_pkn(ctx, U, r, eta, 128, rho, K, even_only=True, precision=precision)
        assert (np.abs(even - ref) < tol[:, None]).all()


def test_sum_over_sectors_is_click_distribution(ctx):
    M = 20
    U, r = g.haar_unitary(M, 22), g.squeezing(M, 10, 0.5, 0.9, 22)
    got, st = gpu_pkn(ctx, U, r, 0.7, 256, 1.0, 255)
    logp, kappa = ctx.click_distribution(st["O"], st["logdet"])
    pn = np.exp(logp.cpu().numpy())
    big = pn > 1e-6
    assert np.allclose(got.sum(axis=0)[big], pn[big], rtol=1e-8)


@pytest.mark.parametrize("precision", ["fp64", "ff"])
@pytest.mark.parametrize("eta", [1.0, 0.5])
def test_sum_over_clicks_is_photon_distribution(ctx, eta, precision):
    M, K = 16, 80
    U, r = g.haar_unitary(M, 23), g.squeezing(M, 8, 0.6, 0.9, 23)
    got, _ = gpu_pkn(ctx, U, r, eta, 256, 1.0, K, precision=precision)
    tol = ATOL if precision == "fp64" else ATOL_FF
    assert np.abs(got.sum(axis=1) - photon_distribution(r, eta, K)).max() < tol
    if eta == 1.0:
        assert np.abs(got[1::2]).max() < tol


@pytest.mark.parametrize("L,rho,K,M", [(100, 1.0, 10, 8), (64, 1.5, 10, 8), (64, 1.0, 64, 8), (64, 1.0, 10, 3),
                                       (64, 1.0, 10, 37)])
def test_rejects_bad_arguments(ctx, L, rho, K, M):
    from paper_2106_01445_gb300._lib import GbsError
    U, r = g.haar_unitary(M, 1), g.squeezing(M, M // 2, 0.5, 0.5, 1)
    st = ctx.build_state(U, r, 1.0)
    with pytest.raises(GbsError):
        ctx.sector_distribution(st["O"], st["logdet"], L=L, rho=rho, K=K)


# ---- the approximation's fitted sector curves (gbs_approx_sector_curves) ---------------
@pytest.mark.parametrize("order,precision", [(2, "fp64"), (3, "fp64"), (4, "fp64"), (4, "ff")])
def test_curves_match_oracle(ctx, order, precision):
    """Whole-device curves (S = all 8 modes) against the oracle's fit, row by row: the fit's
    parameters agree to the 1e-8 of the last points (gbs_prob's tolerance), relative to the
    row's largest value."""
    M, K = 8, 255
    U, r = g.haar_unitary(M, 24), g.squeezing(M, 4, 0.7, 1.0, 24)
    st = ctx.build_state(U, r, 0.8)
    pat = g.modes_to_pattern(range(M))[None]
    curves, logP, status = ctx.approx_sector_curves(st["O"], st["logdet"], pat, order=order,
                                                    precision=precision, K=K)
    got = curves.cpu().numpy()
    so = oracle.build_state(U, r, 0.8)
    ref = ap.approx_sector_curves(so.O, so.logdet, M, range(M), order, K)
    # plus a floor for the rows one side leaves empty: sectors past the oracle's exact range
    # (the kernel's Chernoff bound reaches further; their mass is below 1e-14) and sectors
    # under the noise floor (1e-12 of the largest tilted sector)
    tol = (1e-8 if precision == "fp64" else 1e-6) * np.abs(ref).max(axis=1, keepdims=True) + 1e-11 * ref.max()
    assert (np.abs(got - ref) <= tol).all()
    # the all-clicked column summed over the sectors (every row of the pattern's sector
    # range: K covers it here) is the pattern's estimate
    assert abs(np.log(got[:, M].sum()) - logP.item()) < 1e-12


def test_curves_at_full_order_are_the_exact_sectors(ctx):
    M = 5
    U, r = g.haar_unitary(M, 25), g.squeezing(M, 3, 0.6, 0.9, 25)
    st = ctx.build_state(U, r, 0.6)
    pat = g.modes_to_pattern(range(M))[None]
    curves, _, _ = ctx.approx_sector_curves(st["O"], st["logdet"], pat, order=4, precision="fp64", K=60)
    exact = ctx.sector_distribution(st["O"], st["logdet"], L=128, rho=1.0, K=60)
    assert np.abs(curves.cpu().numpy() - exact.cpu().numpy()).max() < ATOL


def test_curves_reject_a_wrong_click_count(ctx):
    from paper_2106_01445_gb300._lib import GbsError, GBS_FP64
    from paper_2106_01445_gb300.api import _ptr, patterns_tensor
    M = 8
    U, r = g.haar_unitary(M, 26), g.squeezing(M, 4, 0.7, 0.7, 26)
    st = ctx.build_state(U, r, 1.0)
    pats = patterns_tensor(g.modes_to_pattern(range(M))[None], ctx.device)
    curves = torch.empty((11, 8), dtype=torch.float64, device=ctx.device)
    lp = torch.empty(1, dtype=torch.float64, device=ctx.device)
    stt = torch.empty(1, dtype=torch.int32, device=ctx.device)
    with pytest.raises(GbsError):
        ctx._check(ctx.lib.gbs_approx_sector_curves(ctx.h, M, _ptr(st["O"]), _ptr(st["logdet"]), _ptr(pats), 7, 4,
                                                    GBS_FP64, 10, _ptr(curves), _ptr(lp), _ptr(stt)))
