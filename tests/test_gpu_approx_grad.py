"""GPU gradient of the moment approximation (gbs_grad_approx) against the oracle's
(oracle/approx.py: approx_logprob_grad, which differentiates the exact sector series
through the minors' eigenvectors, where the GPU differentiates its discrete Fourier
transform and the minors' Schur complements), against the exact gradient at orders
where the fit interpolates, and through the autograd function and the mesh.  The
forward passes agree to ~1e-10 in log P; the gradients to ~1e-9 of their largest
entry."""
import numpy as np
import pytest
import torch

import gbs_inputs as g
import oracle
from oracle import grad as og
from paper_2106_01445_gb300._lib import GbsError

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(cuda_ok):
    from paper_2106_01445_gb300 import build
    build.build()
    from paper_2106_01445_gb300.api import Context
    return Context(0)


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


def _device(M=10, seed=31, eta=0.6):
    U = g.haar_unitary(M, seed)
    r = g.squeezing(M, M // 2, 0.6, 1.2, seed)
    return U, r, eta


@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_matches_oracle(ctx, order):
    U, r, eta = _device()
    M = U.shape[0]
    rng = np.random.default_rng(7)
    sets = [sorted(rng.choice(M, size=n, replace=False)) for n in (0, 1, 2, 3, 5, 6, 8, 9)]
    pats = np.stack([g.modes_to_pattern(m) for m in sets])
    w = rng.standard_normal(len(pats))
    st = ctx.build_state(U, r, eta)
    dsq, logP, status = ctx.grad_approx(st["O"], st["logdet"], pats, dev(w), order)
    torch.cuda.synchronize()
    ref, ref_lp = og.grad_sigmaQ_approx(oracle.build_state(U, r, eta), pats, w, order)
    assert (status.cpu().numpy() == 0).all()
    assert np.abs(logP.cpu().numpy() - ref_lp).max() < 1e-9
    got = dsq.cpu().numpy()
    assert np.abs(got - ref).max() < 1e-8 * np.abs(ref).max(), np.abs(got - ref).max()
    # the forward is gbs_prob's FP64 approximation
    lp = ctx.prob(st["O"], st["logdet"], pats, order=order, precision="fp64")["logP"]
    assert torch.equal(lp, logP)


def test_interpolating_orders_equal_the_exact_gradient(ctx):
    # order >= n - 1: the fit interpolates every sector; approximation = exact P
    U, r, eta = _device(M=9, seed=5, eta=0.75)
    M = U.shape[0]
    rng = np.random.default_rng(3)
    sets = [sorted(rng.choice(M, size=n, replace=False)) for n in (1, 2, 3, 4, 5, 5)]
    pats = np.stack([g.modes_to_pattern(m) for m in sets])
    w = rng.standard_normal(len(pats))
    st = ctx.build_state(U, r, eta)
    dsq, logP, status = ctx.grad_approx(st["O"], st["logdet"], pats, dev(w), 4)
    ref = og.grad_sigmaQ(oracle.build_state(U, r, eta), pats, w)
    ref_lp = oracle.prob_exact(oracle.build_state(U, r, eta), pats, dd=True)["logP"]
    assert (status.cpu().numpy() == 0).all()
    assert np.abs(logP.cpu().numpy() - ref_lp).max() < 1e-9
    assert np.abs(dsq.cpu().numpy() - ref).max() < 1e-8 * np.abs(ref).max()


def test_contour_chunks_do_not_change_the_result(ctx):
    # one pattern alone runs its contour points on many CTAs; inside a batch of 320 on one
    # each: the same gradient up to the order of the sums over the chunks
    U, r, eta = _device(M=12, seed=8, eta=0.5)
    M = U.shape[0]
    st = ctx.build_state(U, r, eta)
    pats = g.gen_patterns(41, M, 3, 7, 320)
    one = pats[17:18]
    dsq1, lp1, st1 = ctx.grad_approx(st["O"], st["logdet"], one, dev(np.ones(1)), 3)
    w = np.zeros(len(pats))
    w[17] = 1.0
    dsqb, lpb, stb = ctx.grad_approx(st["O"], st["logdet"], pats, dev(w), 3)
    assert st1.item() == 0 and stb[17].item() == 0
    assert lp1.item() == lpb[17].item()
    a, b = dsq1.cpu().numpy(), dsqb.cpu().numpy()
    assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()


def test_autograd_through_the_mesh(ctx):
    from paper_2106_01445_gb300.api import LogProbClementsApprox
    M = 8
    th, ph = g.clements_phases(M, 13)
    r = g.squeezing(M, 4, 0.6, 1.1, 13)
    eta = 0.65
    pats = np.stack([g.modes_to_pattern(m) for m in ([0, 2, 3, 6], [1, 2, 4, 5, 7], [0, 1, 3, 4, 5, 6])])
    w = np.array([0.7, -1.1, 1.4])
    rt = dev(r).requires_grad_(True)
    eta_t = torch.tensor(eta, dtype=torch.float64, device="cuda", requires_grad=True)
    tht, pht = dev(th).requires_grad_(True), dev(ph).requires_grad_(True)
    logp = LogProbClementsApprox.apply(rt, eta_t, tht, pht, pats, ctx, 2)
    (logp * dev(w)).sum().backward()
    U = g.clements_unitary(M, th, ph)
    dsq, _ = og.grad_sigmaQ_approx(oracle.build_state(U, r, eta), pats, w, 2)
    rU, rr, re = og.chain_params(U, r, eta, dsq)
    rth, rph = og.chain_clements(M, th, ph, rU)
    assert np.abs(rt.grad.cpu().numpy() - rr).max() < 1e-8 * max(1, np.abs(rr).max())
    assert abs(eta_t.grad.item() - re) < 1e-8 * max(1, abs(re))
    assert np.abs(tht.grad.cpu().numpy() - rth).max() < 1e-8 * max(1, np.abs(rth).max())
    assert np.abs(pht.grad.cpu().numpy() - rph).max() < 1e-8 * max(1, np.abs(rph).max())


def test_bad_arguments(ctx):
    U, r, eta = _device()
    st = ctx.build_state(U, r, eta)
    pats = np.stack([g.modes_to_pattern([0, 1, 2])])
    for order in (0, 5):
        with pytest.raises(GbsError) as e:
            ctx.grad_approx(st["O"], st["logdet"], pats, dev(np.ones(1)), order)
        assert e.value.code == 1
    with pytest.raises(GbsError) as e:          # detector >= M
        ctx.grad_approx(st["O"], st["logdet"], np.stack([g.modes_to_pattern([0, 11])]), dev(np.ones(1)), 2)
    assert e.value.code == 1
    # more than 48 clicks
    M = 50
    U2 = g.haar_unitary(M, 2)
    st2 = ctx.build_state(U2, g.squeezing(M, 10, 0.5, 0.8, 2), 0.5)
    with pytest.raises(GbsError) as e:
        ctx.grad_approx(st2["O"], st2["logdet"], np.stack([g.modes_to_pattern(range(49))]), dev(np.ones(1)), 2)
    assert e.value.code == 1
