"""GPU gradient path against the oracle gradient and finite differences.

The adjoint is accumulated in double-double like the oracle's, so dL/dsigma_Q
agrees to ~1e-10 relative; the chains through the state build and the mesh are
plain FP64 products (1e-12 relative); finite differences (h = 1e-6) of the
double-double log P are good to ~1e-7."""
import math

import numpy as np
import pytest
import torch

import gbs_inputs as g
import oracle
from oracle import grad as og

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(cuda_ok):
    from paper_2106_01445_gb300 import build
    build.build()
    from paper_2106_01445_gb300.api import Context
    return Context(0)


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


def test_clements_forward_and_adjoint(ctx):
    M = 7
    th, ph = g.clements_phases(M, 5)
    Ud = ctx.clements_unitary(dev(th), dev(ph), M)
    U = Ud.cpu().numpy().view(np.complex128).reshape(M, M)
    assert np.abs(U - g.clements_unitary(M, th, ph)).max() < 1e-14
    rng = np.random.default_rng(1)
    dU = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
    dth, dph = ctx.clements_grad(dev(th), dev(ph), Ud, dev(dU.view(np.float64).reshape(M, 2 * M)))
    rth, rph = og.chain_clements(M, th, ph, dU)
    assert np.abs(dth.cpu().numpy() - rth).max() < 1e-12 * max(1, np.abs(rth).max())
    assert np.abs(dph.cpu().numpy() - rph).max() < 1e-12 * max(1, np.abs(rph).max())


def test_grad_params_chain(ctx):
    M = 6
    U = g.haar_unitary(M, 9)
    r = g.squeezing(M, 4, 0.5, 1.0, 9)
    eta = 0.55
    rng = np.random.default_rng(2)
    dsq = rng.standard_normal((2 * M, 2 * M))
    Ud = torch.view_as_real(dev(U)).reshape(M, 2 * M).contiguous()
    dU, dr, deta = ctx.grad_params(Ud, dev(r), eta, dev(dsq))
    rU, rr, re = og.chain_params(U, r, eta, dsq)
    got = dU.cpu().numpy().view(np.complex128).reshape(M, M)
    assert np.abs(got - rU).max() < 1e-12 * max(1, np.abs(rU).max())
    assert np.abs(dr.cpu().numpy() - rr).max() < 1e-12 * max(1, np.abs(rr).max())
    assert abs(deta.item() - re) < 1e-12 * max(1, abs(re))


@pytest.mark.parametrize("eta", [1.0, 0.6])
def test_dsigmaQ_matches_oracle(ctx, eta):
    # sizes below, at and above the 7-mode subtree of a unit: n > 7 runs 2^(n-7) units
    # with up to n - 7 eliminated prefix modes
    M = 14
    U = g.haar_unitary(M, 21)
    r = g.squeezing(M, 8, 0.5, 1.1, 21)
    rng = np.random.default_rng(4)
    mode_sets = [sorted(rng.choice(M, size=n, replace=False)) for n in (0, 1, 3, 5, 7, 8, 10, 12)]
    pats = np.stack([g.modes_to_pattern(m) for m in mode_sets])
    w = rng.standard_normal(len(pats))
    st = ctx.build_state(U, r, eta)
    dsq, logP, status = ctx.grad(st["O"], st["logdet"], pats, dev(w))
    torch.cuda.synchronize()
    ref = og.grad_sigmaQ(oracle.build_state(U, r, eta), pats, w)
    got = dsq.cpu().numpy()
    assert (status.cpu().numpy() == 0).all()
    assert np.abs(got - ref).max() < 1e-10 * np.abs(ref).max()
    ref_lp = oracle.prob_exact(oracle.build_state(U, r, eta), pats, dd=True)["logP"]
    assert np.abs(logP.cpu().numpy() - ref_lp).max() < 1e-12


def test_m32_workload_gradients(ctx):
    # the Clements workload: a slice of its patterns (kappa 1e14..1e19) through the
    # autograd function, against the oracle gradient and central differences
    from paper_2106_01445_gb300.api import LogProbClements
    c = g.CONFIGS["m32_grad"]
    th, ph = g.clements_phases(c.M, c.seed)
    r = c.squeezing()
    pats = c.patterns()
    n = np.array([len(g.pattern_modes(p)) for p in pats])
    sel = pats[np.nonzero(n <= 10)[0][:6]]
    w = np.linspace(0.5, 1.5, len(sel))
    rt = dev(r).requires_grad_(True)
    eta_t = torch.tensor(c.eta, dtype=torch.float64, device="cuda", requires_grad=True)
    tht, pht = dev(th).requires_grad_(True), dev(ph).requires_grad_(True)
    logp = LogProbClements.apply(rt, eta_t, tht, pht, sel, ctx)
    (logp * dev(w)).sum().backward()
    U = g.clements_unitary(c.M, th, ph)
    st = oracle.build_state(U, r, c.eta)
    rU, rr, re = og.chain_params(U, r, c.eta, og.grad_sigmaQ(st, sel, w))
    rth, rph = og.chain_clements(c.M, th, ph, rU)
    assert np.abs(rt.grad.cpu().numpy() - rr).max() < 1e-8 * max(1, np.abs(rr).max())
    assert abs(eta_t.grad.item() - re) < 1e-8 * max(1, abs(re))
    assert np.abs(tht.grad.cpu().numpy() - rth).max() < 1e-8 * max(1, np.abs(rth).max())
    assert np.abs(pht.grad.cpu().numpy() - rph).max() < 1e-8 * max(1, np.abs(rph).max())
    # central differences of the GPU's own double-double log P; their noise is
    # ~1e-14 |L| / h (the FP64 state build), i.e. ~5e-6 absolute here
    h = 1e-6
    def L(rv, ev, tv, pv):
        with torch.no_grad():
            return float((LogProbClements.apply(dev(rv), torch.tensor(ev, dtype=torch.float64, device="cuda"),
                                                dev(tv), dev(pv), sel, ctx) * dev(w)).sum())
    for j in (0, 7):
        e = np.zeros(c.M); e[j] = h
        fd = (L(r + e, c.eta, th, ph) - L(r - e, c.eta, th, ph)) / (2 * h)
        assert abs(fd - rt.grad[j].item()) < 1e-6 * abs(fd) + 5e-6
    fd = (L(r, c.eta + h, th, ph) - L(r, c.eta - h, th, ph)) / (2 * h)
    assert abs(fd - eta_t.grad.item()) < 1e-6 * abs(fd) + 5e-6
    for cc in (3, 200, 495):
        e = np.zeros(len(th)); e[cc] = h
        fd = (L(r, c.eta, th + e, ph) - L(r, c.eta, th - e, ph)) / (2 * h)
        assert abs(fd - tht.grad[cc].item()) < 1e-6 * abs(fd) + 5e-6, cc


def test_n20_gradient_against_central_differences(ctx):
    # a 20-click pattern of the 24-mode device (2^13 units of the tree adjoint): dL/dr
    # through the chain against central differences of the fixed-point log P
    c = g.CONFIGS["m24_exact"]
    U, r = c.unitary(), c.squeezing()
    modes = [m for m in range(24) if m not in (2, 9, 15, 22)]
    pats = g.modes_to_pattern(modes)[None]
    st = ctx.build_state(U, r, c.eta)
    dsq, logP, status = ctx.grad(st["O"], st["logdet"], pats, dev(np.ones(1)))
    assert status.item() == 0
    Ud = torch.view_as_real(dev(U)).reshape(c.M, 2 * c.M).contiguous()
    _, dr, deta = ctx.grad_params(Ud, dev(r), c.eta, dsq)
    lp_fx = ctx.prob(st["O"], st["logdet"], pats, precision="fx")["logP"].item()
    assert abs(logP.item() - lp_fx) < 1e-10

    def lp(rv, ev):
        s2 = ctx.build_state(U, rv, ev)
        return ctx.prob(s2["O"], s2["logdet"], pats, precision="fx")["logP"].item()

    h = 1e-6
    for j in (0, 5, 11):
        e = np.zeros(c.M); e[j] = h
        fd = (lp(r + e, c.eta) - lp(r - e, c.eta)) / (2 * h)
        assert abs(fd - dr[j].item()) < 1e-6 * abs(fd) + 1e-7, (j, fd, dr[j].item())
    fd = (lp(r, c.eta + h) - lp(r, c.eta - h)) / (2 * h)
    assert abs(fd - deta.item()) < 1e-6 * abs(fd) + 1e-7


def test_batch_chunks_match_single_pattern_calls(ctx):
    """A batch large enough for chunks of several units each (about eight chunks per SM
    over 96 patterns of 14 clicks, 128 units each) gives the sum of the one-pattern calls
    (each a chunk per unit): the chunking changes only the order of the double-double sums."""
    M = 20
    U, r = g.haar_unitary(M, 41), g.squeezing(M, 10, 0.6, 1.0, 41)
    st = ctx.build_state(U, r, 0.7)
    pats = g.gen_patterns(41, M, 14, 14, 96)
    w = torch.linspace(0.5, 1.5, len(pats), dtype=torch.float64, device="cuda")
    dsq, logP, status = ctx.grad(st["O"], st["logdet"], pats, w)
    assert (status.cpu().numpy() == 0).all()
    acc = torch.zeros_like(dsq)
    lps = []
    for i in range(len(pats)):
        d1, lp1, s1 = ctx.grad(st["O"], st["logdet"], pats[i:i + 1], w[i:i + 1])
        acc += d1
        lps.append(lp1.item())
    # the -1/2 (sum w) A term is linear in w: the single calls add up to the batch's
    got, ref = dsq.cpu().numpy(), acc.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()
    assert np.abs(logP.cpu().numpy() - np.array(lps)).max() < 1e-12


def test_grad_rejects_large_patterns(ctx):
    from paper_2106_01445_gb300 import GbsError
    M = 30
    st = ctx.build_state(g.haar_unitary(M, 3), g.squeezing(M, 5, 0.5, 1.0, 3), 0.7)
    pats = g.modes_to_pattern(list(range(25)))[None]
    with pytest.raises(GbsError):
        ctx.grad(st["O"], st["logdet"], pats, dev(np.ones(1)))
