"""GPU parity of the 192-bit fixed-point exact sweep (GBS_FX192) where the signed sum cancels
beyond what 128-bit fixed point and double-double resolve (kappa 1e22 .. 1e31), against the
60-digit marginal form of the oracle stored by tests/golden/make_fx192_cases.py; and against
the double-double oracle on ordinary patterns.  Bound: 1e-10 in log P, with the returned
a-posteriori bound below 1e-10 as well (the 128-bit sweep's own bound exceeds it on these)."""
import json
import os

import numpy as np
import pytest
import torch

import gbs_inputs as g
import oracle

pytestmark = pytest.mark.gpu

with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fx192_cases.json")) as f:
    CASES = json.load(f)


@pytest.fixture(scope="module")
def ctx(cuda_ok):
    from paper_2106_01445_gb300 import build
    build.build()
    from paper_2106_01445_gb300.api import Context
    return Context(0)


def gpu(ctx, U, r, eta, pats, precision):
    st = ctx.build_state(U, r, eta)
    out = ctx.prob(st["O"], st["logdet"], pats, precision=precision)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def test_single_devices_against_multiprecision(ctx):
    for e in CASES["single"]:
        U, r = g.haar_unitary(e["M"], e["seed"]), g.squeezing(e["M"], e["K"], e["r"][0], e["r"][1], e["seed"])
        pat = g.modes_to_pattern(e["modes"])[None]
        res = gpu(ctx, U, r, e["eta"], pat, "fx192")
        assert res["status"][0] == 0, (e["name"], e["modes"], res["status"][0])
        assert abs(res["logP"][0] - e["logP"]) < 1e-10, (e["name"], len(e["modes"]), res["logP"][0] - e["logP"])
        assert res["err_bound"][0] < 1e-10
        assert abs(res["kappa"][0] / e["kappa"] - 1.0) < 1e-3   # sum |terms| kept in FP32
        # the 128-bit sweep holds to its own (larger) bound
        fx = gpu(ctx, U, r, e["eta"], pat, "fx")
        if fx["status"][0] == 0:
            assert abs(fx["logP"][0] - e["logP"]) <= max(1e-10, fx["err_bound"][0])


def test_block_diagonal_30_clicks_kappa_4e28(ctx):
    """Three 10-mode blocks: the 30-click pattern (2^30 subsets, kappa ~4e28, the size and
    cancellation of the 100-mode workload's anchors) against the product of the blocks'
    60-digit probabilities."""
    B = CASES["block"]
    m, k = B["M"], len(B["seeds"])
    U = np.zeros((m * k, m * k), dtype=complex)
    r = np.zeros(m * k)
    for b, s in enumerate(B["seeds"]):
        U[b * m:(b + 1) * m, b * m:(b + 1) * m] = g.haar_unitary(m, s)
        r[b * m:(b + 1) * m] = g.squeezing(m, m, B["r"][0], B["r"][1], s)
    pat = g.modes_to_pattern(list(range(m * k)))[None]
    res = gpu(ctx, U, r, B["eta"], pat, "fx192")
    assert res["status"][0] == 0
    assert abs(res["logP"][0] - B["logP"]) < 1e-10, res["logP"][0] - B["logP"]
    assert res["err_bound"][0] < 1e-10
    assert abs(res["kappa"][0] / B["kappa"] - 1.0) < 1e-3
    fx = gpu(ctx, U, r, B["eta"], pat, "fx")
    assert fx["err_bound"][0] > 1e-10           # beyond the 128-bit sweep
    assert abs(fx["logP"][0] - B["logP"]) <= fx["err_bound"][0]


def test_ordinary_patterns_against_double_double_oracle(ctx):
    c = g.CONFIGS["m8_all"]
    U, r = c.unitary(), c.squeezing()
    pats = c.patterns()
    res = gpu(ctx, U, r, 0.7, pats, "fx192")
    ref = oracle.prob_exact(oracle.build_state(U, r, 0.7), pats, dd=True)
    assert (res["status"] == 0).all()
    assert np.abs(res["logP"] - ref["logP"]).max() < 1e-10
    assert abs(np.exp(res["logP"]).sum() - 1.0) < 1e-12
    c = g.CONFIGS["m24_exact"]
    U, r = c.unitary(), c.squeezing()
    allp = c.patterns()
    n = np.array([len(g.pattern_modes(p)) for p in allp])
    sel = np.argsort(n, kind="stable")[:6]
    res = gpu(ctx, U, r, c.eta, allp[sel], "fx192")
    ref = oracle.prob_exact(oracle.build_state(U, r, c.eta), allp[sel], dd=True)
    assert (res["status"] == 0).all()
    assert np.abs(res["logP"] - ref["logP"]).max() < 1e-10


def test_range_status_and_anchor_bounds(ctx):
    # out of the fixed-point range: two modes squeezed so strongly (r = 4, identity U) that
    # their pivot determinants fall below 2^-8 report GBS_E_RANGE, the others stay exact
    M = 6
    r = np.array([4.0, 4.0, 0.5, 0.6, 0.7, 0.8])
    mode_sets = [[2, 3], [0], [1, 2], [2, 3, 4, 5]]
    pats = np.stack([g.modes_to_pattern(m) for m in mode_sets])
    res = gpu(ctx, np.eye(M, dtype=complex), r, 1.0, pats, "fx192")
    ref = oracle.prob_exact(oracle.build_state(np.eye(M, dtype=complex), r, 1.0), pats, dd=True)
    assert list(res["status"]) == [0, 8, 8, 0]
    assert np.abs(res["logP"][[0, 3]] - ref["logP"][[0, 3]]).max() < 1e-10
    # two 30-click anchors of the 100-mode workload: resolved to 1e-10, and within the
    # 128-bit sweep's own bound of it
    c = g.CONFIGS["m100_approx"]
    U, r = c.unitary(), c.squeezing()
    anc = c.anchor_patterns()[:2]
    res = gpu(ctx, U, r, c.eta, anc, "fx192")
    fx = gpu(ctx, U, r, c.eta, anc, "fx")
    assert (res["status"] == 0).all()
    assert (res["err_bound"] < 1e-10).all(), res["err_bound"]
    ok = fx["status"] == 0
    assert (np.abs(res["logP"][ok] - fx["logP"][ok]) <= fx["err_bound"][ok] + 1e-10).all()


def test_auto_escalates_beyond_the_128_bit_bound(ctx):
    """GBS_AUTO reruns in 192-bit fixed point exactly the valid results whose 128-bit bound
    exceeds 1e-10: the strongly cancelling patterns then match the 60-digit values to 1e-10
    with a bound below it; a pattern the 128-bit sweep resolves keeps its result bit for bit."""
    cases = [e for e in CASES["single"] if e["name"] == "m12_k6"]
    e = cases[0]
    U, r = g.haar_unitary(e["M"], e["seed"]), g.squeezing(e["M"], e["K"], e["r"][0], e["r"][1], e["seed"])
    pats = np.stack([g.modes_to_pattern(c["modes"]) for c in cases] + [g.modes_to_pattern([1, 4, 7])])
    auto = gpu(ctx, U, r, e["eta"], pats, "auto")
    fx = gpu(ctx, U, r, e["eta"], pats, "fx")
    wide = gpu(ctx, U, r, e["eta"], pats, "fx192")
    assert (auto["status"] == 0).all(), auto["status"]
    assert (auto["err_bound"] < 1e-10).all(), auto["err_bound"]
    for i, c in enumerate(cases):
        assert abs(auto["logP"][i] - c["logP"]) < 1e-10, (i, auto["logP"][i] - c["logP"])
    redo = (fx["status"] == 0) & (fx["err_bound"] > 1e-10)
    assert redo[:len(cases)].any() and not redo[-1]
    assert np.array_equal(auto["logP"][redo], wide["logP"][redo])
    assert np.array_equal(auto["logP"][~redo], fx["logP"][~redo])
    assert np.array_equal(auto["err_bound"][~redo], fx["err_bound"][~redo])
