"""GPU parity of the batch split across GPUs (gbs_prob_partial + gbs_prob_combine).

Runs here on one GPU: the N slices a multi-GPU job would give its N ranks are swept one
after another on the same device (no kernel waits on another), and their per-pattern
partial sums are combined in slice order, as api.prob_sharded does after its
all_gather.  The combined result must equal the whole-batch gbs_prob to 1e-12 in log P
(only the order of the double-double additions differs) and the double-double oracle to
1e-10; statuses must match."""
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


def sliced(ctx, st, pats, nparts, precision):
    parts, flags = [], []
    for k in range(nparts):
        p, f = ctx.prob_partial(st["O"], pats, k, nparts, precision=precision)
        parts.append(p)
        flags.append(f)
    out = ctx.prob_combine(st["logdet"], pats, torch.stack(parts), torch.stack(flags), precision=precision)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("precision", ["fx", "dd", "fp64"])
@pytest.mark.parametrize("nparts", [1, 2, 3, 8])
def test_slices_combine_to_whole_batch(ctx, precision, nparts):
    c = g.CONFIGS["m24_exact"]
    st = ctx.build_state(c.unitary(), c.squeezing(), c.eta)
    pats = c.patterns()
    whole = ctx.prob(st["O"], st["logdet"], pats, precision=precision)
    torch.cuda.synchronize()
    whole = {k: v.cpu().numpy() for k, v in whole.items()}
    res = sliced(ctx, st, pats, nparts, precision)
    assert np.array_equal(res["status"], whole["status"])
    ok = whole["status"] == 0
    assert np.abs(res["logP"][ok] - whole["logP"][ok]).max() < 1e-12
    assert np.allclose(res["kappa"][ok], whole["kappa"][ok], rtol=1e-9)


def test_one_large_pattern_cut_by_prefix(ctx):
    # a single 20-click pattern over 7 slices: every slice holds part of its subsets
    c = g.CONFIGS["m24_exact"]
    U, r = c.unitary(), c.squeezing()
    st = ctx.build_state(U, r, c.eta)
    pats = c.patterns()
    n = np.array([len(g.pattern_modes(p)) for p in pats])
    one = pats[n == 20][:1]
    res = sliced(ctx, st, one, 7, "fx")
    ref = oracle.prob_exact(oracle.build_state(U, r, c.eta), one, dd=True)
    assert res["status"][0] == 0
    assert abs(res["logP"][0] - ref["logP"][0]) < 1e-10
    for k in range(7):
        p, _ = ctx.prob_partial(st["O"], one, k, 7, precision="fx")
        assert p[0, 2].item() > 0.0          # sum |terms| of the slice: it holds subsets


def test_slices_against_oracle_and_bad_patterns(ctx):
    M = 12
    U, r = g.haar_unitary(M, 77), g.squeezing(M, 6, 0.6, 1.2, 77)
    st = ctx.build_state(U, r, 0.7)
    pats = np.concatenate([g.gen_patterns(77, M, 0, 12, 40), np.array([[1 << 13, 0]], dtype=np.uint64)])
    res = sliced(ctx, st, pats, 5, "fx")
    ref = oracle.prob_exact(oracle.build_state(U, r, 0.7), pats[:-1], dd=True)
    assert res["status"][-1] == 1                              # a detector beyond M: invalid
    assert (res["status"][:-1] == 0).all()
    assert np.abs(res["logP"][:-1] - ref["logP"]).max() < 1e-10
