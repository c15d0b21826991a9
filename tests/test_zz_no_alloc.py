"""The allocation-free entry point gbs_prob_noalloc, for callers that cannot
call cudaMalloc (work captured into another owner's CUDA graph, device memory
held by another framework's pool, serving loops that must not wait on the
allocator).  It must give the same results as gbs_prob, call after call, with
its scratch in the library's fixed device array.  This file is collected last."""
import numpy as np
import pytest
import torch

import gbs_inputs as g

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(cuda_ok):
    from paper_2106_01445_gb300 import build
    build.build()
    from paper_2106_01445_gb300.api import Context
    return Context(0)


@pytest.mark.parametrize("precision", ["dd", "fx", "fp64", "fp32"])
def test_noalloc_matches_gbs_prob_twice(ctx, precision):
    c = g.CONFIGS["m24_exact"]
    st = ctx.build_state(c.unitary(), c.squeezing(), c.eta)
    pats = c.patterns()
    n_max = max(len(g.pattern_modes(p)) for p in pats)
    ref = ctx.prob(st["O"], st["logdet"], pats, precision=precision)
    torch.cuda.synchronize()
    ref = {k: v.cpu().numpy() for k, v in ref.items()}
    for _ in range(2):      # the shared scratch keeps the last call's contents
        out = ctx.prob_noalloc(st["O"], st["logdet"], pats, n_max, precision=precision)
        torch.cuda.synchronize()
        out = {k: v.cpu().numpy() for k, v in out.items()}
        assert np.array_equal(out["status"], ref["status"])
        ok = ref["status"] == 0
        d = np.abs(out["logP"][ok] - ref["logP"][ok])
        tol = 1e-10 if precision in ("dd", "fx") else np.maximum(1e-10, ref["err_bound"][ok])
        assert (d <= tol).all()


def test_noalloc_rejects_oversized_batches(ctx):
    from paper_2106_01445_gb300 import GbsError
    c = g.CONFIGS["m24_exact"]
    st = ctx.build_state(c.unitary(), c.squeezing(), c.eta)
    pats = np.repeat(c.patterns()[:1], 20000, axis=0)
    with pytest.raises(GbsError):
        ctx.prob_noalloc(st["O"], st["logdet"], pats, 20, precision="fp64")
    with pytest.raises(GbsError):
        ctx.prob_noalloc(st["O"], st["logdet"], c.patterns(), 40, precision="dd")
