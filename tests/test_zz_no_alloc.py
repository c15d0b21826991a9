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


def test_noalloc_matches_the_oracle(ctx):
    """The allocation-free sweep against the double-double oracle directly, on the
    smallest patterns of the 24-mode batch (fixed point and double-double, 1e-10)."""
    import oracle
    c = g.CONFIGS["m24_exact"]
    U, r = c.unitary(), c.squeezing()
    st = ctx.build_state(U, r, c.eta)
    pats = c.patterns()
    n = np.array([len(g.pattern_modes(p)) for p in pats])
    sel = np.argsort(n, kind="stable")[:12]
    ref = oracle.prob_exact(oracle.build_state(U, r, c.eta), pats[sel], dd=True)
    assert (ref["status"] == 0).all()
    for precision in ("fx", "dd"):
        for _ in range(2):
            out = ctx.prob_noalloc(st["O"], st["logdet"], pats[sel], int(n[sel].max()), precision=precision)
            torch.cuda.synchronize()
            assert (out["status"].cpu().numpy() == 0).all()
            d = np.abs(out["logP"].cpu().numpy() - ref["logP"])
            assert d.max() <= 1e-10, (precision, d.max())


def test_noalloc_understated_n_max_reports_nomem(ctx):
    """A caller that understates n_max passes the size check, but the batch's real work
    units do not fit in the fixed array: nothing is evaluated and every pattern reports
    GBS_E_NOMEM (the plan kernel sees the overflow; the sweep does no work)."""
    c = g.CONFIGS["m24_exact"]
    st = ctx.build_state(c.unitary(), c.squeezing(), c.eta)
    pats = c.patterns()
    n = np.array([len(g.pattern_modes(p)) for p in pats])
    big = np.repeat(pats[n == 20][:1], 4096, axis=0)   # 4096 x 256 units x 24 B > 8 MiB
    for _ in range(2):
        out = ctx.prob_noalloc(st["O"], st["logdet"], big, 10, precision="fx")
        torch.cuda.synchronize()
        assert (out["status"].cpu().numpy() == 3).all()    # GBS_E_NOMEM
        assert np.isnan(out["logP"].cpu().numpy()).all()
    # the next call that fits is unaffected by the overflowed one
    ok = ctx.prob_noalloc(st["O"], st["logdet"], pats[:64], int(n[:64].max()), precision="fx")
    ref = ctx.prob(st["O"], st["logdet"], pats[:64], precision="fx")
    torch.cuda.synchronize()
    assert np.array_equal(ok["status"].cpu().numpy(), ref["status"].cpu().numpy())
    assert np.abs(ok["logP"].cpu().numpy() - ref["logP"].cpu().numpy()).max() <= 1e-10
