"""GPU parity of the exact path (state build, pattern generation, signed subset
sweep) against the oracle, through the C ABI.

Improbable click patterns cancel by many orders of magnitude in the signed
sum (kappa = sum|term|/|T| reaches 1e13 on the 24-mode workload), so the
reference is the double-double oracle.  Bounds: the double-double and the
fixed-point paths must match it to 1e-10 in log P; the FP64 path to 1e-10 wherever its own
a-posteriori bound is below that, else within the bound; the FP32 split within
its bound, or it reports GBS_E_NONPOSITIVE when its sum loses the sign."""
import math

import numpy as np
import pytest
import torch

import gbs_inputs as g
import oracle

pytestmark = pytest.mark.gpu

# |d log P| bounds: FP64 path 1e-10 wherever the a-posteriori bound is below it;
# otherwise (and in the FP32 split) the library's own err_bound must hold.
TOL64 = 1e-10


@pytest.fixture(scope="module")
def ctx(cuda_ok):
    from paper_2106_01445_gb300 import build
    build.build()
    from paper_2106_01445_gb300.api import Context
    return Context(0)


def gpu_state(ctx, U, r, eta):
    return ctx.build_state(U, r, eta, want_sigma=True)


def gpu_prob(ctx, st, pats, precision, order=0):
    out = ctx.prob(st["O"], st["logdet"], pats, order=order, precision=precision)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def check_against_oracle(res, ref, precision):
    ok = ref["status"] == 0
    st = res["status"][ok]
    if precision == "fp32":
        assert np.isin(st, (0, 4)).all(), st
        ok = ok & (res["status"] == 0)
    else:
        assert (st == 0).all(), st
    d = np.abs(res["logP"][ok] - ref["logP"][ok])
    bound = res["err_bound"][ok]
    if precision in ("dd", "fx"):
        assert (d <= TOL64).all(), (d.max(), res["kappa"][ok][d.argmax()])
    elif precision == "fp64":
        assert (d <= np.maximum(TOL64, bound)).all(), (d.max(), bound[d.argmax()])
        tight = bound <= 1e-11
        assert (d[tight] <= TOL64).all()
    else:
        assert (d <= bound).all(), (d.max(), bound[d.argmax()], res["kappa"][ok][d.argmax()])
    return d


def oracle_dd(U, r, eta, pats):
    return oracle.prob_exact(oracle.build_state(U, r, eta), pats, dd=True)


@pytest.mark.parametrize("name,eta", [("m8_all", 1.0), ("m24_exact", 0.5), ("m100_approx", 0.3),
                                      ("m32_grad", 0.6)])
def test_state_build_parity(ctx, name, eta):
    c = g.CONFIGS[name]
    U, r = c.unitary(), c.squeezing()
    st = gpu_state(ctx, U, r, eta)
    ref = oracle.build_state(U, r, eta)
    assert np.abs(st["O"].cpu().numpy() - ref.O).max() < 1e-13
    assert np.abs(st["sigma"].cpu().numpy() - ref.sigma).max() < 1e-12 * np.abs(ref.sigma).max()
    assert abs(st["logdet"].item() - ref.logdet) < 1e-12 * max(1.0, abs(ref.logdet))


def test_state_build_rejects_bad_input(ctx):
    from paper_2106_01445_gb300 import GbsError
    U = g.haar_unitary(5, 1)
    with pytest.raises(GbsError):
        ctx.build_state(1.01 * U, np.full(5, 0.5), 0.5)
    with pytest.raises(GbsError):
        ctx.build_state(U, np.array([0.5, -0.1, 0, 0, 0]), 0.5)
    with pytest.raises(GbsError):
        ctx.build_state(U, np.full(5, 0.5), 1.5)


@pytest.mark.parametrize("M,n_lo,n_hi,n_pat,seed,stream", [
    (24, 12, 20, 1024, 2, 2), (50, 10, 40, 4096, 3, 2), (100, 40, 90, 3000, 5, 2),
    (100, 30, 30, 64, 5, 3), (128, 0, 128, 500, 7, 2), (8, 0, 8, 333, 0, 2)])
def test_gen_patterns_bit_exact(ctx, M, n_lo, n_hi, n_pat, seed, stream):
    from paper_2106_01445_gb300.api import patterns_numpy
    dev = patterns_numpy(ctx.gen_patterns(seed, stream, M, n_lo, n_hi, n_pat))
    host = g.gen_patterns(seed, M, n_lo, n_hi, n_pat, stream=stream)
    assert np.array_equal(dev, host)


@pytest.mark.parametrize("precision", ["dd", "fx", "fp64", "fp32"])
@pytest.mark.parametrize("eta", [1.0, 0.5])
def test_all_patterns_m8(ctx, precision, eta):
    c = g.CONFIGS["m8_all"]
    U, r = c.unitary(), c.squeezing()
    pats = g.all_patterns(8)
    res = gpu_prob(ctx, gpu_state(ctx, U, r, eta), pats, precision)
    ref = oracle_dd(U, r, eta, pats)
    check_against_oracle(res, ref, precision)
    p = np.exp(res["logP"])
    if precision != "fp32":
        assert abs(p.sum() - 1.0) < (1e-14 if precision in ("dd", "fx") else 1e-12)
    else:
        assert abs(np.nansum(p) - 1.0) < 1e-4


@pytest.fixture(scope="module")
def uneven():
    # patterns of every size 0..18 (ragged: the padding n < B, one-unit, multi-unit
    # and multi-sub-unit shapes of every precision) in one launch
    M = 26
    U = g.haar_unitary(M, 101)
    r = g.squeezing(M, 13, 0.6, 1.2, 101)
    rng = np.random.default_rng(5)
    sizes = list(range(0, 19)) + [3, 7, 13, 14, 15, 17]
    modes_list = [sorted(rng.choice(M, size=n, replace=False)) for n in sizes]
    pats = np.stack([g.modes_to_pattern(m) for m in modes_list])
    return U, r, pats, oracle_dd(U, r, 0.55, pats)


@pytest.mark.parametrize("precision", ["dd", "fx", "fp64", "fp32"])
def test_uneven_batch_all_sizes(ctx, uneven, precision):
    U, r, pats, ref = uneven
    st = gpu_state(ctx, U, r, 0.55)
    res = gpu_prob(ctx, st, pats, precision)
    check_against_oracle(res, ref, precision)
    assert abs(res["logP"][0] + 0.5 * st["logdet"].item()) < 1e-14   # empty pattern


@pytest.fixture(scope="module")
def m24_sample():
    # the 24-mode workload; the oracle checks a sample spanning the click counts
    c = g.CONFIGS["m24_exact"]
    U, r = c.unitary(), c.squeezing()
    pats = c.patterns()
    n = np.array([len(g.pattern_modes(p)) for p in pats])
    idx = []
    for k in range(12, 19):
        w = np.nonzero(n == k)[0]
        idx += list(w[: (2 if k <= 16 else 1)])
    idx = np.array(idx)
    return c, U, r, pats, idx, oracle_dd(U, r, c.eta, pats[idx])


@pytest.mark.parametrize("precision", ["dd", "fx", "fp64", "fp32"])
def test_m24_config_sample(ctx, m24_sample, precision):
    # the benchmark's launch shape: all 1024 patterns in one call
    c, U, r, pats, idx, ref = m24_sample
    res = gpu_prob(ctx, gpu_state(ctx, U, r, c.eta), pats, precision)
    sub = {k: v[idx] for k, v in res.items()}
    check_against_oracle(sub, ref, precision)
    if precision != "fp32":
        assert (res["status"] == 0).all()


def test_precisions_agree_full_config(ctx):
    # every pattern of the workload: FP64 and FP32 results lie within their bounds
    # of the double-double result
    c = g.CONFIGS["m24_exact"]
    st = gpu_state(ctx, c.unitary(), c.squeezing(), c.eta)
    ref = gpu_prob(ctx, st, c.patterns(), "dd")
    assert (ref["status"] == 0).all()
    for prec in ("fp64", "fp32"):
        a = gpu_prob(ctx, st, c.patterns(), prec)
        ok = a["status"] == 0
        assert (ok | (prec == "fp32")).all()
        d = np.abs(a["logP"][ok] - ref["logP"][ok])
        assert (d <= a["err_bound"][ok] + 1e-12).all(), prec


def test_block_diagonal_factorises_at_n30(ctx):
    # Property at full size: with a block-diagonal interferometer the click
    # probability factorises over blocks; each block is exact from the
    # double-double oracle.  30 clicks fill three 10-mode blocks (kappa multiplies
    # over clicked blocks, so few clicked blocks keep it within double-double).
    M, bs = 100, 10
    U = np.zeros((M, M), dtype=complex)
    for b in range(M // bs):
        U[b * bs:(b + 1) * bs, b * bs:(b + 1) * bs] = g.haar_unitary(bs, 200 + b)
    r = g.squeezing(M, M, 1.3, 1.6, 77)
    eta = 0.9
    clicked_blocks = [(0, 3, 7), (1, 2, 9)]
    pats = np.stack([g.modes_to_pattern([m for b in cb for m in range(b * bs, (b + 1) * bs)])
                     for cb in clicked_blocks])
    st = gpu_state(ctx, U, r, eta)
    refs = []
    for cb in clicked_blocks:
        lp = 0.0
        for b in range(M // bs):
            blk = list(range(b * bs, (b + 1) * bs))
            sub = oracle.build_state(U[np.ix_(blk, blk)], r[blk], eta)
            loc = list(range(bs)) if b in cb else []
            lp += oracle.prob_exact(sub, g.modes_to_pattern(loc)[None], dd=True)["logP"][0]
        refs.append(lp)
    for precision in ("dd", "fx", "fp64"):
        res = gpu_prob(ctx, st, pats, precision)
        for i in range(len(pats)):
            assert res["status"][i] == 0
            d = abs(res["logP"][i] - refs[i])
            if precision in ("dd", "fx"):
                assert res["err_bound"][i] < 1e-10 and d <= TOL64, (i, d, res["kappa"][i])
            else:
                assert d <= max(TOL64, res["err_bound"][i]), (precision, i)


def test_large_pattern_against_parallel_oracle(ctx):
    # one 20-click pattern of the 24-mode device, double-double oracle over 1M
    # subsets in parallel
    c = g.CONFIGS["m24_exact"]
    U, r = c.unitary(), c.squeezing()
    modes = [m for m in range(24) if m not in (3, 8, 17, 21)]
    st = gpu_state(ctx, U, r, c.eta)
    ref_state = oracle.build_state(U, r, c.eta)
    T = oracle.subset_sum(ref_state.A, 24, modes, nchunk=256, dd=True)
    ref = -0.5 * ref_state.logdet + math.log(T[0]) + math.log1p(T[1] / T[0])
    for precision in ("dd", "fx", "fp64"):
        res = gpu_prob(ctx, st, g.modes_to_pattern(modes)[None], precision)
        tol = TOL64 if precision in ("dd", "fx") else max(TOL64, res["err_bound"][0])
        assert abs(res["logP"][0] - ref) <= tol, precision


def test_deterministic(ctx):
    c = g.CONFIGS["m24_exact"]
    st = gpu_state(ctx, c.unitary(), c.squeezing(), c.eta)
    for precision in ("dd", "fx", "fp64", "fp32"):
        a = gpu_prob(ctx, st, c.patterns(), precision)["logP"]
        b = gpu_prob(ctx, st, c.patterns(), precision)["logP"]
        assert np.array_equal(a, b, equal_nan=True)


def test_fixed_point_range_flagged(ctx):
    # two modes squeezed so strongly (r = 4: sigma_Q has eigenvalue ~1490) that their
    # pivot determinants fall below 2^-8: the fixed-point path reports GBS_E_RANGE
    # for every pattern that clicks one of them and stays exact on the others
    M = 6
    U = np.eye(M, dtype=complex)
    r = np.array([4.0, 4.0, 0.5, 0.6, 0.7, 0.8])
    mode_sets = [[2, 3], [2, 3, 4, 5], [4], [0], [1, 2], [0, 1, 4]]
    pats = np.stack([g.modes_to_pattern(m) for m in mode_sets])
    st = gpu_state(ctx, U, r, 1.0)
    res = gpu_prob(ctx, st, pats, "fx")
    ref = oracle_dd(U, r, 1.0, pats)
    in_range = np.array([not ({0, 1} & set(m)) for m in mode_sets])
    assert (res["status"][~in_range] == 8).all(), res["status"]
    assert (res["status"][in_range] == 0).all(), res["status"]
    assert np.abs(res["logP"][in_range] - ref["logP"][in_range]).max() <= TOL64
    dd = gpu_prob(ctx, st, pats, "dd")
    assert (dd["status"] == 0).all()
    assert np.abs(dd["logP"] - ref["logP"]).max() <= TOL64


def test_auto_precision_reruns_out_of_range_patterns(ctx):
    """GBS_AUTO: the fixed-point pass, then double-double for the patterns it flagged out of
    range, on the device: every pattern ok; the in-range ones carry the fixed-point result bit
    for bit, the others the double-double one."""
    M = 6
    U = np.eye(M, dtype=complex)
    r = np.array([4.0, 4.0, 0.5, 0.6, 0.7, 0.8])
    mode_sets = [[2, 3], [2, 3, 4, 5], [4], [0], [1, 2], [0, 1, 4], [3, 5], [0, 2, 3, 4, 5]]
    pats = np.stack([g.modes_to_pattern(m) for m in mode_sets])
    st = gpu_state(ctx, U, r, 1.0)
    auto = gpu_prob(ctx, st, pats, "auto")
    fx = gpu_prob(ctx, st, pats, "fx")
    dd = gpu_prob(ctx, st, pats, "dd")
    ref = oracle_dd(U, r, 1.0, pats)
    assert (auto["status"] == 0).all(), auto["status"]
    flagged = fx["status"] == 8
    assert flagged.any() and (~flagged).any()
    assert np.array_equal(auto["logP"][~flagged], fx["logP"][~flagged])
    assert np.array_equal(auto["logP"][flagged], dd["logP"][flagged])
    assert np.abs(auto["logP"] - ref["logP"]).max() <= TOL64


def test_invalid_patterns_flagged(ctx):
    M = 10
    st = gpu_state(ctx, g.haar_unitary(M, 3), g.squeezing(M, 5, 0.5, 1.0, 3), 0.7)
    pats = np.array([[1 << 12, 0], [0b1011, 0], [0, 1], [(1 << 41) - 1, 0]], dtype=np.uint64)
    res = gpu_prob(ctx, st, pats, "fp64")
    assert res["status"][0] == 1 and res["status"][2] == 1    # detector index >= M
    assert res["status"][1] == 0
    assert res["status"][3] == 1                               # beyond M


def test_host_entry_point_matches_device_path(ctx):
    c = g.CONFIGS["m24_exact"]
    U, r, pats = c.unitary(), c.squeezing(), c.patterns()[:200]
    dev = gpu_prob(ctx, gpu_state(ctx, U, r, c.eta), pats, "fp32")
    host = ctx.run_host(U, r, c.eta, pats, precision="fp32")
    assert np.array_equal(dev["logP"], host["logP"], equal_nan=True)
    assert np.array_equal(dev["status"], host["status"])
