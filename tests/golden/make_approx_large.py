"""Writes approx_large.json: the approximation oracle's log P on large patterns of the
50-mode and 100-mode workloads (Methods, "Approximation method"), for the GPU parity
tests that the oracle is too slow to run inline.

Only the oracle is called.  Every entry also records two measures of how sharply the
estimate depends on rounding at that pattern (each sector's fit extrapolates to the
all-clicked point, which is ill-conditioned at large n and order 4):
  spread   -- how far the oracle's log P moves when its contour radius is moved by -3%
              (or +0.5% near rho = 1): the estimate does not depend on the radius
              mathematically;
  sens     -- for relative table noise delta = 1e-12 (the rounding of FP64 minors), 3e-11
              (float-float: its unit roundoff ~2^-48 is 32 times FP64's) and 1e-5 (FP32
              minors): the largest change of log P when every entry
              of the oracle's moment tables D_w^(k) is multiplied by (1 + delta u), u
              uniform in [-1, 1] (four seeds), and the fits are run again.

    python tests/golden/make_approx_large.py [--workers 8]
"""
import argparse
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "approx_large.json")

# (workload, clicks, patterns with that many clicks, orders)
PLAN = [
    ("m50_approx", 23, 1, (2, 4)), ("m50_approx", 25, 1, (2, 4)), ("m50_approx", 28, 1, (2, 4)),
    ("m50_approx", 30, 1, (2, 4)), ("m50_approx", 33, 1, (2, 4)), ("m50_approx", 35, 1, (2, 4)),
    ("m50_approx", 38, 1, (2, 4)), ("m50_approx", 40, 1, (2, 4)),
    ("m100_approx", 41, 1, (4,)), ("m100_approx", 44, 1, (4,)), ("m100_approx", 45, 1, (4,)),
    ("m100_approx", 88, 1, (2,)), ("m100_approx", 90, 2, (2,)),
]


def job(args):
    name, idx, order = args
    sys.path.insert(0, ROOT)
    import numpy as np
    import gbs_inputs as g
    import oracle
    from oracle import approx as ap
    c = g.CONFIGS[name]
    st = oracle.build_state(c.unitary(), c.squeezing(), c.eta)
    modes = g.pattern_modes(c.patterns()[idx])
    t0 = time.time()
    lp, info = ap.approx_logprob(st.O, st.logdet, c.M, modes, order)
    rho, D = info["rho"], info["D"]
    f = 0.97 if rho * 0.97 >= 1.0 else 1.005
    lp2, _ = ap.approx_logprob(st.O, st.logdet, c.M, modes, order, rho=rho * f)
    sens = {}
    for delta in (1e-12, 3e-11, 1e-5):
        worst = 0.0
        for seed in range(4):
            u = np.random.default_rng(seed).uniform(-1.0, 1.0, size=D.shape)
            lpn, _, _ = ap.logprob_from_tables(D * (1.0 + delta * u), len(modes), order, rho, st.logdet)
            worst = max(worst, abs(lpn - lp))
        sens["%g" % delta] = worst
    return dict(workload=name, index=int(idx), n=len(modes), order=order, logP=lp, rho=rho, K=int(info["K"]),
                flag=int(info["flag"]), spread=abs(lp2 - lp), sens=sens, seconds=time.time() - t0)


def main():
    ap_ = argparse.ArgumentParser()
    ap_.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    a = ap_.parse_args()
    sys.path.insert(0, ROOT)
    import numpy as np
    import gbs_inputs as g
    jobs = []
    for name, nn, count, orders in PLAN:
        pats = g.CONFIGS[name].patterns()
        n = np.array([len(g.pattern_modes(p)) for p in pats])
        for idx in np.nonzero(n == nn)[0][:count]:
            jobs += [(name, int(idx), o) for o in orders]
    # the heaviest first
    jobs.sort(key=lambda j: -(len(g.pattern_modes(g.CONFIGS[j[0]].patterns()[j[1]])) ** j[2]))
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    with mp.get_context("spawn").Pool(a.workers) as pool:
        res = pool.map(job, jobs, chunksize=1)
    res.sort(key=lambda d: (d["workload"], d["n"], d["index"], d["order"]))
    with open(OUT, "w") as f:
        json.dump({"source": "oracle/approx.py approx_logprob (FP64, exact power series)",
                   "entries": res}, f, indent=1)
    print("wrote %d entries to %s" % (len(res), OUT))


if __name__ == "__main__":
    main()
