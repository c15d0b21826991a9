"""Writes fx192_cases.json: exact log P of click patterns whose signed sums cancel by
kappa = 1e22 .. 1e31, for the GPU tests of the 192-bit fixed-point sweep.

Only the oracle is called: oracle.mp.logprob_marginal, the marginal form of P(S) (Methods,
"Probability of any sample") in 60-digit arithmetic.  Two kinds of case:
  * single devices with weak squeezing, where improbable patterns cancel by up to 1e31;
  * a block-diagonal device of three 10-mode blocks (block-diagonal interferometer, loss and
    squeezing per mode, so the state and every subset determinant factorise): the 30-click
    pattern's P is the product of the blocks' all-click probabilities, each evaluated on its
    own, and its kappa the product of theirs (~4e28, like the 30-click anchors of the
    100-mode workload), while the GPU sweeps all 2^30 subsets of the whole device.

    python tests/golden/make_fx192_cases.py [--workers 8]
"""
import argparse
import json
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "fx192_cases.json")

# name -> (M, squeezed inputs, r_lo, r_hi, eta, seed, patterns as mode lists)
SINGLE = {
    "m12_k6": (12, 6, 0.1, 0.2, 0.2, 7, [list(range(12)), list(range(10)), [0, 2, 3, 5, 6, 8, 9, 11]]),
    "m12_weak": (12, 12, 0.02, 0.05, 0.3, 10, [list(range(10)), list(range(12))]),
}
# three blocks of BLOCK_M modes, block b: Haar seed 20 + b, every input squeezed, r ~ U[0.4, 0.8]
BLOCK_M, BLOCK_R, BLOCK_ETA, BLOCK_SEEDS = 10, (0.4, 0.8), 0.4, (20, 21, 22)


def job(a):
    sys.path.insert(0, ROOT)
    import gbs_inputs as g
    import oracle
    from oracle import mp as omp
    kind, key, extra = a
    if kind == "single":
        M, K, rlo, rhi, eta, seed, pats = SINGLE[key]
        U, r = g.haar_unitary(M, seed), g.squeezing(M, K, rlo, rhi, seed)
        modes = pats[extra]
    else:
        M, seed = BLOCK_M, key
        U, r = g.haar_unitary(M, seed), g.squeezing(M, M, BLOCK_R[0], BLOCK_R[1], seed)
        modes, eta = list(range(M)), BLOCK_ETA
    st = oracle.build_state(U, r, eta)
    lp, kap = omp.logprob_marginal(st.sigmaQ, M, modes, dps=60)
    return kind, key, extra, lp, kap


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    jobs = [("single", k, i) for k, v in SINGLE.items() for i in range(len(v[6]))]
    jobs += [("block", s, 0) for s in BLOCK_SEEDS]
    with mp.get_context("spawn").Pool(a.workers) as pool:
        res = pool.map(job, jobs, chunksize=1)
    out = {"source": "oracle/mp.py logprob_marginal, 60 digits", "single": [], "block": {}}
    for kind, key, extra, lp, kap in res:
        if kind == "single":
            M, K, rlo, rhi, eta, seed, pats = SINGLE[key]
            out["single"].append(dict(name=key, M=M, K=K, r=[rlo, rhi], eta=eta, seed=seed, modes=pats[extra],
                                      logP=lp, kappa=kap))
        else:
            out["block"].setdefault("blocks", []).append(dict(seed=key, logP=lp, kappa=kap))
    out["block"].update(M=BLOCK_M, r=list(BLOCK_R), eta=BLOCK_ETA, seeds=list(BLOCK_SEEDS),
                        logP=sum(b["logP"] for b in out["block"]["blocks"]),
                        kappa=float(__import__("math").prod(b["kappa"] for b in out["block"]["blocks"])))
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
