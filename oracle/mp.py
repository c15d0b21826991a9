"""Arbitrary-precision evaluation of P(S) for signed sums that cancel beyond double-double
(test infrastructure only: the tests and the scripts that write their stored values).

Methods, "Probability of any sample": the probability that every detector of S clicks and
every other detector stays dark is the inclusion-exclusion over the subsets Z of S of the
probabilities that every detector outside Z is dark,
    P(S) = sum_{Z subset S} (-1)^{|S| - |Z|} det(sigma_Q restricted to the modes not in Z)^{-1/2},
the marginal form (independent of A = sigma_Q^{-1} and of the determinant recursion the GPU
uses).  Every determinant and the sum are taken in mpmath with `dps` decimal digits, the
entries of sigma_Q (FP64) exact, so log P is exact to far below 1e-10 for kappa up to about
10^(dps - 20).
"""
from __future__ import annotations

import numpy as np


def logprob_marginal(sigmaQ: np.ndarray, M: int, modes, dps: int = 60):
    """(log P(S), kappa) with kappa = sum of |terms| / |P|, in mpmath at `dps` digits."""
    import mpmath
    modes = list(modes)
    n = len(modes)
    with mpmath.workdps(dps):
        total = mpmath.mpf(0)
        absum = mpmath.mpf(0)
        for z in range(1 << n):
            Z = {modes[i] for i in range(n) if z >> i & 1}
            W = [i for i in range(M) if i not in Z]
            rows = W + [i + M for i in W]
            d = mpmath.det(mpmath.matrix(sigmaQ[np.ix_(rows, rows)].tolist())) if rows else mpmath.mpf(1)
            term = 1 / mpmath.sqrt(d)
            absum += term
            total += term if (n - len(Z)) % 2 == 0 else -term
        return float(mpmath.log(total)), float(absum / abs(total))
