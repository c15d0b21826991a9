"""Pins of the multiprecision oracle (oracle/mp.py), which holds the stored values of the
192-bit fixed-point tests: it must equal the double-double oracle where that one is exact
(kappa <= 1e13: a different formula, the subset determinants of A = sigma_Q^-1), and on a
block-diagonal device the probability of a pattern must be the product of its blocks'
(the state and every determinant factorise), also where kappa is far beyond double-double."""
import numpy as np
import pytest

import gbs_inputs as g
import oracle

mpmath = pytest.importorskip("mpmath")
from oracle import mp as omp  # noqa: E402


def test_marginal_form_equals_double_double_oracle():
    M = 9
    U, r = g.haar_unitary(M, 31), g.squeezing(M, 9, 0.4, 0.9, 31)
    st = oracle.build_state(U, r, 0.6)
    for modes in ([0, 1, 2, 3, 4, 5, 6, 7, 8], [1, 2, 4, 6, 7], [3]):
        lp, kap = omp.logprob_marginal(st.sigmaQ, M, modes, dps=50)
        ref = oracle.prob_exact(st, g.modes_to_pattern(modes)[None], dd=True)
        assert ref["kappa"][0] < 1e13
        assert abs(lp - ref["logP"][0]) < 1e-13, (modes, lp - ref["logP"][0])
        assert abs(kap / ref["kappa"][0] - 1.0) < 1e-10


def test_block_diagonal_device_factorises_beyond_double_double():
    # two 5-mode blocks with weak squeezing: every all-click block cancels by ~1e12, the
    # 10-click pattern of the whole device by the product
    m = 5
    blocks = [(g.haar_unitary(m, s), g.squeezing(m, m, 0.05, 0.1, s)) for s in (41, 42)]
    U = np.zeros((2 * m, 2 * m), dtype=complex)
    r = np.zeros(2 * m)
    parts = []
    for b, (Ub, rb) in enumerate(blocks):
        U[b * m:(b + 1) * m, b * m:(b + 1) * m] = Ub
        r[b * m:(b + 1) * m] = rb
        stb = oracle.build_state(Ub, rb, 0.5)
        parts.append(omp.logprob_marginal(stb.sigmaQ, m, list(range(m)), dps=60))
    st = oracle.build_state(U, r, 0.5)
    lp, kap = omp.logprob_marginal(st.sigmaQ, 2 * m, list(range(2 * m)), dps=60)
    assert kap > 1e20
    assert abs(lp - (parts[0][0] + parts[1][0])) < 1e-12
    assert abs(kap / (parts[0][1] * parts[1][1]) - 1.0) < 1e-9
