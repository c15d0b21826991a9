"""The flop counts behind `roofline.achieved` (bench.py): the include/exclude recursion's
algorithmic count against a walk of the tree itself, small cases by hand, and the per-subset
limits the series give (44 for the method's count, 50 for the kernels' own)."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
bench = importlib.util.module_from_spec(spec)
spec.loader.exec_module(bench)


def tree_walk(m, u):
    """Sum of u(r) over the include steps of the include/exclude tree on m modes: a node
    with m modes left includes its first one (r = m - 1 left after it) and has two children
    of m - 1 modes; leaves (m = 0) cost nothing."""
    if m == 0:
        return 0
    return u(m - 1) + 2 * tree_walk(m - 1, u)


def u_alg(r):
    return 8 * r * r + 10 * r + 10


def u_exec(r):
    return 8 * r * r + 16 * r + 9


@pytest.mark.parametrize("n", range(1, 13))
def test_counts_equal_a_walk_of_the_tree(n):
    assert bench.schur_flops(n) == tree_walk(n, u_alg)
    assert bench.schur_flops_executed(n) == tree_walk(n, u_exec) + 2 ** n   # one add per leaf


def test_small_cases_by_hand():
    assert bench.schur_flops(1) == 10             # one include step with nothing left
    assert bench.schur_flops(2) == 28 + 2 * 10    # u(1) at the root, u(0) at both children


def test_per_subset_limits():
    # sum_r r^2 / 2^(r+1) = 3, sum_r r / 2^(r+1) = 1, sum_r 1 / 2^(r+1) = 1
    assert abs(bench.schur_flops(60) / 2 ** 60 - (8 * 3 + 10 * 1 + 10 * 1)) < 1e-9
    assert abs(bench.schur_flops_executed(60) / 2 ** 60 - (8 * 3 + 16 * 1 + 9 * 1 + 1)) < 1e-9
    assert abs(bench.schur_flops(8) / 2 ** 8 - 41.02) < 0.005
