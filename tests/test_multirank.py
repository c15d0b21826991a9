"""The N > 1 host paths on two gloo ranks (CPU): bench.py's shard of the weak-scaling
batch and the reductions that make the whole job's number (the slowest rank's time, the
sum of the ranks' work); and the data-parallel gradient (api.grad_sharded: round-robin
shards, one all-reduce of dL/dsigma_Q), with the per-rank gradient supplied by the
oracle in place of the GPU context."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

import gbs_inputs as g


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        c, U, r, pats, n = bench.workload("m24_exact", rank, world)
        mx = bench.max_over_ranks(1.5 * (rank + 1), world, "cpu")
        sm = bench.sum_over_ranks(float(n.sum()), world, "cpu")
        q.put((rank, pats, n, mx, sm))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_and_reduce():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(k, world, port, q)) for k in range(world)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(world):
        rank, pats, n, mx, sm = q.get(timeout=300)
        got[rank] = (pats, n, mx, sm)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    c = g.CONFIGS["m24_exact"]
    full = g.gen_patterns(c.seed, c.M, c.n_lo, c.n_hi, c.n_pat * world)
    # rank k holds patterns k n_pat .. (k + 1) n_pat - 1 of the job's batch; rank 0's shard
    # is the one-GPU batch itself
    assert np.array_equal(np.concatenate([got[0][0], got[1][0]]), full)
    assert np.array_equal(got[0][0], c.patterns())
    for k in range(world):
        assert got[k][2] == 3.0                                   # the slowest rank's time
        assert got[k][3] == float(got[0][1].sum() + got[1][1].sum())  # the job's work


class _OracleCtx:
    """Stands in for the GPU context in grad_sharded: the same grad / grad_approx calls,
    answered by the oracle on the CPU."""

    def __init__(self, state):
        self.state = state

    def grad(self, O, logdet, pats, w):
        import torch
        from oracle import grad as og
        from paper_2106_01445_gb300.api import patterns_numpy
        d = og.grad_sigmaQ(self.state, patterns_numpy(pats), w.numpy())
        return torch.from_numpy(d), torch.zeros(len(pats), dtype=torch.float64), torch.zeros(len(pats),
                                                                                             dtype=torch.int32)

    def grad_approx(self, O, logdet, pats, w, order):
        import torch
        from oracle import grad as og
        from paper_2106_01445_gb300.api import patterns_numpy
        d, lp = og.grad_sigmaQ_approx(self.state, patterns_numpy(pats), w.numpy(), order)
        return torch.from_numpy(d), torch.from_numpy(lp), torch.zeros(len(pats), dtype=torch.int32)


def _grad_case():
    import oracle
    M = 8
    U = g.haar_unitary(M, 6)
    r = g.squeezing(M, 4, 0.6, 1.0, 6)
    st = oracle.build_state(U, r, 0.7)
    pats = g.gen_patterns(6, M, 1, 5, 7)          # 7 patterns: uneven shards over 2 ranks
    w = np.linspace(-1.0, 1.5, 7)
    return st, pats, w


def _grad_rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2106_01445_gb300.api import grad_sharded
        st, pats, w = _grad_case()
        out = {}
        for order in (0, 2):
            dsq, idx, _, _ = grad_sharded(_OracleCtx(st), torch.from_numpy(st.O), torch.tensor([st.logdet]),
                                          pats, w, order=order)
            out[order] = (dsq.numpy(), idx.numpy())
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gradient_all_reduce():
    from oracle import grad as og
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_grad_rank, args=(k, world, port, q)) for k in range(world)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(world):
        rank, out = q.get(timeout=300)
        got[rank] = out
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    st, pats, w = _grad_case()
    full = {0: og.grad_sigmaQ(st, pats, w), 2: og.grad_sigmaQ_approx(st, pats, w, 2)[0]}
    for order in (0, 2):
        # round-robin shards: every pattern on exactly one rank
        assert sorted(np.concatenate([got[0][order][1], got[1][order][1]]).tolist()) == list(range(len(pats)))
        for k in range(world):
            d = got[k][order][0]
            assert np.abs(d - full[order]).max() < 1e-12 * np.abs(full[order]).max(), (order, k)


class _OracleSliceCtx:
    """Stands in for the GPU context in prob_sharded: slice k of N of every pattern's
    subsets (the mask range [2^n k / N, 2^n (k + 1) / N)) summed by the double-double
    oracle, and the slices combined in order with TwoSum, as the library's combine does."""

    def __init__(self, state):
        self.state = state

    def prob_partial(self, O, patterns, part, nparts, precision="fx"):
        import torch
        import oracle
        pats = np.asarray(patterns, dtype=np.uint64).reshape(-1, 2)
        out = np.zeros((len(pats), 3))
        for p, pat in enumerate(pats):
            modes = g.pattern_modes(pat)
            b, e = (1 << len(modes)) * part // nparts, (1 << len(modes)) * (part + 1) // nparts
            if e > b:
                out[p] = oracle.subset_sum(self.state.A, self.state.M, modes, b, e, dd=True)
        return torch.from_numpy(out), torch.zeros(len(pats), dtype=torch.int32)

    def prob_combine(self, logdet, patterns, partials, pflags, precision="fx"):
        import math
        import torch
        P = partials.numpy()
        logP = np.zeros(P.shape[1])
        for p in range(P.shape[1]):
            h = l = 0.0
            for q in range(P.shape[0]):
                s = h + P[q, p, 0]
                bp = s - h
                e = (h - (s - bp)) + (P[q, p, 0] - bp)
                h, l = s, l + P[q, p, 1] + e
            logP[p] = -0.5 * float(logdet[0]) + math.log(h) + math.log1p(l / h)
        return dict(logP=torch.from_numpy(logP), status=torch.zeros(P.shape[1], dtype=torch.int32))


def _strong_case():
    import oracle
    M = 14
    U = g.haar_unitary(M, 21)
    r = g.squeezing(M, 7, 0.6, 1.1, 21)
    st = oracle.build_state(U, r, 0.6)
    pats = g.gen_patterns(21, M, 3, 13, 9)
    return st, pats


def _strong_rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2106_01445_gb300.api import prob_sharded
        st, pats = _strong_case()
        out = prob_sharded(_OracleSliceCtx(st), torch.from_numpy(st.O),
                           torch.tensor([st.logdet], dtype=torch.float64), pats)
        q.put((rank, out["logP"].numpy()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_strong_split_combines_to_one_rank():
    """One batch evaluated by two ranks together: each sweeps its slice of every pattern's
    subsets, one all_gather exchanges the per-pattern double-double partial sums, and each
    rank combines them in rank order.  Both ranks hold the same log P, bit for bit, and it
    equals the one-rank (whole-batch) double-double result."""
    import oracle
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_strong_rank, args=(k, world, port, q)) for k in range(world)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(world):
        rank, lp = q.get(timeout=300)
        got[rank] = lp
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    st, pats = _strong_case()
    one = oracle.prob_exact(st, pats, dd=True)["logP"]
    assert np.array_equal(got[0], got[1])
    assert np.abs(got[0] - one).max() < 1e-12
