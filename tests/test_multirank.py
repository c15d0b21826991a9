"""The N > 1 host path of bench.py on two gloo ranks (CPU): each rank's shard of the
weak-scaling batch, and the reductions that make the whole job's number (the slowest
rank's time, the sum of the ranks' work)."""
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
