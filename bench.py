"""Benchmark: exact click-pattern probabilities on one GB300 (or N, one rank each).

One step = the whole exact path on one batch: state build (sigma, O, log det
sigma_Q from U, r, eta) plus the signed subset sweep for every click pattern of
the batch.  Default workload: 24 modes, 12 squeezed inputs r ~ U[0.6, 1.2],
eta = 0.5, Haar U, 1024 patterns with n ~ U{12..20} clicks (2.4e8 subsets).
These uniformly drawn patterns are improbable and their signed sums cancel by
kappa = 1e10..1e15, so the default precision is the 128-bit fixed-point sweep
(accuracy of double-double, the other precision that meets 1e-10 in log P here,
on the integer pipes); double-double, FP64 and the FP32 split are timed
alongside and the error of each against the double-double oracle is reported.
Metric: subset log-dets per second (whole job), plus patterns per second.

    python bench.py [--gpus N --steps K --warmup W --precision fx|dd|fp64|fp32]
    python bench.py --impl reference     # the FP64 CPU oracle on the host cores
    python bench.py --profile sweep|approx|grad --precision ...   # one call, for ncu
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gbs_inputs as g  # noqa: E402

METRIC = "subset logdets/sec and click-pattern log P/sec at stated rel. error vs FP64 oracle"
# dram__bytes_read.sum + dram__bytes_write.sum of one sweep launch on this workload
# (ncu captures summarised under profiles/); None where no capture of the current kernel exists
DRAM_TRAFFIC = {"fp32": 129536.0, "dd": 396800.0, "fp64": 130048.0, "fx": 182784.0}
UNIT = "subset logdets/s"
# 32-bit multiply-adds of one fixed-point update entry: two 128 x 128-bit products
# truncated to their top 128 bits, 23 IMAD each (3 + 5 + 7 + 8 over the four rows)
FX_IMAD_PER_ENTRY = 46
L2_FLUSH_BYTES = 512 << 20      # > 129 MB L2


def schur_flops(n: int) -> float:
    """Algorithmic flops of the include/exclude Schur recursion over n modes, counted
    as the method must do them: every internal node at depth k includes its next mode
    with r = n-1-k modes left, costing u(r) = 8 r^2 + 10 r + 10 (2x2 Cholesky ~10,
    triangular solve of the 2 x 2r pivot rows ~6r, rank-2 symmetric update of the
    2r x 2r rest 4r(2r+1)); F(n) = sum_k 2^k u(n-1-k), which tends to 44 flops per
    subset (8 * 3 + 10 * 1 + 10 * 1, from sum_r r^2/2^(r+1) = 3, sum_r r/2^(r+1) = 1
    and sum_r 1/2^(r+1) = 1)."""
    tot = 0.0
    for k in range(n):
        r = n - 1 - k
        tot += (1 << k) * (8 * r * r + 10 * r + 10)
    return tot


def schur_flops_executed(n: int) -> float:
    """The same recursion counted as the kernels execute it: pivot det 3, rsqrt 1,
    inverse 4, tau 1, W = B Q 12 r, rank-2 update 4 r (2r + 1), plus one add per leaf
    (tends to 50 flops per subset)."""
    tot = float(1 << n)
    for k in range(n):
        r = n - 1 - k
        tot += (1 << k) * (8 * r * r + 16 * r + 9)
    return tot


def approx_unit_flops(n: int, j: int) -> float:
    """Algorithmic real flops of one (pattern, nu) unit of the approximation: the
    sweep-operator inverse of the 2n x 2n complex symmetric I - t O_S (2n pivots, each a
    complex multiply and multiply-subtract on (2n)^2 / 2 entries: 14 flops) and the group
    minors det(G_WW)^{-1/2} for every |W| <= j (LDL^T with complex pivots and inverse
    square roots: 60, 240 and 300 flops for w = 1, 2, 3; w = 4 reuses its triple's
    factors through a 2x2 Schur block: 100)."""
    N = 2 * n
    f = 14.0 * N * N * N / 2
    per = {1: 60, 2: 240, 3: 300, 4: 100}
    for w in range(1, j + 1):
        f += math.comb(n, w) * per[w]
    return f


def adjoint_flops(n: int) -> float:
    """Algorithmic flops of the exact adjoint Gbar = dT/dA_S in reverse mode through
    the Schur recursion: the forward recursion F(n) (schur_flops) and its reverse, 3 F(n)
    (per include step Z = B Gamma costs 4 flops per trailing entry against the forward
    update's 2, plus the rest-block combination)."""
    return 4.0 * schur_flops(n)


def workload(name: str, rank: int, world: int):
    c = g.CONFIGS[name]
    U, r = c.unitary(), c.squeezing()
    # weak scaling: rank k evaluates its own batch (pattern counters k*n_pat ...)
    allp = g.gen_patterns(c.seed, c.M, c.n_lo, c.n_hi, c.n_pat * world) if world > 1 else c.patterns()
    pats = allp[rank * c.n_pat:(rank + 1) * c.n_pat]
    n = np.array([len(g.pattern_modes(p)) for p in pats])
    return c, U, r, pats, n


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest x over the ranks (the timed region ends with the slowest rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def sum_over_ranks(x: float, world: int, device) -> float:
    """The total of x over the ranks (each rank evaluates its own patterns)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.item()


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def oracle_rate(U, r, eta, pats, n, budget_s: float = 12.0, start: int = 0):
    """The double-double oracle as it stands on this host's cores: patterns taken in
    batch order from `start` (wrapping), each one's 2^n subsets split into mask ranges
    over every core, until the time budget is used.  Returns (subsets/s, detail)."""
    import oracle
    st = oracle.build_state(U, r, eta)
    nt = oracle.max_threads()
    t0 = time.perf_counter()
    done, subsets = 0, 0
    while done < len(pats) and time.perf_counter() - t0 < budget_s:
        i = (start + done) % len(pats)
        oracle.subset_sum(st.A, st.M, g.pattern_modes(pats[i]), nchunk=4 * nt, dd=True)
        subsets += 1 << int(n[i])
        done += 1
    el = time.perf_counter() - t0
    return subsets / el, dict(cores=nt, patterns=done, subsets=subsets, seconds=el)


def cpu_baseline(U, r, eta, pats, n, budget_s: float = 12.0):
    """The oracle on the host cores, on a bounded sample of the workload (the
    double-double oracle: on these improbable patterns it is the CPU code that meets
    1e-10 in log P, like the GPU path it is compared with)."""
    val, d = oracle_rate(U, r, eta, pats, n, budget_s)
    return dict(value=val, unit=UNIT, cores=d["cores"], kind="oracle",
                sample="double-double oracle, the first %d of %d patterns in batch order (%d subsets, "
                       "mask ranges over %d threads) in %.1f s" % (d["patterns"], len(pats), d["subsets"],
                                                                    d["cores"], d["seconds"]))


def run_reference(args):
    """The oracle on the host cores: each step evaluates the next `per_step` patterns of
    the batch (rotating) with the double-double oracle, every pattern's subsets split
    into mask ranges over all cores.  Rank 0 alone runs it."""
    world, rank, local = dist_setup()
    if rank != 0:
        return 0
    c, U, r, pats, n = workload(args.workload, 0, 1)
    import oracle
    st = oracle.build_state(U, r, c.eta)
    nt = oracle.max_threads()
    per_step = 1

    def step(i):
        tot = 0
        for j in range(per_step):
            k = (i * per_step + j) % len(pats)
            oracle.subset_sum(st.A, st.M, g.pattern_modes(pats[k]), nchunk=4 * nt, dd=True)
            tot += 1 << int(n[k])
        return tot
    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    subsets = sum(step(args.warmup + i) for i in range(args.steps))
    el = time.perf_counter() - t0
    val = subsets / el
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64x2",
            "data": "synthetic", "config": {"workload": c.name, "M": c.M, "n_pat_per_step": per_step,
                                            "clicks": [c.n_lo, c.n_hi], "eta": c.eta,
                                            "oracle": "double-double (1e-10 in log P on this workload)"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": nt, "kind": "oracle",
                             "sample": "%d patterns per step, rotating through the %d-pattern batch; each "
                                       "pattern's subsets in mask ranges over %d threads"
                                       % (per_step, len(pats), nt)},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def write_detail(args, detail):
    """The long per-workload study goes to a side file; the headline line stays short."""
    path = args.detail_out
    try:
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        with open(path, "w") as f:
            json.dump(detail, f, indent=1, default=float)
        return os.path.relpath(os.path.abspath(path), ROOT)
    except OSError as e:
        return "not written: %s" % e


def compact(x, digits=5):
    """Round floats for the headline line (keeps it short)."""
    if isinstance(x, float):
        return float("%.*g" % (digits, x)) if math.isfinite(x) else None
    if isinstance(x, dict):
        return {k: compact(v, digits) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [compact(v, digits) for v in x]
    return x


def run_gpu(args):
    import torch
    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2106_01445_gb300 import build as b
    if rank == 0:
        b.build()
    if world > 1:
        dist.barrier()
    from paper_2106_01445_gb300.api import Context, patterns_tensor, _complex_interleaved

    c, U, r, pats, n = workload(args.workload, rank, world)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    ctx = Context(local, stream)
    # the autotuner picks the work split of the headline precision on this batch, then
    # the reservation sizes the workspace for it (no allocation or sync in the steps)
    st0 = ctx.build_state(U, r, c.eta)
    tuned = {}
    for pk in ("fx", "dd", "fp64", "fp32"):
        sp, tms = ctx.autotune(st0["O"], st0["logdet"], pats, precision=pk)
        tuned[pk] = {"split": sp, "sweep_ms": tms}
    ctx.reserve(len(pats), int(n.max()))
    Ud = _complex_interleaved(U, dev)
    rd = torch.as_tensor(r, device=dev)
    pd = patterns_tensor(pats, dev)
    M = c.M
    O = torch.empty((2 * M, 2 * M), dtype=torch.float64, device=dev)
    logdet = torch.empty(1, dtype=torch.float64, device=dev)
    sst = torch.zeros(1, dtype=torch.int32, device=dev)
    out = {k: torch.empty(len(pats), dtype=torch.float64, device=dev) for k in ("logP", "kappa", "err_bound")}
    out["status"] = torch.empty(len(pats), dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step(prec):
        ctx.build_state_into(Ud, rd, c.eta, O, logdet, sst)
        ctx.prob(O, logdet, pd, order=0, precision=prec, out=out)

    subsets = float(sum(2.0 ** k for k in n))
    subsets_all = sum_over_ranks(subsets, world, dev)   # the whole job's units per step
    flops = float(sum(schur_flops(int(k)) for k in n))
    flops_exec = float(sum(schur_flops_executed(int(k)) for k in n))
    prec = args.precision

    def timed(prec, K, W, clocks=None):
        for _ in range(W):
            step(prec)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ctx.timing(True)
        ctx.timing_read(reset=True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        if clocks:
            clocks.start()
            time.sleep(0.3)
        torch.cuda.synchronize()
        for i in range(K):
            ev[i][0].record(stream)
            step(prec)
            ev[i][1].record(stream)
            flush.fill_(float(i))           # L2 flush between timed steps (not timed)
        torch.cuda.synchronize()
        ck = clocks.stop() if clocks else None
        ms = sum(a.elapsed_time(bb) for a, bb in ev)
        sweep_ms, launches = ctx.timing_read(reset=True)
        ctx.timing(False)
        ms = max_over_ranks(ms, world, dev)
        return ms, sweep_ms, launches, ck

    clocks = ClockSampler(local)
    ms, sweep_ms, launches, ck = timed(prec, args.steps, args.warmup, clocks)
    res_main = None
    step(prec)
    torch.cuda.synchronize()
    res_main = {k: v.cpu().numpy().copy() for k, v in out.items()}
    # the other precisions, for the comparison (shorter runs)
    others = {}
    if args.compare:
        for other in ("fx", "dd", "fp64", "fp32"):
            if other == prec:
                continue
            Ko = max(3, args.steps // 20)
            ms_o, sweep_o, launches_o, _ = timed(other, Ko, 2)
            step(other)
            torch.cuda.synchronize()
            others[other] = dict(ms_per_step=ms_o / Ko, kernel_ms=sweep_o / max(launches_o, 1),
                                 value=subsets_all * Ko / (ms_o * 1e-3),
                                 logP=out["logP"].cpu().numpy().copy(),
                                 status=out["status"].cpu().numpy().copy())
    value = subsets_all * args.steps / (ms * 1e-3)

    # end to end through the public host-buffer entry point (copies inside the region),
    # every rank at once: the whole job's subsets over the slowest rank's time
    K2 = max(3, min(args.steps, 50))
    for _ in range(2):
        ctx.run_host(U, r, c.eta, pats, precision=prec)
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(K2):
        ctx.run_host(U, r, c.eta, pats, precision=prec)
    el = max_over_ranks(time.perf_counter() - t0, world, dev)
    e2e = {"value": subsets_all * K2 / el, "unit": UNIT,
           "h2d_bytes_per_step": 16 * M * M + 8 * M + 16 * len(pats),
           "d2h_bytes_per_step": len(pats) * (8 + 8 + 8 + 4) + 4}
    if rank != 0:
        return 0
    # roofline of the dominant kernel (the subset sweep): plain ALU pipes, no tensor
    # cores, no DRAM traffic to speak of.  FP32: algorithmic flops against SMs x 128
    # lanes x 2 x max clock.  FP64: against the measured FP64 FMA loop.  Double-double
    # and fixed point: against the measured loop of the sweep's own update entry in that
    # arithmetic (4 flops per entry), i.e. the rate the sweep would reach if every
    # algorithmic flop cost what its main update costs.
    props = torch.cuda.get_device_properties(dev)
    smax = (ck or {}).get("sm_max_mhz") or 2070.0
    fp32_peak = props.multi_processor_count * 128 * 2 * smax * 1e6
    meas = {k: ctx.peak_flops(k) for k in ("fp32", "fp64", "dd", "fx", "imad")}
    all_peaks = {"fp32": fp32_peak, "fp64": meas["fp64"], "dd": meas["dd"], "fx": meas["fx"]}
    peak = all_peaks[prec]
    kms = sweep_ms / max(launches, 1)
    achieved = flops / (kms * 1e-3)
    kname = {"fp32": "float", "fp64": "double", "dd": "dd", "fx": "fx"}[prec]
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": DRAM_TRAFFIC.get(prec),
                "kernel": "sweep_kernel<%s>" % kname, "kernel_ms": kms, "flops_per_launch": flops,
                "flop_count": "8r^2+10r+10 per include step (44/subset)",
                "frac_executed_count": flops_exec / (kms * 1e-3) / peak,
                "peak_basis": {"fp32": "SMs x 128 FP32 lanes x 2 x max SM clock (derived)",
                               "fp64": "measured FP64 FMA loop",
                               "dd": "measured loop of the sweep's double-double update entry, 4 flops",
                               "fx": "measured loop of the sweep's fixed-point update entry, 4 flops"}[prec]}
    if prec == "fx":
        # the integer pipe: each fixed-point update entry is two truncated 128-bit products of
        # 23 IMAD each (FX_IMAD_PER_ENTRY); at the measured IMAD issue rate that bounds the
        # entry rate, and so the sweep's flops, from above
        imad_bound = meas["imad"] / FX_IMAD_PER_ENTRY * 4.0
        roofline["int_pipe"] = {"imad_per_s": meas["imad"], "imad_per_entry": FX_IMAD_PER_ENTRY,
                                "entry_loop_frac_of_imad_bound": meas["fx"] / imad_bound,
                                "frac_of_imad_bound": achieved / imad_bound}
    # oracle on the host cores: baseline, and the stated error of every precision
    # against the double-double oracle on a sample
    cb = cpu_baseline(U, r, c.eta, pats, n, budget_s=args.cpu_budget)
    import oracle
    sample = np.nonzero(n <= args.dd_sample_nmax)[0][: args.dd_sample]
    ref = oracle.prob_exact(oracle.build_state(U, r, c.eta), pats[sample], dd=True)["logP"]
    errs = {}
    allres = dict(others)
    allres[prec] = dict(logP=res_main["logP"], status=res_main["status"])
    for pk, rv in allres.items():
        lp, stt = rv["logP"][sample], rv["status"][sample]
        okm = stt == 0
        d = np.abs(lp[okm] - ref[okm])
        errs[pk] = {"max_abs_dlogP": float(d.max()) if d.size else None,
                    "median_abs_dlogP": float(np.median(d)) if d.size else None,
                    "status_ok_fraction_all_patterns": float((rv["status"] == 0).mean())}
    other_prec = {}
    for k, v in others.items():
        ach = flops / (v["kernel_ms"] * 1e-3)
        other_prec[k] = {kk: vv for kk, vv in v.items() if kk not in ("logP", "status")}
        other_prec[k]["roofline"] = {"achieved_tflops": ach / 1e12, "peak_tflops": all_peaks[k] / 1e12,
                                     "frac": ach / all_peaks[k]}
        other_prec[k]["max_abs_dlogP_vs_dd_oracle"] = errs[k]["max_abs_dlogP"]
    detail = {"workload": c.name, "autotune": tuned, "other_precisions": other_prec,
              "loop_measured_tflops": {k: v / 1e12 for k, v in meas.items()},
              "error_vs_oracle": {"reference": "double-double oracle", "patterns_checked": int(sample.size),
                                  "clicks_checked": [int(n[sample].min()), int(n[sample].max())]
                                  if sample.size else None, "per_precision": errs}}
    if args.workloads == "all":
        detail["workloads"] = run_workloads(dev, stream, meas, fp32_peak)
    detail["note"] = ("other_precisions: the same batch with the other sweeps; workloads: one pass of "
                      "the other workloads (timings, rooflines, accuracy against the oracle)")
    where = write_detail(args, detail)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "fp64": "f64", "dd": "f64x2", "fx": "i128"}[prec],
            "data": "synthetic",
            "config": {"workload": c.name, "M": c.M, "squeezed": c.K, "eta": c.eta, "n_pat": len(pats),
                       "clicks": [c.n_lo, c.n_hi], "subsets_per_step": subsets_all, "precision": prec,
                       "l2": "flushed between timed steps (512 MB write)"},
            "patterns_per_s": len(pats) * world * args.steps / (ms * 1e-3),
            "gpu_launches": 4 * args.steps,
            "max_abs_dlogP_vs_dd_oracle": errs[prec]["max_abs_dlogP"],
            "roofline": roofline, "cpu_baseline": cb, "e2e": e2e, "clocks": ck,
            "other_precisions_subsets_per_s": {k: v["value"] for k, v in others.items()},
            "detail": where}
    print(json.dumps(compact(line)), flush=True)
    return 0


def run_workloads(dev, stream, meas, fp32_peak):
    """The other four workloads, one pass each (one GPU): timings with CUDA events on the
    library's stream, the dominant kernel's roofline, accuracy against the oracle on a
    bounded sample, and the approximation against the exact sum where the exact sum is
    run (reported, not gated).  A context of its own (no reservation: workspaces grow)."""
    import torch
    import oracle
    from oracle import approx as oap
    from oracle import grad as ograd
    from paper_2106_01445_gb300.api import Context, LogProbClements, patterns_tensor
    ctx = Context(dev.index, stream)

    def timed(fn, reps=1):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ctx.timing(True)
        ctx.timing_read(reset=True)
        e0.record(stream)
        for _ in range(reps):
            r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        kms, launches = ctx.timing_read(reset=True)
        ctx.timing(False)
        return e0.elapsed_time(e1) / reps, kms / max(launches, 1), r

    def host(out):
        return {k: v.cpu().numpy() for k, v in out.items()}

    def nclicks(pats):
        return np.array([len(g.pattern_modes(p)) for p in pats])

    res = {}
    # ---- the 24-mode batch split into N equal-cost slices (the multi-GPU strong-scaling
    # partition), run one after another on this GPU: each slice's sweep time, the balance
    # (slowest / mean: what N GPUs would wait for) and the combine, against the whole batch
    c = g.CONFIGS["m24_exact"]
    st = ctx.build_state(c.unitary(), c.squeezing(), c.eta)
    pd = patterns_tensor(c.patterns(), dev)
    ms_whole, kms_whole, whole = timed(lambda: ctx.prob(st["O"], st["logdet"], pd, precision="fx"))
    split = {"whole_batch_sweep_ms": kms_whole}
    for N in (2, 4, 8):
        parts, flags, kms = [], [], []
        for k in range(N):
            _, kk, (pp, ff) = timed(lambda: ctx.prob_partial(st["O"], pd, k, N, precision="fx"))
            parts.append(pp)
            flags.append(ff)
            kms.append(kk)
        ms_c, _, comb = timed(lambda: ctx.prob_combine(st["logdet"], pd, torch.stack(parts), torch.stack(flags),
                                                       precision="fx"))
        a, b = host(comb), host(whole)
        ok = b["status"] == 0
        split["slices_%d" % N] = {"slice_sweep_ms": kms, "balance_max_over_mean": max(kms) / (sum(kms) / N),
                                  "sum_of_slices_over_whole": sum(kms) / kms_whole, "combine_ms": ms_c,
                                  "max_abs_dlogP_vs_whole": float(np.abs(a["logP"][ok] - b["logP"][ok]).max()),
                                  "status_equal": bool((a["status"] == b["status"]).all())}
    res["m24_split_slices"] = split

    # ---- 8 modes, all 256 patterns: latency of one call; sum of P; every pattern vs the oracle
    c = g.CONFIGS["m8_all"]
    U, r, pats = c.unitary(), c.squeezing(), c.patterns()
    st = ctx.build_state(U, r, c.eta)
    pd = patterns_tensor(pats, dev)
    ref = oracle.prob_exact(oracle.build_state(U, r, c.eta), pats, dd=True)["logP"]
    e = {}
    for prec in ("fx", "fp64"):
        ms, _, out = timed(lambda: ctx.prob(st["O"], st["logdet"], pd, precision=prec), reps=20)
        lp = host(out)["logP"]
        e[prec] = {"ms_per_call": ms, "sum_P_minus_1": float(np.exp(lp).sum() - 1.0),
                   "max_abs_dlogP_vs_dd_oracle": float(np.abs(lp - ref).max())}
    res["m8_all"] = {"patterns": len(pats), "subsets": 3 ** 8, **e}

    # ---- 50 modes, 4096 patterns n = 10..40: approximation orders 2..4; exact on n <= 22
    c = g.CONFIGS["m50_approx"]
    U, r, pats = c.unitary(), c.squeezing(), c.patterns()
    n = nclicks(pats)
    st = ctx.build_state(U, r, c.eta)
    pd = patterns_tensor(pats, dev)
    exi = np.nonzero(n <= c.exact_n_max)[0]
    ms_ex, kms_ex, out = timed(lambda: ctx.prob(st["O"], st["logdet"], pd[torch.as_tensor(exi, device=dev)],
                                                precision="fx"))
    ex = host(out)
    sub_ex = float(sum(2.0 ** k for k in n[exi]))
    entry = {"patterns": len(pats), "exact_fx_on_n_le_%d" % c.exact_n_max: {
        "patterns": int(exi.size), "ms": ms_ex, "subsets_per_s": sub_ex / (ms_ex * 1e-3),
        "status_ok_fraction": float((ex["status"] == 0).mean())}}
    st_or = oracle.build_state(U, r, c.eta)
    small = [i for i in np.argsort(n, kind="stable") if n[i] <= 12][:2]
    for order in (2, 3, 4):
        for prec in (("fp32", "ff", "fp64") if order == 2 else ("fp32", "ff")):
            ms, kms, out = timed(lambda: ctx.prob(st["O"], st["logdet"], pd, order=order, precision=prec))
            a = host(out)
            units = (a["kappa"].astype(np.int64) + 1) // 2 + 1
            fl = float(sum(u * approx_unit_flops(int(k), order) for u, k in zip(units, n)))
            # float-float: algorithmic flops against the FP32 peak (its own cost per flop
            # is the price of the precision)
            peak = meas["fp64"] if prec == "fp64" else fp32_peak
            ok = (ex["status"] == 0) & np.isin(a["status"][exi], (0, 7))
            rel = np.abs(np.expm1(a["logP"][exi][ok] - ex["logP"][ok]))
            orc = []
            for i in small:
                lp_o, _ = oap.approx_logprob(st_or.O, st_or.logdet, c.M, g.pattern_modes(pats[i]), order)
                orc.append(abs(a["logP"][i] - lp_o))
            entry["order%d_%s" % (order, prec)] = {
                "ms": ms, "patterns_per_s": len(pats) / (ms * 1e-3),
                "status_ok_fraction": float((a["status"] == 0).mean()),
                "fit_fallback_fraction": float((a["status"] == 7).mean()),
                "below_fp32_floor_fraction": float((a["status"] == 9).mean()),
                "roofline_minors": {"bound": "alu", "kernel": "approx_minors_kernel<%s>" % (
                    {"fp32": "float", "ff": "ff", "fp64": "double"}[prec]), "kernel_ms": kms, "flops": fl,
                    "achieved_tflops": fl / (kms * 1e-3) / 1e12, "peak_tflops": peak / 1e12,
                    "frac": fl / (kms * 1e-3) / peak},
                "vs_exact_n_le_%d" % c.exact_n_max: {"median_rel_dP": float(np.median(rel)),
                                                     "max_rel_dP": float(rel.max())},
                "max_abs_dlogP_vs_oracle_approx": float(max(orc)), "oracle_patterns_n": [int(n[i]) for i in small]}
    res["m50_approx"] = entry

    # ---- 32-mode Clements mesh, 512 patterns n = 8..16: log P and its gradient
    c = g.CONFIGS["m32_grad"]
    th, ph = g.clements_phases(c.M, c.seed)
    r, pats = c.squeezing(), c.patterns()
    n = nclicks(pats)
    pd = patterns_tensor(pats, dev)
    rt = torch.tensor(r, device=dev, requires_grad=True)
    et = torch.tensor(c.eta, dtype=torch.float64, device=dev, requires_grad=True)
    tt = torch.tensor(th, device=dev, requires_grad=True)
    pt = torch.tensor(ph, device=dev, requires_grad=True)
    wts = torch.linspace(-1.0, 1.0, len(pats), dtype=torch.float64, device=dev)

    def step():
        lp = LogProbClements.apply(rt, et, tt, pt, pd, ctx)
        return torch.autograd.grad((wts * lp).sum(), (rt, et, tt, pt))

    step()
    ms, _, _ = timed(step, reps=3)
    Ud = ctx.clements_unitary(torch.as_tensor(th, device=dev), torch.as_tensor(ph, device=dev), c.M)
    st = ctx.build_state(torch.view_as_complex(Ud.view(c.M, c.M, 2)), torch.as_tensor(r, device=dev), c.eta)
    ms_adj, kms_adj, (dsq, _, _) = timed(lambda: ctx.grad(st["O"], st["logdet"], pd, wts))
    fl = float(sum(adjoint_flops(int(k)) for k in n))
    chk = [i for i in np.argsort(n, kind="stable")][:2]
    U = g.clements_unitary(c.M, th, ph)
    st_or = oracle.build_state(U, r, c.eta)
    ds_gpu = ctx.grad(st["O"], st["logdet"], pd[torch.as_tensor(chk, device=dev)],
                      torch.ones(len(chk), dtype=torch.float64, device=dev))[0].cpu().numpy()
    ds_orc = ograd.grad_sigmaQ(st_or, pats[chk], np.ones(len(chk)))
    res["m32_grad"] = {"patterns": len(pats), "params": 2 * len(th) + c.M + 1,
                       "ms_forward_and_backward": ms, "patterns_per_s": len(pats) / (ms * 1e-3),
                       "roofline_adjoint": {"bound": "alu", "kernel": "grad_tree_kernel (double-double)",
                                            "kernel_ms": kms_adj, "flops": fl,
                                            "achieved_tflops": fl / (kms_adj * 1e-3) / 1e12,
                                            "peak_tflops": meas["dd"] / 1e12,
                                            "frac": fl / (kms_adj * 1e-3) / meas["dd"]},
                       "max_abs_d_dsigmaQ_vs_oracle": float(np.abs(ds_gpu - ds_orc).max()),
                       "oracle_patterns_n": [int(n[i]) for i in chk]}
    # the order-j approximation and its gradient (gbs_grad_approx, FP64 minors) on the same
    # device, through the mesh: all 512 patterns at order 2, the first 64 at order 4; the
    # gradient against the oracle's on the two smallest patterns.  An informational entry:
    # a failure here is reported in the line, not raised
    try:
        from paper_2106_01445_gb300.api import LogProbClementsApprox
        ap = {}
        for order, npat in ((2, len(pats)), (4, 64)):
            pdo, wo = pd[:npat], wts[:npat]

            def astep():
                lp = LogProbClementsApprox.apply(rt, et, tt, pt, pdo, ctx, order)
                return torch.autograd.grad((wo * lp).sum(), (rt, et, tt, pt))

            astep()
            ms_a, _, _ = timed(astep, reps=2)
            ap["order%d" % order] = {"patterns": npat, "ms_forward_and_backward": ms_a,
                                     "patterns_per_s": npat / (ms_a * 1e-3)}
        ones = torch.ones(len(chk), dtype=torch.float64, device=dev)
        ds_a = ctx.grad_approx(st["O"], st["logdet"], pd[torch.as_tensor(chk, device=dev)], ones, 4)[0]
        ds_ao, _ = ograd.grad_sigmaQ_approx(st_or, pats[chk], np.ones(len(chk)), 4)
        ap["max_abs_d_dsigmaQ_vs_oracle_order4"] = float(np.abs(ds_a.cpu().numpy() - ds_ao).max())
        ap["max_abs_dsigmaQ_order4"] = float(np.abs(ds_ao).max())
        res["m32_grad"]["approx_gradient"] = ap
    except Exception as e:
        res["m32_grad"]["approx_gradient"] = {"error": repr(e)[:300]}

    # ---- 100 modes: approximation on a slice of the 16384 patterns (n = 40..90); exact
    # fixed point on 8 of the 64 n = 30 anchors and the approximation against it
    c = g.CONFIGS["m100_approx"]
    U, r = c.unitary(), c.squeezing()
    pats = c.patterns()[:64]
    anc = c.anchor_patterns()[:8]
    n = nclicks(pats)
    st = ctx.build_state(U, r, c.eta)
    pd, ad = patterns_tensor(pats, dev), patterns_tensor(anc, dev)
    ms_a, kms_a, out = timed(lambda: ctx.prob(st["O"], st["logdet"], ad, precision="fx"))
    exa = host(out)
    # the anchors cancel by kappa ~1e27: beyond 128-bit fixed point, resolved by 192-bit
    ms_6, kms_6, out6 = timed(lambda: ctx.prob(st["O"], st["logdet"], ad, precision="fx192"))
    ex6 = host(out6)
    entry = {"slice_patterns": len(pats), "slice_clicks": [int(n.min()), int(n.max())],
             "anchors_exact_fx": {"anchors": len(anc), "clicks": c.anchor_n, "ms": ms_a,
                                  "subsets_per_s": len(anc) * 2.0 ** c.anchor_n / (ms_a * 1e-3),
                                  "status_ok_fraction": float((exa["status"] == 0).mean()),
                                  "max_err_bound": float(np.nanmax(exa["err_bound"]))},
             "anchors_exact_fx192": {"anchors": len(anc), "clicks": c.anchor_n, "ms": ms_6,
                                     "subsets_per_s": len(anc) * 2.0 ** c.anchor_n / (ms_6 * 1e-3),
                                     "status_ok_fraction": float((ex6["status"] == 0).mean()),
                                     "max_err_bound": float(np.nanmax(ex6["err_bound"])),
                                     "max_kappa": float(np.nanmax(ex6["kappa"])),
                                     "max_abs_dlogP_vs_fx": float(np.nanmax(np.abs(ex6["logP"] - exa["logP"])))}}
    exa = ex6   # the anchors' reference for the approximation below
    for order in (2, 3, 4):
        for prec in ("fp32", "auto"):
            ms, kms, out = timed(lambda: ctx.prob(st["O"], st["logdet"], pd, order=order, precision=prec))
            a = host(out)
            units = (a["kappa"].astype(np.int64) + 1) // 2 + 1
            fl = float(sum(u * approx_unit_flops(int(k), order) for u, k in zip(units, n)))
            e = {"ms": ms, "patterns_per_s": len(pats) / (ms * 1e-3),
                 "status_ok_fraction": float((a["status"] == 0).mean()),
                 "fit_fallback_fraction": float((a["status"] == 7).mean()),
                 "below_fp32_floor_fraction": float((a["status"] == 9).mean()),
                 "roofline_minors": {"bound": "alu", "kernel": "approx_minors_kernel<%s>%s" % (
                     "float" if prec == "fp32" else "ff", "" if prec == "fp32" else " and approx_minors_pair_kernel<ff>"),
                     "kernel_ms": kms, "flops": fl, "achieved_tflops": fl / (kms * 1e-3) / 1e12,
                     "peak_tflops": fp32_peak / 1e12, "frac": fl / (kms * 1e-3) / fp32_peak}}
            if prec == "auto":
                # the anchors against the exact sum: float-float minors (n = 30)
                aa = host(ctx.prob(st["O"], st["logdet"], ad, order=order, precision="ff"))
                ok = (exa["status"] == 0) & np.isin(aa["status"], (0, 7))
                rel = np.abs(np.expm1(aa["logP"][ok] - exa["logP"][ok]))
                e["anchors_ff_vs_exact"] = {"median_rel_dP": float(np.median(rel)), "max_rel_dP": float(rel.max())}
            entry["order%d_%s" % (order, "fp32" if prec == "fp32" else "auto_ff")] = e
    res["m100_approx"] = entry

    # ---- the paper's device shape (30 modes, 15 inputs squeezed r = 1.4, lossless): the
    # exact click-number distribution over all 2^30 subsets, and the all-click point by
    # orders 2-4 (float-float minors) against the exact sum
    c = g.CONFIGS["m30_device"]
    U, r = c.unitary(), c.squeezing()
    st = ctx.build_state(U, r, c.eta)
    ms, kms, (logp, kap) = timed(lambda: ctx.click_distribution(st["O"], st["logdet"]))
    pn = np.exp(logp.cpu().numpy())
    allp = g.modes_to_pattern(list(range(c.M)))[None]
    ex = host(ctx.prob(st["O"], st["logdet"], allp, precision="fx"))
    entry = {"M": c.M, "subsets": 2.0 ** c.M, "click_distribution_ms": ms, "sweep_kernel_ms": kms,
             "subsets_per_s": 2.0 ** c.M / (ms * 1e-3), "sum_p_minus_1": float(pn.sum() - 1.0),
             "p_n": [float(x) for x in pn], "kappa_max": float(np.nanmax(kap.cpu().numpy())),
             "all_click": {"exact_logP": float(ex["logP"][0]), "err_bound": float(ex["err_bound"][0])}}
    for order in (2, 3, 4):
        a = host(ctx.prob(st["O"], st["logdet"], allp, order=order, precision="ff"))
        entry["all_click"]["order%d_rel_dev" % order] = float(np.expm1(a["logP"][0] - ex["logP"][0]))
    # the photon-number sectors p_k(n) of the same device (lossless: even sectors only),
    # 256 circle points (65 complex float-float sweeps of 2^30 subsets; FP64 takes twice as long)
    ms, kms, pkn = timed(lambda: ctx.sector_distribution(st["O"], st["logdet"], L=256, rho=1.0, K=255,
                                                         even_only=True, precision="ff"))
    pkn = pkn.cpu().numpy()
    entry["sectors"] = {"L": 256, "sweeps": 65, "precision": "ff", "ms": ms, "sweep_kernel_ms_per_sweep": kms,
                        "subsets_per_s": 2.0 ** c.M / (kms * 1e-3),
                        "max_abs_sum_k_minus_p_n": float(np.abs(pkn.sum(axis=0) - pn).max()),
                        "max_abs_odd_sector": float(np.abs(pkn[1::2]).max()),
                        "p_k_n": {str(k): [float(x) for x in pkn[k]] for k in (20, 50, 80, 110, 140, 170)},
                        "peak_n": {str(k): int(np.argmax(pkn[k])) for k in (20, 50, 80, 110, 140, 170)}}
    # the approximation's fitted sector curves of the all-click pattern (the whole device)
    # against these exact sectors: the k = 110 curve and every sector's all-click point
    # (the paper's Fig. 3a and 3b)
    fig3 = {}
    main = pkn[110] > 1e-3 * pkn[110].max()
    w30 = pkn[:, c.M]
    big = w30 > 1e-3 * w30.max()
    for order in (2, 3, 4):
        cur, lp, _ = ctx.approx_sector_curves(st["O"], st["logdet"], allp, order=order, precision="ff", K=255)
        cur = cur.cpu().numpy()
        dev110 = np.abs(cur[110] / np.where(main, pkn[110], 1.0) - 1.0)[main]
        dev30 = np.abs(cur[big, c.M] / w30[big] - 1.0)
        fig3["order%d" % order] = {"k110_max_rel_dev_main_body": float(dev110.max()),
                                   "k110_rel_dev_at_n30": float(cur[110, c.M] / pkn[110, c.M] - 1.0),
                                   "k110_curve": [float(x) for x in cur[110]],
                                   "all_click_sectors_rel_dev_median": float(np.median(dev30)),
                                   "all_click_sectors_rel_dev_max": float(dev30.max()),
                                   "all_click_sum_rel_dev": float(cur[:, c.M].sum() / w30.sum() - 1.0)}
    entry["sectors"]["fit_vs_exact"] = fig3
    res["m30_device"] = entry

    # ---- the fourth-order accuracy study (the paper's Fig. 4): relative deviation of the
    # order-4 estimate (float-float minors) from the exact sum over 100 random outcomes per
    # point; the exact sum in fixed point, with double-double for patterns outside its range
    def study_point(c):
        U, r, pats = c.unitary(), c.squeezing(), c.patterns()
        st = ctx.build_state(U, r, c.eta)
        ex = host(ctx.prob(st["O"], st["logdet"], pats, precision="fx"))
        redo = np.nonzero(ex["status"] != 0)[0]
        if redo.size:
            ex2 = host(ctx.prob(st["O"], st["logdet"], pats[redo], precision="dd"))
            for kk in ex:
                ex[kk][redo] = ex2[kk]
        ap = host(ctx.prob(st["O"], st["logdet"], pats, order=4, precision="ff"))
        ok = (ex["status"] == 0) & (ap["status"] == 0)
        dev_ = np.abs(np.expm1(ap["logP"][ok] - ex["logP"][ok]))
        return {"M": c.M, "n": c.n_lo, "r": c.r_lo, "outcomes": int(len(pats)), "ok": int(ok.sum()),
                "mean_rel_dev": float(dev_.mean()), "std_rel_dev": float(dev_.std()),
                "median_rel_dev": float(np.median(dev_)), "max_rel_dev": float(dev_.max()),
                "fit_fallbacks": int((ap["status"] == 7).sum())}
    grid = g.accuracy_study()
    t0 = time.time()
    res["accuracy_study_order4"] = {"vs_m_r1.6": [study_point(c) for c in grid["vs_m"]],
                                    "vs_r_m30_n20": [study_point(c) for c in grid["vs_r"]]}
    res["accuracy_study_order4"]["wall_s"] = time.time() - t0
    ctx.close()
    return res


def run_m100(args):
    """The 100-mode workload's approximation at orders 2, 3 and 4 in the automatic
    precision (float-float minors; patterns above 79 clicks on CTA pairs) over its first
    --m100-npat patterns (all 16384 by default), one timed call per order (CUDA events on
    the library's stream); the fit-fallback fraction and the status counts per order.
    Written to the side file; the printed line is a summary."""
    import torch
    from paper_2106_01445_gb300 import build as b
    b.build()
    from paper_2106_01445_gb300.api import Context, patterns_tensor
    c = g.CONFIGS["m100_approx"]
    U, r = c.unitary(), c.squeezing()
    pats = c.patterns()[:args.m100_npat]
    n = np.array([len(g.pattern_modes(p)) for p in pats])
    ctx = Context(0)
    stream = torch.cuda.current_stream()
    st = ctx.build_state(U, r, c.eta)
    pd = patterns_tensor(pats, ctx.device)
    res = {"workload": c.name, "patterns": int(len(pats)), "clicks": [int(n.min()), int(n.max())],
           "patterns_above_79_clicks": int((n > 79).sum()), "precision": "auto (float-float minors)"}
    for order in args.m100_orders:
        torch.cuda.synchronize()
        ctx.timing(True)
        ctx.timing_read(reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = ctx.prob(st["O"], st["logdet"], pd, order=order, precision="auto")
        e1.record(stream)
        torch.cuda.synchronize()
        kms, nl = ctx.timing_read(reset=True)
        ctx.timing(False)
        stt = out["status"].cpu().numpy()
        lp = out["logP"].cpu().numpy()
        res["order%d" % order] = {"ms": e0.elapsed_time(e1), "minors_kernel_ms": kms,
                                  "patterns_per_s": len(pats) / (e0.elapsed_time(e1) * 1e-3),
                                  "status_counts": {str(k): int(v) for k, v in zip(*np.unique(stt, return_counts=True))},
                                  "fit_fallback_fraction": float((stt == 7).mean()),
                                  "fit_fallback_fraction_above_79": float((stt[n > 79] == 7).mean()) if (n > 79).any() else None,
                                  "finite_logP_fraction": float(np.isfinite(lp).mean())}
        print(json.dumps({"order": order, **res["order%d" % order]}), flush=True)
    args.detail_out = args.detail_out.replace("bench_detail", "bench_m100")
    where = write_detail(args, res)
    print(json.dumps({"m100": {k: v for k, v in res.items() if not k.startswith("order")}, "detail": where}))
    return 0


def run_profile_case(args):
    """One warm-up and one measured call of a kernel path, for ncu captures."""
    import torch
    from paper_2106_01445_gb300 import build as b
    b.build()
    from paper_2106_01445_gb300.api import Context
    if args.profile == "peak":
        ctx = Context(0)
        for k in ("fx", "imad", "fp64", "fp32", "dd"):
            print("peak loop %s: %.4g per s" % (k, ctx.peak_flops(k)))
        return 0
    if args.profile == "grad":
        c = g.CONFIGS["m32_grad"]
        ctx = Context(0)
        st = ctx.build_state(c.unitary(), c.squeezing(), c.eta)
        pats = c.patterns()
        w = torch.ones(len(pats), dtype=torch.float64, device="cuda")
        for _ in range(2):
            dsq, lp, stt = ctx.grad(st["O"], st["logdet"], pats, w)
        torch.cuda.synchronize()
        print("profile case grad: %d patterns, %d ok" % (len(pats), int((stt == 0).sum().item())))
        return 0
    c = g.CONFIGS[args.workload if args.profile == "sweep" else "m50_approx"]
    ctx = Context(0)
    st = ctx.build_state(c.unitary(), c.squeezing(), c.eta)
    pats = c.patterns() if args.profile == "sweep" else c.patterns()[:args.npat]
    order = 0 if args.profile == "sweep" else args.order
    out = ctx.prob(st["O"], st["logdet"], pats, order=order, precision=args.precision)
    torch.cuda.synchronize()
    ctx.timing(True)
    ctx.timing_read(reset=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    out = ctx.prob(st["O"], st["logdet"], pats, order=order, precision=args.precision)
    e1.record()
    torch.cuda.synchronize()
    kms, launches = ctx.timing_read(reset=True)
    print("profile case %s %s order %d: %d patterns, %d ok, %d fit fallbacks; call %.3f ms, timed kernel %.3f ms"
          % (args.profile, args.precision, order, len(pats), int((out["status"] == 0).sum().item()),
             int((out["status"] == 7).sum().item()), e0.elapsed_time(e1), kms / max(launches, 1)))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fx", choices=["fp32", "fp64", "dd", "fx", "ff", "fx192"],
                    help="ff (float-float minors) serves --profile approx only, fx192 --profile sweep only")
    ap.add_argument("--dd-sample", type=int, default=24)
    ap.add_argument("--dd-sample-nmax", type=int, default=15)
    ap.add_argument("--workload", default="m24_exact")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--profile", choices=["sweep", "approx", "grad", "peak"], default=None,
                    help="run one kernel path twice (for ncu) instead of the benchmark")
    ap.add_argument("--order", type=int, default=4)
    ap.add_argument("--workloads", choices=["all", "none", "m100"], default="all",
                    help="also run one pass of the other four workloads (on rank 0); m100: only the "
                         "100-mode approximation at orders 2-4 over --m100-npat patterns")
    ap.add_argument("--m100-npat", type=int, default=16384)
    ap.add_argument("--m100-orders", type=int, nargs="+", default=[2, 3, 4])
    ap.add_argument("--npat", type=int, default=128)
    ap.add_argument("--compare", type=int, default=1,
                    help="also time the other three precisions of the exact sweep (short runs)")
    ap.add_argument("--detail-out", default=os.path.join(ROOT, "bench_out", "bench_detail.json"),
                    help="side file for the per-workload study (the headline line stays short)")
    args = ap.parse_args()
    if args.profile:
        return run_profile_case(args)
    if args.workloads == "m100":
        return run_m100(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.precision in ("ff", "fx192"):
        ap.error("--precision %s serves --profile only (the benchmark times fx, dd, fp64 or fp32)" % args.precision)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
